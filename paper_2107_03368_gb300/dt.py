"""Python binding of libdt.so (include/dt.h): argument marshalling only.

Every function here converts torch tensors to raw pointers, calls the C
entry point of the same name and raises on a non-zero status.  All work runs
in the library's CUDA kernels; there is no CPU fallback — if libdt.so cannot
be built or loaded, importing this module fails.

Tensor conventions (torch has no unsigned 64/32/16-bit arithmetic, so the
unsigned C arrays are carried in signed tensors of the same width):
  descriptors  int64 [n, 64] CUDA tensor holding the uint64 words
  idx          int32 [nq, k]  (uint32 in C; 0xFFFFFFFF reads as -1)
  score        float32 [nq, k]
  ab           int16 [nq, k, 2]  (uint16 A, B)
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _build

_lib = None

DT_OK, DT_EINVAL, DT_ENOMEM, DT_ECUDA, DT_ETIMEOUT, DT_EUNSUPPORTED, DT_EIO = 0, -1, -2, -3, -4, -5, -6
DT_MAX_K = 32
WORDS = 64


class DtError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        lib = load()
        name = lib.dt_status_string(status).decode()
        msg = lib.dt_last_error().decode()
        super().__init__("%s failed: %s (%s)" % (where, name, msg))


class BuildParams(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int32), ("use_and_image", ctypes.c_int32),
                ("fused_cap", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class IndexInfo(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("depth", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("n", ctypes.c_int64), ("use_and_image", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class TuneReport(ctypes.Structure):
    _fields_ = [("tree_threads", ctypes.c_int32), ("tree_blocks_per_sm", ctypes.c_int32),
                ("popc_splits", ctypes.c_int32), ("tc_splits", ctypes.c_int32),
                ("tree_ms", ctypes.c_float), ("popc_ms", ctypes.c_float), ("tc_ms", ctypes.c_float),
                ("candidates_timed", ctypes.c_int32), ("tc_prewiden", ctypes.c_int32),
                ("tree_tc_splits", ctypes.c_int32), ("tree_tc_prewiden", ctypes.c_int32),
                ("tree_tc_ms", ctypes.c_float), ("retrieve_engine", ctypes.c_int32),
                ("retrieve_blocks_per_sm", ctypes.c_int32), ("retrieve_ms", ctypes.c_float)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("nodes_visited", ctypes.c_int64), ("leaves_visited", ctypes.c_int64),
                ("descs_scanned", ctypes.c_int64), ("bounds_evaluated", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def load():
    """Build (if stale) and load libdt.so; raises if that is impossible."""
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build_dt())
        P, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
        sig = {
            "dt_build": ([P, i64, P, P, P], ctypes.c_int),
            "dt_insert": ([P, P, i64, P], ctypes.c_int),
            "dt_keep_widened": ([P, i32, P], ctypes.c_int),
            "dt_save": ([P, ctypes.c_char_p], ctypes.c_int),
            "dt_load": ([ctypes.c_char_p, P, i64, P, P], ctypes.c_int),
            "quicci_generate": ([P, i64, P, i64, P, P, i64, ctypes.c_float, i32, P, P],
                                ctypes.c_int),
            "dt_get_info": ([P, P], ctypes.c_int),
            "dt_export": ([P, P, P, P, P, P, P, P], ctypes.c_int),
            "dt_search": ([P, P, i64, i32, P, P, P, P, P], ctypes.c_int),
            "dt_search_seeded": ([P, P, i64, i32, P, i32, P, P, P, P, P], ctypes.c_int),
            "dt_search_path": ([P, P, i64, i32, P, i32, P, P, P, P, i32, P], ctypes.c_int),
            "bf_search": ([P, i64, P, i64, i32, P, P, P, i32, P], ctypes.c_int),
            "bf_search_noalloc": ([P, i64, P, i64, i32, P, P, P, P], ctypes.c_int),
            "retrieve_objects": ([P, P, i32, P, P, i32, i64, i32, u64, P, P, P, i32, P],
                                 ctypes.c_int),
            "dt_sync_status": ([P], ctypes.c_int),
            "object_scores": ([P, i64, P, i32, P, P, i32, i64, P, P], ctypes.c_int),
            "dt_debug_fail_allocation": ([i32], None),
            "dt_kernel_timing": ([i32], ctypes.c_int),
            "dt_kernel_time": ([ctypes.c_char_p, P, P], ctypes.c_int),
            "dt_debug_inject_missing_copy": ([i32], None),
            "dt_autotune": ([P, P, i64, P, i64, i32, P, P], ctypes.c_int),
            "dt_autotune_retrieve": ([P, P, i32, P, P, i32, i64, i32, P, P], ctypes.c_int),
            "dt_tune_save": ([ctypes.c_char_p], ctypes.c_int),
            "dt_tune_load": ([ctypes.c_char_p], ctypes.c_int),
            "dt_tune_clear": ([], None),
            "dt_free": ([P], None),
            "dt_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "dt_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def _check(status, where):
    if status != DT_OK:
        raise DtError(status, where)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _desc(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int64
            and t.dim() == 2 and t.shape[1] == WORDS and t.is_contiguous()):
        raise ValueError("%s must be a contiguous CUDA int64 tensor of shape [n, 64]" % name)
    return t


class Index:
    """Owns a dt_index*; freed by free() or when garbage-collected."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("index has been freed")
        return self._h

    def info(self):
        inf = IndexInfo()
        _check(load().dt_get_info(self.handle, ctypes.byref(inf)), "dt_get_info")
        return {f: getattr(inf, f) for f, _ in IndexInfo._fields_ if f != "reserved"}

    def export(self, with_and=False):
        """Flattened tree as numpy arrays (child, begin, count, level, or_img, and_img, perm)."""
        import numpy as np
        inf = self.info()
        m, n = inf["n_nodes"], inf["n"]
        child = np.empty((m, 2), np.int64)
        begin = np.empty(m, np.int64)
        count = np.empty(m, np.int64)
        level = np.empty(m, np.int32)
        or_img = np.empty((m, WORDS), np.uint64)
        and_img = np.empty((m, WORDS), np.uint64) if with_and else None
        perm = np.empty(n, np.int64)
        p = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)
        _check(load().dt_export(self.handle, p(child), p(begin), p(count), p(level), p(or_img),
                                p(and_img), p(perm)), "dt_export")
        return dict(child=child, begin=begin, count=count, level=level, or_img=or_img,
                    and_img=and_img, perm=perm)

    def save(self, path):
        """Writes the tree (not the descriptors) to `path` (dt_save)."""
        _check(load().dt_save(self.handle, os.fsencode(path)), "dt_save")

    def free(self):
        if self._h is not None:
            load().dt_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def dt_build(db, leaf_size=32, use_and_image=False, fused_cap=0, stream=None) -> Index:
    db = _desc(db, "db")
    params = BuildParams(leaf_size, 1 if use_and_image else 0, fused_cap, 0)
    out = ctypes.c_void_p()
    _check(load().dt_build(_ptr(db), db.shape[0], ctypes.byref(params), _stream(stream),
                           ctypes.byref(out)), "dt_build")
    return Index(out)


def dt_load(path, db, stream=None) -> Index:
    """Loads a tree written by Index.save over the database `db` [n, 64]
    (device; the rows it was built and grown over, in original-index order)."""
    db = _desc(db, "db")
    out = ctypes.c_void_p()
    _check(load().dt_load(os.fsencode(path), _ptr(db), db.shape[0], _stream(stream),
                          ctypes.byref(out)), "dt_load")
    return Index(out)


def dt_insert(index: Index, new, stream=None) -> Index:
    """Appends the descriptors ``new`` [m, 64] (device) to ``index`` in place;
    they take original indices n .. n+m-1.  Returns ``index``."""
    new = _desc(new, "new")
    _check(load().dt_insert(index.handle, _ptr(new), new.shape[0], _stream(stream)), "dt_insert")
    return index


def dt_keep_widened(index: Index, on: bool = True, stream=None) -> Index:
    """Keeps (or releases) the index's resident tensor-core copy of its rows
    (4 KB per descriptor), so batched searches skip widening them per call."""
    _check(load().dt_keep_widened(index.handle, 1 if on else 0, _stream(stream)), "dt_keep_widened")
    return index


def quicci(vertices, triangles, points, normals, support_radius=100.0, modified=False,
           out=None, stream=None):
    """QUICCI (or modified QUICCI) descriptors of oriented points on a mesh.
    vertices float32 [nv, 3], triangles int32 [nt, 3], points / normals
    float32 [n, 3] (contiguous CUDA tensors); returns int64 [n, 64]."""
    def f3(t, name, dtype):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.dim() == 2
                and t.shape[1] == 3 and t.is_contiguous()):
            raise ValueError("%s must be a contiguous CUDA %s tensor of shape [n, 3]" % (name, dtype))
        return t
    vertices = f3(vertices, "vertices", torch.float32)
    triangles = f3(triangles, "triangles", torch.int32)
    points, normals = f3(points, "points", torch.float32), f3(normals, "normals", torch.float32)
    if points.shape != normals.shape:
        raise ValueError("points and normals must have the same shape")
    if out is None:
        out = torch.empty((points.shape[0], WORDS), dtype=torch.int64, device=points.device)
    _check(load().quicci_generate(_ptr(vertices), vertices.shape[0], _ptr(triangles),
                                  triangles.shape[0], _ptr(points), _ptr(normals), points.shape[0],
                                  float(support_radius), 1 if modified else 0, _ptr(out),
                                  _stream(stream)), "quicci_generate")
    return out


def _outputs(nq, k, device, with_ab, out):
    if out is not None:
        return out
    idx = torch.empty((nq, k), dtype=torch.int32, device=device)
    score = torch.empty((nq, k), dtype=torch.float32, device=device)
    ab = torch.empty((nq, k, 2), dtype=torch.int16, device=device) if with_ab else None
    return idx, score, ab


def dt_search(index: Index, q, k, with_ab=False, stats=False, out=None, stream=None):
    """Returns (idx, score, ab or None, stats dict or None)."""
    q = _desc(q, "q")
    idx, score, ab = _outputs(q.shape[0], k, q.device, with_ab, out)
    st = Stats() if stats else None
    _check(load().dt_search(index.handle, _ptr(q), q.shape[0], k, _ptr(idx), _ptr(score),
                            _ptr(ab), ctypes.byref(st) if st is not None else None,
                            _stream(stream)), "dt_search")
    return idx, score, ab, (st.as_dict() if st is not None else None)


def dt_search_seeded(index: Index, q, k, seeds, with_ab=False, stats=False, out=None,
                     stream=None):
    """dt_search with a warm start from candidate indices seeds [nq, n_seed]
    (int32/uint32 device tensor, -1 = none).  Same results as dt_search."""
    q = _desc(q, "q")
    if seeds.dim() != 2 or seeds.shape[0] != q.shape[0]:
        raise ValueError("seeds must be [nq, n_seed]")
    if seeds.dtype not in (torch.int32, torch.uint32) or not seeds.is_contiguous():
        raise ValueError("seeds must be a contiguous int32 tensor")
    if seeds.device != q.device:
        raise ValueError("seeds must be on the queries' device")
    idx, score, ab = _outputs(q.shape[0], k, q.device, with_ab, out)
    st = Stats() if stats else None
    _check(load().dt_search_seeded(index.handle, _ptr(q), q.shape[0], k, _ptr(seeds),
                                   seeds.shape[1], _ptr(idx), _ptr(score), _ptr(ab),
                                   ctypes.byref(st) if st is not None else None,
                                   _stream(stream)), "dt_search_seeded")
    return idx, score, ab, (st.as_dict() if st is not None else None)


def dt_search_path(index: Index, q, k, path, seeds=None, with_ab=False, stats=False, out=None,
                   stream=None):
    """dt_search (seeds None) or dt_search_seeded with the traversal forced:
    path 0 automatic, 1 per query, 2 batched.  Same results on every path."""
    q = _desc(q, "q")
    n_seed = 0
    if seeds is not None:
        if seeds.dim() != 2 or seeds.shape[0] != q.shape[0]:
            raise ValueError("seeds must be [nq, n_seed]")
        if seeds.dtype not in (torch.int32, torch.uint32) or not seeds.is_contiguous():
            raise ValueError("seeds must be a contiguous int32 tensor")
        n_seed = seeds.shape[1]
    idx, score, ab = _outputs(q.shape[0], k, q.device, with_ab, out)
    st = Stats() if stats else None
    _check(load().dt_search_path(index.handle, _ptr(q), q.shape[0], k,
                                 _ptr(seeds) if n_seed else None, n_seed, _ptr(idx), _ptr(score),
                                 _ptr(ab), ctypes.byref(st) if st is not None else None, path,
                                 _stream(stream)), "dt_search_path")
    return idx, score, ab, (st.as_dict() if st is not None else None)


def bf_search(db, q, k, with_ab=False, path=0, out=None, stream=None):
    """Returns (idx, score, ab or None)."""
    db, q = _desc(db, "db"), _desc(q, "q")
    idx, score, ab = _outputs(q.shape[0], k, q.device, with_ab, out)
    _check(load().bf_search(_ptr(db), db.shape[0], _ptr(q), q.shape[0], k, _ptr(idx),
                            _ptr(score), _ptr(ab), path, _stream(stream)), "bf_search")
    return idx, score, ab


def bf_search_noalloc(db, q, k, out, stream=None):
    """bf_search that allocates nothing, neither in the library nor here: the
    caller provides out = (idx, score, ab or None).  For callers that must
    not have device memory allocated behind their back (a fixed per-process
    memory plan, an external arena); limit nq * k <= 2,097,152."""
    db, q = _desc(db, "db"), _desc(q, "q")
    idx, score, ab = out
    _check(load().bf_search_noalloc(_ptr(db), db.shape[0], _ptr(q), q.shape[0], k, _ptr(idx),
                                    _ptr(score), _ptr(ab), _stream(stream)), "bf_search_noalloc")
    return idx, score, ab


def retrieve_objects(index: Index, object_of, n_objects, qdesc, qoffsets, vote_threshold=0,
                     seed=0, with_consumed=True, engine=0, out=None, stream=None):
    """Returns (votes int32 [nq, n_objects] (uint32 counts), winner int32 [nq],
    consumed int64 [nq] or None).  engine: 0 auto, 1 tree traversal per
    descriptor, 2 tensor-core scan, 3 batched tree search (identical results)."""
    qdesc = _desc(qdesc, "qdesc")
    if not (object_of.is_cuda and object_of.dtype == torch.int32 and object_of.is_contiguous()):
        raise ValueError("object_of must be a contiguous CUDA int32 tensor")
    if not (qoffsets.is_cuda and qoffsets.dtype == torch.int64 and qoffsets.is_contiguous()):
        raise ValueError("qoffsets must be a contiguous CUDA int64 tensor")
    nq = qoffsets.shape[0] - 1
    dev = qdesc.device
    if out is None:
        votes = torch.empty((nq, n_objects), dtype=torch.int32, device=dev)
        winner = torch.empty(nq, dtype=torch.int32, device=dev)
        consumed = torch.empty(nq, dtype=torch.int64, device=dev) if with_consumed else None
    else:
        votes, winner, consumed = out
    _check(load().retrieve_objects(index.handle, _ptr(object_of), n_objects, _ptr(qdesc),
                                   _ptr(qoffsets), nq, qdesc.shape[0], vote_threshold,
                                   ctypes.c_uint64(seed), _ptr(votes), _ptr(winner),
                                   _ptr(consumed), engine, _stream(stream)),
           "retrieve_objects")
    return votes, winner, consumed


def dt_autotune(index=None, db=None, q=None, k=10, stream=None):
    """Time launch shapes on these inputs and remember the fastest (returns the report)."""
    q = _desc(q, "q")
    if db is not None:
        db = _desc(db, "db")
    rep = TuneReport()
    _check(load().dt_autotune(index.handle if index is not None else None, _ptr(db),
                              db.shape[0] if db is not None else 0, _ptr(q), q.shape[0], k,
                              _stream(stream), ctypes.byref(rep)), "dt_autotune")
    return rep.as_dict()


def dt_autotune_retrieve(index: Index, object_of, n_objects, qdesc, qoffsets, vote_threshold=0,
                         stream=None):
    """Time retrieve_objects' engines on these partial queries (a sample of
    the workload) and remember the fastest for engine 0 (returns the report)."""
    qdesc = _desc(qdesc, "qdesc")
    rep = TuneReport()
    _check(load().dt_autotune_retrieve(index.handle, _ptr(object_of), n_objects, _ptr(qdesc),
                                       _ptr(qoffsets), qoffsets.shape[0] - 1, qdesc.shape[0],
                                       vote_threshold, _stream(stream), ctypes.byref(rep)),
           "dt_autotune_retrieve")
    return rep.as_dict()


def dt_tune_save(path):
    _check(load().dt_tune_save(str(path).encode()), "dt_tune_save")


def dt_tune_load(path):
    n = load().dt_tune_load(str(path).encode())
    if n < 0:
        raise DtError(n, "dt_tune_load")
    return n


def dt_tune_clear():
    load().dt_tune_clear()


def dt_sync_status(stream=None):
    _check(load().dt_sync_status(_stream(stream)), "dt_sync_status")


def object_scores(db, object_of, n_objects, qdesc, qoffsets, stream=None):
    """float64 [nq, n_objects]: per query object and database object, the sum
    of its descriptors' distances to their nearest descriptor of the object."""
    db, qdesc = _desc(db, "db"), _desc(qdesc, "qdesc")
    if not (object_of.is_cuda and object_of.dtype == torch.int32 and object_of.is_contiguous()):
        raise ValueError("object_of must be a contiguous CUDA int32 tensor")
    if not (qoffsets.is_cuda and qoffsets.dtype == torch.int64 and qoffsets.is_contiguous()):
        raise ValueError("qoffsets must be a contiguous CUDA int64 tensor")
    nq = qoffsets.shape[0] - 1
    out = torch.empty((nq, n_objects), dtype=torch.float64, device=db.device)
    _check(load().object_scores(_ptr(db), db.shape[0], _ptr(object_of), n_objects, _ptr(qdesc),
                                _ptr(qoffsets), nq, qdesc.shape[0], _ptr(out), _stream(stream)),
           "object_scores")
    return out


def dt_kernel_timing(on):
    """Clear the kernel timing totals and switch timing on or off."""
    _check(load().dt_kernel_timing(1 if on else 0), "dt_kernel_timing")


def dt_kernel_time(name):
    """(total milliseconds, launches) of the named kernel since timing was
    switched on (see include/dt.h for the names)."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(load().dt_kernel_time(name.encode(), ctypes.byref(ms), ctypes.byref(n)),
           "dt_kernel_time")
    return ms.value, n.value


def dt_debug_fail_allocation(nth):
    """Test hook: the nth scratch allocation from now fails (0 = off)."""
    load().dt_debug_fail_allocation(int(nth))


def dt_debug_inject_missing_copy(on):
    """Test hook: popcount brute-force launches lose one tile copy and time
    out (dt_sync_status then reports DT_ETIMEOUT) until switched off."""
    load().dt_debug_inject_missing_copy(1 if on else 0)


def dt_status_string(status):
    return load().dt_status_string(status).decode()


def dt_last_error():
    return load().dt_last_error().decode()
