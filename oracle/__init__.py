"""CPU oracle for the weighted-Hamming search path — TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It is a plain, slow, FP64 restatement of the
paper (arXiv 2107.03368) in C (``oracle.c``), loaded through ctypes; it shares
no code with the CUDA library and never calls it.

Functions and the passages they follow:
  wh_bytes / wh_bitwise / wh     Eq. 1 (§2.3) weighted Hamming distance
  bf_topk                        sequential search (§6.2), exact top-k
  build                          Dissimilarity Tree construction (§4.1)
  insert                         incremental insertion (§4.1, reading R14)
  quicci                         QUICCI and modified QUICCI generation (§2.2, §5, R15)
  node_bound                     node lower bound (§4.2)
  tree_search                    best-first Dissimilarity Tree query (§4.2)
  permutation / retrieve         voting pipeline (§3)
  object_scores                  object distance score (§6.4)

Every function is pinned by tests under ``tests/`` against closed forms,
invariants and brute force (see ``tests/test_oracle_*.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
SO = os.path.join(HERE, "liboracle.so")

WORDS = 64


def compile_library(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, OpenMP for query loops)."""
    if force or not os.path.exists(SO) or os.path.getmtime(SRC) > os.path.getmtime(SO):
        tmp = SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-o", tmp, SRC, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
        os.replace(tmp, SO)
    return SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(compile_library())
        P = ctypes.c_void_p
        i64, u64, i32, f64 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
        lib.orc_wh_bytes.argtypes = [P, P, ctypes.c_int, P, P]
        lib.orc_wh_bytes.restype = f64
        lib.orc_wh_bitwise.argtypes = [P, P, P, P]
        lib.orc_wh_bitwise.restype = f64
        lib.orc_wh.argtypes = [P, P, P, P]
        lib.orc_wh.restype = f64
        lib.orc_bf_topk.argtypes = [P, i64, P, i64, i32, P, P, P, i32]
        lib.orc_bf_topk.restype = None
        lib.orc_build.argtypes = [P, i64, i32, i32, i32, P, P, P, P, P, P, P]
        lib.orc_build.restype = i64
        lib.orc_insert.argtypes = [P, i64, i64, i32, i32, i64, P, P, P, P, P, P, P]
        lib.orc_insert.restype = i64
        lib.orc_quicci.argtypes = [P, i64, P, i64, P, P, i64, f64, i32, i32, P]
        lib.orc_quicci.restype = None
        lib.orc_node_bound.argtypes = [P, P, P]
        lib.orc_node_bound.restype = i64
        lib.orc_tree_search.argtypes = [P, i64, P, P, P, P, P, P, P, i64, i32, P, P, P, P, i32]
        lib.orc_tree_search.restype = None
        lib.orc_splitmix64_next.argtypes = [P]
        lib.orc_splitmix64_next.restype = u64
        lib.orc_permutation.argtypes = [u64, i64, i64, P]
        lib.orc_permutation.restype = None
        lib.orc_retrieve.argtypes = [P, i64, P, i32, P, P, i32, i32, u64, P, P, P, i32]
        lib.orc_object_scores.argtypes = [P, i64, P, i32, P, P, i32, P, i32]
        lib.orc_object_scores.restype = None
        lib.orc_retrieve.restype = None
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _desc(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a.reshape(-1, WORDS)


def _threads(n):
    return int(n) if n else (os.cpu_count() or 1)


# --- Eq. 1 ---------------------------------------------------------------

def wh_bytes(q, t, N):
    """Eq. 1 on an N x N image given one uint8 per bit. Returns (delta, A, B)."""
    q = np.ascontiguousarray(q, dtype=np.uint8).ravel()
    t = np.ascontiguousarray(t, dtype=np.uint8).ravel()
    assert q.size == N * N and t.size == N * N
    a, b = ctypes.c_int32(), ctypes.c_int32()
    d = _load().orc_wh_bytes(_p(q), _p(t), N, ctypes.byref(a), ctypes.byref(b))
    return d, a.value, b.value


def wh_bitwise(q, t):
    """Eq. 1 on packed 64x64 descriptors, bit by bit. Returns (delta, A, B)."""
    q, t = _desc(q), _desc(t)
    a, b = ctypes.c_int32(), ctypes.c_int32()
    d = _load().orc_wh_bitwise(_p(q), _p(t), ctypes.byref(a), ctypes.byref(b))
    return d, a.value, b.value


def wh(q, t):
    """Eq. 1 on packed 64x64 descriptors, word by word. Returns (delta, A, B)."""
    q, t = _desc(q), _desc(t)
    a, b = ctypes.c_int32(), ctypes.c_int32()
    d = _load().orc_wh(_p(q), _p(t), ctypes.byref(a), ctypes.byref(b))
    return d, a.value, b.value


# --- sequential search ---------------------------------------------------

def bf_topk(db, q, k, nthreads=0):
    """Exact top-k by Eq. 1, ties by lowest index.

    Returns idx int64[nq,k] (-1 past n), score float64[nq,k] (inf past n),
    ab int32[nq,k,2] (A, B; -1 past n)."""
    db, q = _desc(db), _desc(q)
    nq = q.shape[0]
    idx = np.empty((nq, k), dtype=np.int64)
    score = np.empty((nq, k), dtype=np.float64)
    ab = np.empty((nq, k, 2), dtype=np.int32)
    _load().orc_bf_topk(_p(db), db.shape[0], _p(q), nq, k, _p(idx), _p(score), _p(ab),
                        _threads(nthreads))
    return idx, score, ab


# --- Dissimilarity Tree ---------------------------------------------------

class Tree:
    """Flattened tree: BFS node numbering, similar child first."""

    def __init__(self, child, begin, count, level, or_img, and_img, perm):
        self.child, self.begin, self.count, self.level = child, begin, count, level
        self.or_img, self.and_img, self.perm = or_img, and_img, perm

    @property
    def n_nodes(self):
        return self.count.shape[0]

    def is_leaf(self, i):
        return self.child[i, 0] < 0

    def members(self, i):
        b, c = self.begin[i], self.count[i]
        return self.perm[b:b + c]


def build(db, leaf_size=32, literal=False, with_and=False, nthreads=0):
    db = _desc(db)
    n = db.shape[0]
    cap = max(2 * n, 1)
    child = np.empty((cap, 2), dtype=np.int64)
    begin = np.empty(cap, dtype=np.int64)
    count = np.empty(cap, dtype=np.int64)
    level = np.empty(cap, dtype=np.int32)
    or_img = np.empty((cap, WORDS), dtype=np.uint64)
    and_img = np.empty((cap, WORDS), dtype=np.uint64) if with_and else None
    perm = np.empty(max(n, 1), dtype=np.int64)
    m = _load().orc_build(_p(db), n, leaf_size, 1 if literal else 0, _threads(nthreads),
                          _p(child), _p(begin),
                          _p(count), _p(level), _p(or_img), _p(and_img), _p(perm))
    return Tree(child[:m].copy(), begin[:m].copy(), count[:m].copy(), level[:m].copy(),
                or_img[:m].copy(), None if and_img is None else and_img[:m].copy(),
                perm[:n].copy())


def insert(db, tree: Tree, n_old, leaf_size=32, nthreads=0):
    """Incremental insertion into a built tree (§4.1, reading R14).

    ``db`` holds all descriptors by original index: rows 0 .. n_old-1 are the
    ones ``tree`` indexes, rows n_old .. are the batch to insert.  AND images
    are kept (and steer the routing) iff ``tree.and_img`` is not None.
    Returns the new tree; ``tree`` is not modified.
    """
    db = _desc(db)
    n = db.shape[0]
    m = n - n_old
    if m < 0 or tree.perm.shape[0] != n_old:
        raise ValueError("db must hold the indexed descriptors followed by the batch")
    nn = tree.n_nodes
    cap = nn + 2 * n + 1
    child = np.full((cap, 2), -1, dtype=np.int64)
    begin = np.zeros(cap, dtype=np.int64)
    count = np.zeros(cap, dtype=np.int64)
    level = np.zeros(cap, dtype=np.int32)
    or_img = np.zeros((cap, WORDS), dtype=np.uint64)
    with_and = tree.and_img is not None
    and_img = np.zeros((cap, WORDS), dtype=np.uint64) if with_and else None
    perm = np.zeros(max(n, 1), dtype=np.int64)
    child[:nn], begin[:nn], count[:nn], level[:nn] = tree.child, tree.begin, tree.count, tree.level
    or_img[:nn] = tree.or_img
    if with_and:
        and_img[:nn] = tree.and_img
    perm[:n_old] = tree.perm
    total = _load().orc_insert(_p(db), n_old, m, leaf_size, _threads(nthreads), nn, _p(child),
                               _p(begin), _p(count), _p(level), _p(or_img), _p(and_img), _p(perm))
    return Tree(child[:total].copy(), begin[:total].copy(), count[:total].copy(),
                level[:total].copy(), or_img[:total].copy(),
                None if and_img is None else and_img[:total].copy(), perm[:n].copy())


def node_bound(q, or_img, and_img=None):
    """Lower bound of Eq. 1 times P*Z over a node's descriptors (§4.2)."""
    q, o = _desc(q), _desc(or_img)
    a = None if and_img is None else _desc(and_img)
    return _load().orc_node_bound(_p(q), _p(o), _p(a))


def tree_search(db, tree: Tree, q, k, use_and=False, nthreads=0):
    """Best-first Dissimilarity Tree search (§4.2).

    Returns (idx, score, ab, stats) with stats int64[nq, 4] = nodes popped,
    leaves scanned, descriptors scanned, bounds evaluated."""
    db, q = _desc(db), _desc(q)
    nq = q.shape[0]
    idx = np.empty((nq, k), dtype=np.int64)
    score = np.empty((nq, k), dtype=np.float64)
    ab = np.empty((nq, k, 2), dtype=np.int32)
    stats = np.empty((nq, 4), dtype=np.int64)
    and_img = tree.and_img if use_and else None
    if use_and and and_img is None:
        raise ValueError("tree was built without AND images")
    _load().orc_tree_search(_p(db), tree.n_nodes, _p(tree.child), _p(tree.begin),
                            _p(tree.count), _p(tree.or_img), _p(and_img), _p(tree.perm),
                            _p(q), nq, k, _p(idx), _p(score), _p(ab), _p(stats),
                            _threads(nthreads))
    return idx, score, ab, stats


# --- voting ---------------------------------------------------------------

def splitmix64(seed, count):
    """The first `count` outputs of SplitMix64 seeded with `seed`."""
    s = ctypes.c_uint64(seed)
    lib = _load()
    return [lib.orc_splitmix64_next(ctypes.byref(s)) for _ in range(count)]


def permutation(seed, j, n):
    out = np.empty(max(n, 1), dtype=np.int64)
    _load().orc_permutation(seed, j, n, _p(out))
    return out[:n].copy()


def retrieve(db, object_of, n_objects, qdesc, offsets, threshold, seed, nthreads=0):
    """Voting pipeline of §3. Returns (votes uint32[nq, n_objects],
    winner int32[nq], consumed int64[nq])."""
    db, qdesc = _desc(db), _desc(qdesc)
    object_of = np.ascontiguousarray(object_of, dtype=np.uint32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    nq = offsets.shape[0] - 1
    votes = np.empty((max(nq, 1), n_objects), dtype=np.uint32)
    winner = np.empty(max(nq, 1), dtype=np.int32)
    consumed = np.empty(max(nq, 1), dtype=np.int64)
    _load().orc_retrieve(_p(db), db.shape[0], _p(object_of), n_objects, _p(qdesc), _p(offsets),
                         nq, threshold, ctypes.c_uint64(seed), _p(votes), _p(winner),
                         _p(consumed), _threads(nthreads))
    return votes[:nq], winner[:nq], consumed[:nq]


def object_scores(db, object_of, n_objects, qdesc, offsets, nthreads=0):
    """scores float64 [nq][n_objects]: for each query object, the sum over its
    descriptors of the Eq. 1 distance to the nearest descriptor of each
    database object (+inf for an object without descriptors)."""
    db, qdesc = _desc(db), _desc(qdesc)
    obj = np.ascontiguousarray(object_of, dtype=np.uint32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nq = off.shape[0] - 1
    out = np.empty((nq, n_objects), dtype=np.float64)
    _load().orc_object_scores(_p(db), db.shape[0], _p(obj), n_objects, _p(qdesc), _p(off), nq,
                              _p(out), _threads(nthreads))
    return out


def quicci(vertices, triangles, points, normals, support_radius=100.0, modified=False,
           nthreads=0):
    """One 64x64-bit QUICCI (or modified QUICCI) per oriented point, counted
    circle by circle in FP64 (§2.2, §5, reading R15).  vertices float [nv, 3],
    triangles int [nt, 3], points / normals float [np, 3]; returns uint64
    [np, 64] (word = layer from the bottom, bit = circle from the innermost)."""
    v = np.ascontiguousarray(vertices, dtype=np.float32).reshape(-1, 3)
    t = np.ascontiguousarray(triangles, dtype=np.int32).reshape(-1, 3)
    p = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 3)
    n = np.ascontiguousarray(normals, dtype=np.float32).reshape(-1, 3)
    if p.shape != n.shape:
        raise ValueError("points and normals must match")
    if t.size and (t.min() < 0 or t.max() >= v.shape[0]):
        raise ValueError("triangle vertex id out of range")
    out = np.zeros((p.shape[0], WORDS), dtype=np.uint64)
    _load().orc_quicci(_p(v), v.shape[0], _p(t), t.shape[0], _p(p), _p(n), p.shape[0],
                       float(support_radius), 1 if modified else 0, _threads(nthreads), _p(out))
    return out

