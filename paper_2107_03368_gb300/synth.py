"""Seeded synthetic inputs shaped like the paper's workloads.

The paper evaluates on QUICCI descriptors (64x64 bits, §6) of SHREC'16 meshes;
that data is not available here, so these generators stand in for it:
curve rasterisations with 2-10% of bits set, grouped per object, and queries
made from database descriptors with part of their bits cleared (partiality)
and a few bits flipped (noise).  See ``csrc/synth.c`` for the model.

This module holds no arithmetic of the retrieval method; the oracle and the
CUDA path both take their inputs from here.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

WORDS = 64  # 64 x uint64 = 4096 bits = 512 bytes per descriptor

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build_synth()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, u64, i32, f64 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
        lib.synth_one.argtypes = [u64, i64, i64, i32, P]
        lib.synth_db.argtypes = [u64, i64, i64, i32, P, P, i32]
        lib.synth_queries.argtypes = [u64, P, i64, i64, f64, f64, P, P, i32]
        lib.synth_partial_plan.argtypes = [u64, i64, i64, i64, f64, f64, i64, i64, P, P, P]
        lib.synth_partial_fill.argtypes = [u64, P, i64, i64, P, P, P, f64, f64, P, i32]
        for f in (lib.synth_one, lib.synth_db, lib.synth_queries,
                  lib.synth_partial_plan, lib.synth_partial_fill):
            f.restype = None
        _lib = lib
    return _lib


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def database(seed: int, n: int, per_object: int = 1000, pool: int = 50, nthreads: int = 0):
    """n descriptors (uint64[n, 64]) and their object ids (uint32[n])."""
    lib = _load()
    db = np.empty((n, WORDS), dtype=np.uint64)
    obj = np.empty(n, dtype=np.uint32)
    lib.synth_db(seed, n, per_object, pool, _ptr(db), _ptr(obj), _threads(nthreads))
    return db, obj


def descriptor(seed: int, i: int, per_object: int = 1000, pool: int = 50):
    """Regenerate database descriptor i alone (same bits as ``database``)."""
    out = np.empty(WORDS, dtype=np.uint64)
    _load().synth_one(seed, i, per_object, pool, _ptr(out))
    return out


def queries(seed: int, db: np.ndarray, nq: int, p_clear: float = 0.30,
            p_flip: float = 0.005, nthreads: int = 0):
    """nq noisy partial copies of random database descriptors.

    Returns (uint64[nq, 64] queries, int64[nq] source database index)."""
    db = np.ascontiguousarray(db, dtype=np.uint64)
    out = np.empty((nq, WORDS), dtype=np.uint64)
    src = np.empty(nq, dtype=np.int64)
    _load().synth_queries(seed, _ptr(db), db.shape[0], nq, p_clear, p_flip,
                          _ptr(out), _ptr(src), _threads(nthreads))
    return out, src


def partial_queries(seed: int, db: np.ndarray, n_objects: int, per_object: int, nq: int,
                    f_lo: float = 0.05, f_hi: float = 0.40, n_min: int = 500,
                    n_max: int = 10000, p_clear: float = 0.30, p_flip: float = 0.005,
                    nthreads: int = 0):
    """Partial-object queries: each a contiguous subset of one object's descriptors.

    Returns (qdesc uint64[total, 64], offsets int64[nq+1], object int64[nq])."""
    lib = _load()
    db = np.ascontiguousarray(db, dtype=np.uint64)
    obj = np.empty(nq, dtype=np.int64)
    start = np.empty(nq, dtype=np.int64)
    count = np.empty(nq, dtype=np.int64)
    lib.synth_partial_plan(seed, n_objects, per_object, nq, f_lo, f_hi, n_min, n_max,
                           _ptr(obj), _ptr(start), _ptr(count))
    offsets = np.zeros(nq + 1, dtype=np.int64)
    np.cumsum(count, out=offsets[1:])
    qdesc = np.empty((int(offsets[-1]), WORDS), dtype=np.uint64)
    lib.synth_partial_fill(seed, _ptr(db), per_object, nq, _ptr(obj), _ptr(start),
                           _ptr(offsets), p_clear, p_flip, _ptr(qdesc), _threads(nthreads))
    return qdesc, offsets, obj


# Workload recipes (seed = 2107_03368 + workload number).
SEED_BASE = 210703368


def workload_small():
    """100,000 descriptors (100 objects x 1,000), 100 queries."""
    seed = SEED_BASE + 0
    db, obj = database(seed, 100_000, per_object=1000)
    q, src = queries(seed, db, 100)
    return dict(seed=seed, db=db, object_of=obj, q=q, src=src)


# --- Synthetic meshes (QUICCI generation inputs) ---------------------------
#
# SHREC'16's scanned objects are not available; these stand in for them:
# closed, smooth, blob-shaped triangle meshes (an icosphere whose radius is
# modulated by a few random waves), and partial views of them made of the
# triangles that face a random viewing direction (no occlusion test).  Units
# follow the paper's support radius of 100: objects are a few hundred units
# across.  Vertex normals are area-weighted averages of the incident faces.


def _icosphere(subdiv: int):
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(x, dtype=np.float64) / np.linalg.norm(x) for x in v]
    faces = f
    for _ in range(subdiv):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                mid[key] = len(verts) - 1
            return mid[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts), np.array(faces, dtype=np.int64)


_ICO = {}


def vertex_normals(vertices: np.ndarray, triangles: np.ndarray) -> np.ndarray:
    """Area-weighted average of the incident faces' normals, unit length."""
    v = vertices.astype(np.float64)
    fn = np.cross(v[triangles[:, 1]] - v[triangles[:, 0]], v[triangles[:, 2]] - v[triangles[:, 0]])
    n = np.zeros_like(v)
    for k in range(3):
        np.add.at(n, triangles[:, k], fn)
    ln = np.linalg.norm(n, axis=1, keepdims=True)
    return (n / np.where(ln > 0, ln, 1.0)).astype(np.float32)


def mesh_object(seed: int, subdiv: int = 4, radius: float = 150.0):
    """A closed blob: returns (vertices float32 [nv, 3], triangles int32
    [nt, 3], vertex normals float32 [nv, 3]).  subdiv 4 gives 2,562 vertices
    and 5,120 triangles; each step multiplies both by about four."""
    if subdiv not in _ICO:
        _ICO[subdiv] = _icosphere(subdiv)
    unit, faces = _ICO[subdiv]
    rng = np.random.default_rng(seed)
    r = np.ones(unit.shape[0])
    for _ in range(6):
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        freq = rng.uniform(1.0, 4.0)
        r += rng.uniform(0.05, 0.25) * np.sin(freq * unit @ axis + rng.uniform(0, 2 * np.pi))
    stretch = rng.uniform(0.6, 1.4, size=3)
    v = unit * (radius * r)[:, None] * stretch[None, :]
    v = v + rng.uniform(-50, 50, size=3)
    verts = v.astype(np.float32)
    tris = faces.astype(np.int32)
    return verts, tris, vertex_normals(verts, tris)


def mesh_partial(seed: int, vertices: np.ndarray, triangles: np.ndarray):
    """The triangles facing a random viewing direction, as a mesh of its own
    (vertices renumbered, normals from the kept faces); returns (vertices,
    triangles, normals, kept vertex ids in the complete mesh)."""
    rng = np.random.default_rng(seed)
    view = rng.normal(size=3)
    view /= np.linalg.norm(view)
    v = vertices.astype(np.float64)
    fn = np.cross(v[triangles[:, 1]] - v[triangles[:, 0]], v[triangles[:, 2]] - v[triangles[:, 0]])
    keep = fn @ view > 0
    tris = triangles[keep]
    used = np.unique(tris)
    remap = np.full(vertices.shape[0], -1, np.int64)
    remap[used] = np.arange(used.size)
    pv = vertices[used].copy()
    pt = remap[tris].astype(np.int32)
    return pv, pt, vertex_normals(pv, pt), used
