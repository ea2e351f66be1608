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
