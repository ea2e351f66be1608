"""Shared helpers of the parity tests (no arithmetic of the method here)."""
import numpy as np

import oracle
from paper_2107_03368_gb300 import synth

SCORE_RTOL = 1e-6   # FP32 score vs FP64 oracle, relative


def to_dev(a):
    import torch
    a = np.ascontiguousarray(a, dtype=np.uint64).reshape(-1, 64)
    return torch.from_numpy(a.view(np.int64)).cuda()


def idx_np(t):
    return t.cpu().numpy().view(np.uint32).astype(np.int64)


def u16_np(t):
    return t.cpu().numpy().view(np.uint16).astype(np.int32)


def mixed_db(seed, n, per_object=None, pool=8):
    """Generated descriptors plus duplicates, an empty and a full descriptor."""
    rng = np.random.default_rng(seed)
    db, _ = synth.database(seed, n, per_object=per_object or max(n // 4, 1), pool=pool)
    db = db.copy()
    if n >= 4:
        dup = rng.integers(0, n, size=max(n // 10, 1))
        db[rng.integers(0, n, size=dup.size)] = db[dup]
        db[rng.integers(0, n)] = 0
        db[rng.integers(0, n)] = np.uint64(0xFFFFFFFFFFFFFFFF)
    return db


def edge_queries(seed, db, nq):
    rng = np.random.default_rng(seed)
    q, _ = synth.queries(seed, db, nq)
    extra = [np.zeros((1, 64), np.uint64), np.full((1, 64), np.uint64(0xFFFFFFFFFFFFFFFF)),
             db[: min(2, db.shape[0])]]
    dense = (rng.random((1, 4096)) < 0.5).astype(np.uint64).reshape(1, 64, 64)
    extra.append((dense << np.arange(64, dtype=np.uint64)).sum(-1).astype(np.uint64))
    return np.concatenate([q] + extra)


def assert_matches_oracle(db, q, k, idx, score, ab=None, oidx=None):
    """Element-by-element comparison with the oracle's exact top-k."""
    o_idx, o_score, o_ab = oracle.bf_topk(db, q, k)
    g_idx = idx_np(idx)
    exp_idx = np.where(o_idx < 0, 0xFFFFFFFF, o_idx)
    assert np.array_equal(g_idx, exp_idx), "indices differ from the oracle"
    g_score = score.cpu().numpy().astype(np.float64)
    fin = np.isfinite(o_score)
    assert np.all(np.isinf(g_score[~fin]))
    np.testing.assert_allclose(g_score[fin], o_score[fin], rtol=SCORE_RTOL, atol=0)
    assert np.all(g_score[fin][o_score[fin] == 0] == 0.0)
    if ab is not None:
        g_ab = u16_np(ab)
        exp_ab = np.where(o_ab < 0, 0xFFFF, o_ab)
        assert np.array_equal(g_ab, exp_ab), "A/B counts differ from the oracle"


def assert_each_result_exact(db, q, idx, score, rows=None):
    """Every reported result is exact for its own row, whatever the search
    examined: the index is a database row, the FP32 score is that row's
    Eq. 1 distance to the query (the oracle's FP64 value, within SCORE_RTOL;
    exactly 0 for distance 0), and each query's list is strictly ascending in
    (exact distance, index) — distances compared as exact rationals A/P + B/Z
    — with padding (0xFFFFFFFF, +inf) only after the valid results."""
    from fractions import Fraction
    g_idx = idx_np(idx)
    g_s = score.cpu().numpy().astype(np.float64)
    rows = range(q.shape[0]) if rows is None else rows
    n = db.shape[0]
    for r in rows:
        pq = int(np.unpackbits(np.ascontiguousarray(q[r]).view(np.uint8)).sum())
        P, Z = max(pq, 1), max(4096 - pq, 1)
        prev, padded = None, False
        for j in range(g_idx.shape[1]):
            t = int(g_idx[r, j])
            if t == 0xFFFFFFFF:
                assert np.isinf(g_s[r, j]), (r, j)
                padded = True
                continue
            assert not padded, "valid result after padding in row %d" % r
            assert 0 <= t < n, (r, j, t)
            d, a, b = oracle.wh(q[r], db[t])
            if d == 0.0:
                assert g_s[r, j] == 0.0, (r, j)
            else:
                assert abs(g_s[r, j] - d) <= SCORE_RTOL * d, (r, j, g_s[r, j], d)
            key = (Fraction(a, P) + Fraction(b, Z), t)
            assert prev is None or prev < key, "row %d not ascending at %d" % (r, j)
            prev = key
