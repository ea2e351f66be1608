"""Pins for the oracle's Eq. 1 (§2.3, weighted Hamming distance).

The oracle is checked against what the paper and arithmetic fix, not against
a retyped copy of its formula: hand-worked 4x4 values, closed forms
(identical images, empty or full images, complements), the Hamming special
case, and an exhaustive sweep over all pairs of 3x3 images in which every
single-bit change of the target moves the distance by the weight of one
type A or type B error.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bits_to_img(spec, nbits):
    img = np.zeros(nbits, dtype=np.uint8)
    if spec.strip() != "-":
        for b in spec.split(","):
            img[int(b)] = 1
    return img


def _pack(bits4096):
    """uint8[4096] (bit i) -> uint64[64] descriptor."""
    bits = np.asarray(bits4096, dtype=np.uint8).reshape(64, 64)
    w = np.zeros(64, dtype=np.uint64)
    for c in range(64):
        w |= bits[:, c].astype(np.uint64) << np.uint64(c)
    return w


def _unpack(desc):
    d = np.asarray(desc, dtype=np.uint64)
    return ((d[:, None] >> np.arange(64, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(
        np.uint8).ravel()


def test_hand_worked_4x4():
    rows = 0
    with open(os.path.join(GOLDEN, "wh_4x4_hand.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            qs, ts, a, b, frac = [x.strip() for x in line.split(";")]
            q, t = _bits_to_img(qs, 16), _bits_to_img(ts, 16)
            d, A, B = oracle.wh_bytes(q, t, 4)
            assert (A, B) == (int(a), int(b))
            assert d == pytest.approx(float(Fraction(frac)), rel=0, abs=1e-15)
            rows += 1
    assert rows >= 9


def test_exhaustive_3x3_single_bit_changes():
    """All 512 x 512 pairs of 3x3 images.  Starting from t = q (distance 0),
    each target bit that is switched on where the query is 0 costs one type B
    error, 1/max(9-|q|,1); each switched off where the query is 1 costs one
    type A error, 1/max(|q|,1).  Both facts hold at every (q, t, bit), which
    fixes every value of the function."""
    n = 9
    imgs = ((np.arange(512)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    D = np.empty((512, 512))
    AB = np.empty((512, 512, 2), dtype=np.int64)
    for qi in range(512):
        for ti in range(512):
            d, a, b = oracle.wh_bytes(imgs[qi], imgs[ti], 3)
            D[qi, ti] = d
            AB[qi, ti] = (a, b)
    assert np.all(np.diag(D) == 0.0)
    pop = imgs.sum(1)
    for bit in range(n):
        t_without = np.array([t for t in range(512) if not (t >> bit) & 1])
        t_with = t_without | (1 << bit)
        q_has = (np.arange(512) >> bit) & 1
        step = D[:, t_with] - D[:, t_without]
        type_a_weight = 1.0 / np.maximum(pop, 1)
        type_b_weight = 1.0 / np.maximum(n - pop, 1)
        expect = np.where(q_has[:, None] == 1, -type_a_weight[:, None], type_b_weight[:, None])
        np.testing.assert_allclose(step, np.broadcast_to(expect, step.shape), rtol=0, atol=1e-12)
    # A and B are counts of the two error types; together the Hamming distance
    ham = np.array([[bin(q ^ t).count("1") for t in range(512)] for q in range(512)])
    assert np.array_equal(AB.sum(-1), ham)


def test_closed_forms_4096():
    rng = np.random.default_rng(1)
    ones = np.full(64, np.uint64(0xFFFFFFFFFFFFFFFF))
    zero = np.zeros(64, dtype=np.uint64)
    for density in (0.001, 0.05, 0.5, 0.95):
        for _ in range(5):
            qb = (rng.random(4096) < density).astype(np.uint8)
            q = _pack(qb)
            nq = int(qb.sum())
            assert oracle.wh(q, q)[0] == 0.0
            if 0 < nq:
                assert oracle.wh(q, zero)[0] == pytest.approx(1.0, abs=1e-15)
            if nq < 4096:
                assert oracle.wh(q, ones)[0] == pytest.approx(1.0, abs=1e-15)
            if 0 < nq < 4096:
                assert oracle.wh(q, ~q)[0] == pytest.approx(2.0, abs=1e-15)
            tb = (rng.random(4096) < density).astype(np.uint8)
            t = _pack(tb)
            assert oracle.wh(zero, t)[0] == pytest.approx(tb.sum() / 4096.0, abs=1e-15)
            sup = q | t                     # target containing the query: no type A error
            assert oracle.wh(q, sup)[1] == 0
            _, a, b = oracle.wh(q, t)
            assert a + b == int(np.unpackbits((q ^ t).view(np.uint8)).sum())
            assert a == int(((qb == 1) & (tb == 0)).sum())
            assert b == int(((qb == 0) & (tb == 1)).sum())


def test_bitwise_and_wordwise_agree_and_layout():
    rng = np.random.default_rng(2)
    for _ in range(200):
        q = rng.integers(0, 2**63, size=64, dtype=np.uint64) & rng.integers(
            0, 2**63, size=64, dtype=np.uint64)
        t = rng.integers(0, 2**63, size=64, dtype=np.uint64) & rng.integers(
            0, 2**63, size=64, dtype=np.uint64)
        assert oracle.wh(q, t) == oracle.wh_bitwise(q, t)
        # same value as the generic N x N byte form with N = 64
        assert oracle.wh_bytes(_unpack(q), _unpack(t), 64) == oracle.wh(q, t)


def test_full_query_has_no_type_b_weight_guard():
    """|q| = 4096: no type B error can occur, the guard keeps Z = 1."""
    ones = np.full(64, np.uint64(0xFFFFFFFFFFFFFFFF))
    zero = np.zeros(64, dtype=np.uint64)
    assert oracle.wh(ones, zero)[0] == pytest.approx(1.0)
    assert oracle.wh(zero, zero)[0] == 0.0
