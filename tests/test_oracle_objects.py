"""Pins for the object distance score of the oracle (§6.4): the sum over a
query object's descriptors of each one's Eq. 1 distance to its nearest
descriptor of a database object.  Checked against an exact rational brute
force (Python fractions over the bit definition), against its closed-form
special cases, and against the oracle's own nearest-neighbour search (the
best object of every descriptor holds its nearest neighbour)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2107_03368_gb300 import synth


def _bits(d):
    return [(int(d[w]) >> b) & 1 for w in range(64) for b in range(64)]


def _delta_exact(q, t):
    """Eq. 1 from its definition, N x N = 4096 bits, as an exact fraction."""
    qb, tb = _bits(q), _bits(t)
    pop = sum(qb)
    a = sum(1 for x, y in zip(qb, tb) if x == 1 and y == 0)
    b = sum(1 for x, y in zip(qb, tb) if x == 0 and y == 1)
    return Fraction(a, max(pop, 1)) + Fraction(b, max(4096 - pop, 1))


def _small_case(seed):
    rng = np.random.default_rng(seed)
    db, obj = synth.database(seed, 40, per_object=10, pool=3)
    obj = obj.astype(np.uint32)
    qd, _ = synth.queries(seed, db, 7)
    off = np.array([0, 3, 3, 7], dtype=np.int64)        # one empty query object
    return db, obj, qd, off, rng


@pytest.mark.parametrize("seed", [1, 2])
def test_matches_exact_rational_brute_force(seed):
    db, obj, qd, off, _ = _small_case(seed)
    n_obj = 5                                            # object 4 has no descriptor
    got = oracle.object_scores(db, obj, n_obj, qd, off)
    for j in range(len(off) - 1):
        for o in range(n_obj):
            members = [t for t in range(db.shape[0]) if obj[t] == o]
            if off[j + 1] == off[j]:
                assert got[j, o] == 0.0                 # a sum over no descriptors
                continue
            if not members:
                assert np.isinf(got[j, o])              # a minimum over no descriptors
                continue
            exact = sum((min(_delta_exact(qd[i], db[t]) for t in members)
                         for i in range(off[j], off[j + 1])), Fraction(0))
            assert abs(got[j, o] - float(exact)) <= 1e-12 * max(1.0, float(exact)), (j, o)


def test_copies_of_an_object_score_zero_against_it_and_the_best_object_holds_the_nn():
    db, obj = synth.database(5, 600, per_object=100, pool=6)
    obj = obj.astype(np.uint32)
    qd = np.concatenate([db[100:110], db[450:455]])     # exact copies: objects 1 and 4
    off = np.array([0, 10, 15], dtype=np.int64)
    s = oracle.object_scores(db, obj, 6, qd, off)
    assert s[0, 1] == 0.0 and s[1, 4] == 0.0
    assert np.all(s >= 0)
    # per descriptor: the minimum over objects is the nearest-neighbour distance
    q, _ = synth.queries(6, db, 9)
    offs = np.arange(q.shape[0] + 1, dtype=np.int64)  # one descriptor per query object
    per = oracle.object_scores(db, obj, 6, q, offs)
    nn_idx, nn_score, _ = oracle.bf_topk(db, q, 1)
    np.testing.assert_allclose(per.min(axis=1), nn_score[:, 0], rtol=1e-12, atol=0)
    assert np.all(per[np.arange(q.shape[0]), obj[nn_idx[:, 0]]] == per.min(axis=1))
