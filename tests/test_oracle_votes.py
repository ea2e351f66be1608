"""Pins for the oracle's voting pipeline (§3) and its random draw order.

- SplitMix64 reproduces the published output sequence (tests/golden).
- The draw order of each query is a permutation, fixed by (seed, query).
- The vote loop agrees with a step-by-step Python replay of §3 over the
  oracle's own nearest neighbours and permutations: one vote per drawn
  descriptor for the object of its nearest neighbour, stop at the first
  object to reach the threshold.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2107_03368_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_sequence():
    lines = [l.strip() for l in open(os.path.join(GOLDEN, "splitmix64.txt"))
             if l.strip() and not l.startswith("#")]
    seed = int(lines[0].split()[1])
    expect = [int(x) for x in lines[1:]]
    assert oracle.splitmix64(seed, len(expect)) == expect


@pytest.mark.parametrize("n", [0, 1, 2, 17, 1000])
def test_permutation_is_a_permutation(n):
    for j in range(4):
        p = oracle.permutation(12345, j, n)
        assert sorted(p.tolist()) == list(range(n))
        assert np.array_equal(p, oracle.permutation(12345, j, n))
    if n > 10:
        assert not np.array_equal(oracle.permutation(1, 0, n), oracle.permutation(1, 1, n))
        assert not np.array_equal(oracle.permutation(1, 0, n), oracle.permutation(2, 0, n))


def test_permutation_first_draw_by_hand():
    """n = 2: one swap decided by the first draw of the query's stream."""
    seed, j = 99, 3
    s0 = (seed + j * 0x9E3779B97F4A7C15) % 2**64
    state = oracle.splitmix64(s0, 1)[0]
    first = oracle.splitmix64(state, 1)[0]
    expect = [1, 0] if first % 2 == 0 else [0, 1]
    assert oracle.permutation(seed, j, 2).tolist() == expect


def _replay(nn_obj, order, threshold, n_objects):
    votes = [0] * n_objects
    used, win = 0, -1
    for i in order:
        o = nn_obj[i]
        votes[o] += 1
        used += 1
        if threshold > 0 and votes[o] == threshold:
            win = o
            break
    if win < 0 and any(votes):
        win = max(range(n_objects), key=lambda o: (votes[o], -o))
    return votes, win, used


@pytest.mark.parametrize("threshold", [0, 1, 3, 10, 1000])
def test_retrieve_matches_stepwise_replay(threshold):
    seed = 77
    n_obj, per = 12, 150
    db, obj = synth.database(seed, n_obj * per, per_object=per, pool=10)
    qd, off, qobj = synth.partial_queries(seed, db, n_obj, per, 6, n_min=20, n_max=60)
    off = off.copy()
    off[3] = off[2]                  # make query 2 empty: no vote, winner -1
    votes, winner, used = oracle.retrieve(db, obj, n_obj, qd, off, threshold, seed)
    nn, _, _ = oracle.bf_topk(db, qd, 1)
    for j in range(len(off) - 1):
        m = off[j + 1] - off[j]
        order = oracle.permutation(seed, j, m)
        nn_obj = [int(obj[nn[off[j] + i, 0]]) for i in range(m)]
        v, w, u = _replay(nn_obj, order, threshold, n_obj)
        assert votes[j].tolist() == v
        assert winner[j] == w
        assert used[j] == u
        if threshold == 0:
            assert votes[j].sum() == m
    assert winner[2] == -1 and used[2] == 0


def test_partial_queries_find_their_object():
    """Generated partial queries mostly vote for the object they come from."""
    seed = 5
    n_obj, per = 20, 200
    db, obj = synth.database(seed, n_obj * per, per_object=per, pool=10)
    qd, off, qobj = synth.partial_queries(seed, db, n_obj, per, 8, n_min=20, n_max=80)
    votes, winner, _ = oracle.retrieve(db, obj, n_obj, qd, off, 10, seed)
    assert (winner == qobj).mean() >= 0.75
