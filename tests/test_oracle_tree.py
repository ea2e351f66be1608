"""Pins for the oracle's Dissimilarity Tree (§4.1 construction, §4.2 query)
and its sequential search (§6.2).

- Sequential search is checked against an exact-rational brute force written
  with Python fractions on tiny databases.
- The literal bit-by-bit construction loop and the closed-form split must
  build identical trees.
- Every tree satisfies the structural facts the paper states: the children
  partition their parent, the OR image covers exactly the node's
  descriptors, leaves hold at most the threshold, and the similar side holds
  no bit of popularity rank up to the stopping bit while the dissimilar side
  reaches half the node only at that bit.
- The node bound never exceeds the distance of any descriptor below it.
- Tree search returns exactly the brute-force result (the query of §4.2 is
  exact), including ties, duplicates, empty and full descriptors and k > n.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2107_03368_gb300 import synth

BITS = 4096


def unpack(db):
    db = np.ascontiguousarray(db, dtype=np.uint64).reshape(-1, 64)
    return ((db[:, :, None] >> np.arange(64, dtype=np.uint64)[None, None, :]) & np.uint64(1)
            ).astype(np.uint8).reshape(db.shape[0], BITS)


def random_db(rng, n, density):
    bits = (rng.random((n, BITS)) < density).astype(np.uint8)
    return pack(bits)


def pack(bits):
    bits = np.asarray(bits, dtype=np.uint64).reshape(-1, 64, 64)
    return (bits << np.arange(64, dtype=np.uint64)[None, None, :]).sum(-1).astype(np.uint64)


def exact_topk(db, q, k):
    """Brute force with exact rationals (Eq. 1), ties by lowest index."""
    tb, qb = unpack(db), unpack(q[None])[0]
    nq = int(qb.sum())
    P, Z = max(nq, 1), max(BITS - nq, 1)
    a = ((qb[None, :] == 1) & (tb == 0)).sum(1)
    b = ((qb[None, :] == 0) & (tb == 1)).sum(1)
    d = [Fraction(int(x), P) + Fraction(int(y), Z) for x, y in zip(a, b)]
    order = sorted(range(len(d)), key=lambda i: (d[i], i))
    return order[:k], [d[i] for i in order[:k]]


def mixed_db(seed, n):
    """Generated descriptors plus duplicates, an empty and a full descriptor."""
    rng = np.random.default_rng(seed)
    db, _ = synth.database(seed, n, per_object=max(n // 4, 1), pool=8)
    db = db.copy()
    dup = rng.integers(0, n, size=max(n // 10, 1))
    db[rng.integers(0, n, size=dup.size)] = db[dup]
    db[rng.integers(0, n)] = 0
    db[rng.integers(0, n)] = np.uint64(0xFFFFFFFFFFFFFFFF)
    return db


@pytest.mark.parametrize("n,k", [(1, 1), (7, 3), (40, 5), (60, 60), (25, 30)])
def test_bf_topk_against_exact_rationals(n, k):
    rng = np.random.default_rng(n * 31 + k)
    db = random_db(rng, n, 0.05)
    db[n // 2] = db[0]                          # a duplicate: tie by index
    qs = [db[0], random_db(rng, 1, 0.05)[0], np.zeros(64, np.uint64),
          np.full(64, np.uint64(0xFFFFFFFFFFFFFFFF))]
    for q in qs:
        idx, score, ab = oracle.bf_topk(db, q[None], k)
        order, dist = exact_topk(db, q, k)
        m = min(k, n)
        assert list(idx[0, :m]) == order
        np.testing.assert_allclose(score[0, :m], [float(x) for x in dist], rtol=1e-15, atol=0)
        assert np.all(idx[0, m:] == -1) and np.all(np.isinf(score[0, m:]))


def _split_facts(tree, db_bits, node):
    """Check one internal node's split against the rule of §4.1."""
    s, d = tree.child[node]
    mem = tree.members(node)
    sim, dis = np.sort(tree.members(s)), np.sort(tree.members(d))
    n = mem.size
    assert sorted(np.concatenate([sim, dis]).tolist()) == sorted(mem.tolist())
    bits = db_bits[mem]
    popularity = bits.sum(0)
    key = popularity.astype(np.int64) * BITS + np.arange(BITS)   # bitOrder rank
    big = np.iinfo(np.int64).max
    minkey = {int(i): int(np.where(db_bits[i] == 1, key, big).min()) for i in mem}
    half = (n + 1) // 2
    nonempty = [int(i) for i in mem if minkey[int(i)] < big]
    ordered = sorted(minkey[i] for i in nonempty)
    # the stop bit of §4.1 read R3: the half-th smallest per-descriptor minimum
    stop = ordered[min(half, len(ordered)) - 1] if ordered else None
    rule_dis = [i for i in nonempty if minkey[i] <= stop] if ordered else []
    if 0 < len(rule_dis) < n:
        kstar = max(minkey[int(i)] for i in dis)
        # dissimilar = every descriptor with a set bit at or before the stop bit
        assert all(minkey[int(i)] <= kstar for i in dis)
        assert all(minkey[int(i)] > kstar for i in sim)
        # stop rule: half reached at that bit, or every non-empty one moved
        assert dis.size >= half or dis.size == len(nonempty)
        assert sum(1 for i in mem if minkey[int(i)] < kstar) < half
    else:
        # a side would be empty: positional cut of the ascending list (R4)
        assert list(sim) == sorted(mem.tolist())[: n // 2]


def _structure(tree, db, leaf_size):
    db_bits = unpack(db)
    n = db.shape[0]
    assert sorted(tree.perm.tolist()) == list(range(n))
    assert tree.begin[0] == 0 and tree.count[0] == n
    for i in range(tree.n_nodes):
        mem = tree.members(i)
        orv = np.bitwise_or.reduce(db[mem], axis=0)
        assert np.array_equal(tree.or_img[i], orv)
        if tree.and_img is not None:
            assert np.array_equal(tree.and_img[i], np.bitwise_and.reduce(db[mem], axis=0))
        if tree.is_leaf(i):
            assert tree.count[i] <= leaf_size
            assert np.all(np.diff(mem) > 0)          # ascending original index
            continue
        assert tree.count[i] > leaf_size
        s, d = tree.child[i]
        assert s > i and d == s + 1                       # breadth-first, similar first
        assert tree.level[s] == tree.level[i] + 1
        assert tree.begin[s] == tree.begin[i]
        assert tree.begin[d] == tree.begin[i] + tree.count[s]
        assert tree.count[s] + tree.count[d] == tree.count[i]
        assert tree.count[s] > 0 and tree.count[d] > 0
        assert np.array_equal(tree.or_img[i], tree.or_img[s] | tree.or_img[d])
        _split_facts(tree, db_bits, i)
    assert np.all(np.diff(tree.level) >= 0)


@pytest.mark.parametrize("n,leaf", [(33, 32), (200, 32), (700, 8), (1500, 32)])
def test_literal_equals_closed_form(n, leaf):
    db = mixed_db(n, n)
    a = oracle.build(db, leaf, literal=True, with_and=True)
    b = oracle.build(db, leaf, literal=False, with_and=True)
    for f in ("child", "begin", "count", "level", "or_img", "and_img", "perm"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    _structure(b, db, leaf)


def test_structure_on_generated_data():
    db, _ = synth.database(5, 3000, per_object=300, pool=20)
    t = oracle.build(db, 32)
    _structure(t, db, 32)


@pytest.mark.parametrize("kind", ["identical", "zeros", "ones", "single"])
def test_degenerate_sets(kind):
    rng = np.random.default_rng(7)
    if kind == "identical":
        db = np.repeat(random_db(rng, 1, 0.05), 100, axis=0)
    elif kind == "zeros":
        db = np.zeros((77, 64), np.uint64)
    elif kind == "ones":
        db = np.full((50, 64), np.uint64(0xFFFFFFFFFFFFFFFF))
    else:
        db = random_db(rng, 1, 0.05)
    for literal in (True, False):
        t = oracle.build(db, 32, literal=literal)
        _structure(t, db, 32)
        q = random_db(rng, 3, 0.05)
        idx, score, _, _ = oracle.tree_search(db, t, q, 5)
        bidx, bscore, _ = oracle.bf_topk(db, q, 5)
        assert np.array_equal(idx, bidx) and np.array_equal(score, bscore)


def test_bound_never_exceeds_distance():
    db = mixed_db(11, 600)
    t = oracle.build(db, 16, with_and=True)
    rng = np.random.default_rng(3)
    qs, _ = synth.queries(11, db, 6)
    qs = np.concatenate([qs, random_db(rng, 2, 0.05), np.zeros((1, 64), np.uint64)])
    for q in qs:
        nq = int(np.unpackbits(q.view(np.uint8)).sum())
        PZ = max(nq, 1) * max(BITS - nq, 1)
        dist = np.array([oracle.wh(q, db[i])[0] for i in range(db.shape[0])])
        for node in range(t.n_nodes):
            mem = t.members(node)
            for and_img in (None, t.and_img[node]):
                lb = oracle.node_bound(q, t.or_img[node], and_img) / PZ
                assert lb <= dist[mem].min() + 1e-12


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 1000])
@pytest.mark.parametrize("k", [1, 10])
def test_tree_search_equals_brute_force(n, k):
    db = mixed_db(n + 100, n) if n > 4 else random_db(np.random.default_rng(n), n, 0.05)
    t = oracle.build(db, 32, with_and=True)
    qs, _ = synth.queries(n, db, 20)
    rng = np.random.default_rng(n)
    qs = np.concatenate([qs, db[: min(n, 3)], np.zeros((1, 64), np.uint64),
                         np.full((1, 64), np.uint64(0xFFFFFFFFFFFFFFFF)),
                         random_db(rng, 3, 0.3)])
    bidx, bscore, bab = oracle.bf_topk(db, qs, k)
    for use_and in (False, True):
        idx, score, ab, stats = oracle.tree_search(db, t, qs, k, use_and=use_and)
        assert np.array_equal(idx, bidx)
        assert np.array_equal(score, bscore)
        assert np.array_equal(ab, bab)
        assert np.all(stats[:, 2] <= n) and np.all(stats[:, 0] >= 1)


def test_ties_keep_lowest_index_across_leaves():
    """Many equal-distance duplicates spread over leaves: pruning only on a
    strictly greater bound keeps the lowest indices."""
    rng = np.random.default_rng(9)
    base = random_db(rng, 8, 0.04)
    db = base[rng.integers(0, 8, size=900)]
    t = oracle.build(db, 4)
    qs = np.concatenate([base, random_db(rng, 4, 0.04)])
    for k in (1, 5, 40):
        bidx, bscore, _ = oracle.bf_topk(db, qs, k)
        idx, score, _, _ = oracle.tree_search(db, t, qs, k)
        assert np.array_equal(idx, bidx)


def test_leaf_size_at_least_n_is_brute_force():
    db = mixed_db(4, 300)
    t = oracle.build(db, 300)
    assert t.n_nodes == 1
    qs, _ = synth.queries(4, db, 10)
    idx, _, _, st = oracle.tree_search(db, t, qs, 3)
    assert np.array_equal(idx, oracle.bf_topk(db, qs, 3)[0])
    assert np.all(st[:, 2] == 300)


def test_ties_at_the_bound():
    """Leaves holding copies of a subset of the query have a bound equal to
    their distance (no type B error, every missing query bit outside the
    OR image).  Equal-distance copies then sit in nodes whose bound equals
    the current k-th result: a search that prunes or stops on equality loses
    the lower index."""
    rng = np.random.default_rng(21)
    for trial in range(80):
        q = random_db(rng, 1, 0.02)[0]
        pats = np.stack([q & random_db(rng, 1, 0.7)[0] for _ in range(3)])
        n = int(rng.integers(8, 60))
        db = pats[rng.integers(0, 3, size=n)]
        leaf = int(rng.integers(1, 4))
        t = oracle.build(db, leaf)
        for k in (1, 2, 3, 5):
            bidx = oracle.bf_topk(db, q[None], k)[0]
            idx = oracle.tree_search(db, t, q[None], k)[0]
            assert np.array_equal(idx, bidx), (trial, k)
