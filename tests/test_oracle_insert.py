"""Pins for the oracle's incremental insertion into a Dissimilarity Tree
(§4.1 conjecture, reading R14).

- A tree that is a single leaf and overflows is rebuilt from its whole,
  ascending list, so the result must be exactly the construction of §4.1
  over all descriptors.
- An empty batch changes nothing.
- Routing follows least widening: on two well separated clusters a new
  descriptor made of one cluster's common bits lands below that cluster's
  node; an empty descriptor widens no OR image, so the tie sends it to the
  similar child (and, with AND images, widens both clusters' AND images by
  the same count, again a tie); with AND images and clusters of unequal
  common-bit counts it joins the cluster with fewer, on either side.
- After insertion every node's images are those of its members, children
  partition their parent, leaves keep at most leaf_size in ascending
  original index, untouched leaves keep their members, every leaf that
  grew keeps its old members first, the rebuilt subtrees obey the split
  rule of §4.1 and are numbered generation by generation after the old
  nodes.
- The query of §4.2 stays exact: tree search after insertion equals the
  sequential search over all descriptors.
"""
import numpy as np
import pytest

import oracle
from test_oracle_tree import _split_facts, mixed_db, pack, random_db, unpack


def _same_tree(a, b):
    assert a.n_nodes == b.n_nodes
    for f in ("child", "begin", "count", "level", "or_img", "perm"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert (a.and_img is None) == (b.and_img is None)
    if a.and_img is not None:
        assert np.array_equal(a.and_img, b.and_img)


def _check_insert(old, new, db, n_old, leaf_size):
    """Structural facts of a tree after one insertion batch."""
    n = db.shape[0]
    bits = unpack(db)
    assert sorted(new.perm.tolist()) == list(range(n))
    assert new.begin[0] == 0 and new.count[0] == n
    nn = old.n_nodes
    for i in range(new.n_nodes):
        mem = new.members(i)
        assert np.array_equal(new.or_img[i], np.bitwise_or.reduce(db[mem], axis=0))
        if new.and_img is not None:
            assert np.array_equal(new.and_img[i], np.bitwise_and.reduce(db[mem], axis=0))
        if new.is_leaf(i):
            assert new.count[i] <= leaf_size
            assert np.all(np.diff(mem) > 0)
            continue
        s, d = new.child[i]
        assert s > i and d == s + 1
        assert new.level[s] == new.level[i] + 1 and new.level[d] == new.level[i] + 1
        assert new.begin[s] == new.begin[i]
        assert new.begin[d] == new.begin[i] + new.count[s]
        assert new.count[s] + new.count[d] == new.count[i]
        if i < nn and not old.is_leaf(i):
            assert tuple(new.child[i]) == tuple(old.child[i])   # old structure kept
        else:
            _split_facts(new, bits, i)                           # a rebuilt node
    # old leaves: old members first, in their old order, then new ones
    roots = []
    for i in range(nn):
        if not old.is_leaf(i):
            continue
        before = old.members(i)
        if new.is_leaf(i):
            after = new.members(i)
            assert np.array_equal(after[: before.size], before)
            assert np.all(after[before.size:] >= n_old)
        else:
            roots.append(i)
            assert np.array_equal(np.sort(new.members(i))[: before.size], before)
    # rebuilt subtrees: numbered after the old nodes, one generation at a time
    gen, next_id = roots, nn
    while gen:
        nxt = []
        for i in gen:
            if new.is_leaf(i):
                continue
            assert tuple(new.child[i]) == (next_id, next_id + 1)
            nxt += [next_id, next_id + 1]
            next_id += 2
        gen = nxt
    assert next_id == new.n_nodes


def _insert(db, n_old, leaf_size, with_and=False):
    old = oracle.build(db[:n_old], leaf_size=leaf_size, with_and=with_and)
    new = oracle.insert(db, old, n_old, leaf_size=leaf_size)
    return old, new


@pytest.mark.parametrize("with_and", [False, True])
@pytest.mark.parametrize("n_old,m", [(1, 40), (20, 50), (32, 1), (5, 300)])
def test_single_leaf_overflow_equals_build(n_old, m, with_and):
    db = mixed_db(11 + n_old + m, n_old + m)
    old, new = _insert(db, n_old, 32, with_and)
    assert old.n_nodes == 1
    _same_tree(new, oracle.build(db, leaf_size=32, with_and=with_and))


@pytest.mark.parametrize("with_and", [False, True])
def test_empty_batch_is_identity(with_and):
    db = mixed_db(3, 500)
    old, new = _insert(db, 500, 16, with_and)
    _same_tree(new, old)


def test_leaf_without_overflow_is_appended():
    db = mixed_db(5, 25)
    old, new = _insert(db, 20, 32)
    assert new.n_nodes == 1 and list(new.perm) == list(range(25))
    assert np.array_equal(new.or_img[0], np.bitwise_or.reduce(db, axis=0))


def _clusters(seed, ca=10, cb=10):
    """Two clusters over disjoint bit ranges with ca and cb common bits."""
    rng = np.random.default_rng(seed)
    bits = np.zeros((80, 4096), np.uint8)
    bits[:40, 10:1000] = rng.random((40, 990)) < 0.02
    bits[40:, 3010:4000] = rng.random((40, 990)) < 0.02
    bits[:40, 0:ca] = 1
    bits[40:, 3000:3000 + cb] = 1
    return bits


@pytest.mark.parametrize("with_and", [False, True])
def test_routing_least_widening(with_and):
    bits = _clusters(7)
    extra = np.zeros((3, 4096), np.uint8)
    extra[0, 0:10] = 1          # cluster A's common bits
    extra[1, 3000:3010] = 1     # cluster B's common bits
    # extra[2] is empty: a tie at the root
    db = pack(np.concatenate([bits, extra]))
    old, new = _insert(db, 80, 32, with_and)
    s, d = old.child[0]
    a_node = s if 0 in set(old.members(s).tolist()) else d
    b_node = d if a_node == s else s
    assert set(old.members(a_node).tolist()) == set(range(40))
    assert 80 in set(new.members(a_node).tolist())
    assert 81 in set(new.members(b_node).tolist())
    # without AND an empty descriptor widens nothing; with AND it clears the
    # ten common bits of either cluster: a tie both ways, so the similar child
    assert 82 in set(new.members(s).tolist())


def test_routing_by_and_image():
    """With AND images an empty descriptor widens each child's AND image by
    that child's number of common bits, so it joins the cluster with fewer
    common bits, whether that cluster is the similar or the dissimilar child."""
    sides = set()
    for ca, cb in [(10, 20), (20, 10)]:
        bits = _clusters(7, ca, cb)
        db = pack(np.concatenate([bits, np.zeros((1, 4096), np.uint8)]))
        old, new = _insert(db, 80, 32, with_and=True)
        s, d = old.child[0]
        a_node = s if 0 in set(old.members(s).tolist()) else d
        b_node = d if a_node == s else s
        assert set(old.members(a_node).tolist()) == set(range(40))
        fewer = a_node if ca < cb else b_node
        assert 80 in set(new.members(fewer).tolist())
        sides.add(fewer == d)
    assert sides == {False, True}     # both orientations were exercised


@pytest.mark.parametrize("with_and", [False, True])
@pytest.mark.parametrize("seed,n_old,m,leaf", [(1, 600, 200, 16), (2, 3000, 1500, 32),
                                                (3, 400, 2000, 8), (4, 2000, 3, 32)])
def test_structure_after_insert(seed, n_old, m, leaf, with_and):
    db = mixed_db(seed, n_old + m)
    old, new = _insert(db, n_old, leaf, with_and)
    _check_insert(old, new, db, n_old, leaf)


def test_duplicates_into_one_leaf():
    rng = np.random.default_rng(9)
    base = mixed_db(9, 1000)
    dup = np.repeat(base[rng.integers(0, 1000)][None], 300, axis=0)
    db = np.concatenate([base, dup])
    old, new = _insert(db, 1000, 32)
    _check_insert(old, new, db, 1000, 32)


@pytest.mark.parametrize("with_and", [False, True])
def test_search_after_insert_equals_brute_force(with_and):
    rng = np.random.default_rng(21)
    db = mixed_db(21, 2600)
    n_old = 2000
    old = oracle.build(db[:n_old], leaf_size=16, with_and=with_and)
    t1 = oracle.insert(db[:2300], old, n_old, leaf_size=16)
    t2 = oracle.insert(db, t1, 2300, leaf_size=16)          # a second batch
    _check_insert(t1, t2, db, 2300, 16)
    q = np.concatenate([db[rng.integers(0, 2600, 20)], random_db(rng, 10, 0.05),
                        np.zeros((1, 64), np.uint64)])
    for k in (1, 7):
        idx, score, _ab, _st = oracle.tree_search(db, t2, q, k, use_and=with_and)
        bidx, bscore, _ = oracle.bf_topk(db, q, k)
        assert np.array_equal(idx, bidx)
        assert np.array_equal(score, bscore)
