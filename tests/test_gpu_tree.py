"""dt_build (§4.1) and dt_search (§4.2) on the GPU against the oracle:
the GPU tree equals the oracle tree node for node; tree search returns the
oracle's exact top-k (bit-exact indices and counts) on both traversals —
per query (path 1) and batched over tiles of queries and tree-ordered rows
on the tensor cores (path 2)."""
import numpy as np
import pytest

import oracle
from helpers import assert_matches_oracle, edge_queries, mixed_db, to_dev
from paper_2107_03368_gb300 import dt, synth

pytestmark = pytest.mark.gpu


def assert_same_tree(g, o, with_and=False):
    assert g["child"].shape == o.child.shape, "node count differs"
    for f in ("child", "begin", "count", "level", "or_img", "perm"):
        assert np.array_equal(g[f], getattr(o, f)), f
    if with_and:
        assert np.array_equal(g["and_img"], o.and_img)


@pytest.mark.parametrize("n,leaf,cap", [(1, 32, 0), (32, 32, 0), (33, 32, 0), (500, 32, 0),
                                        (5000, 32, 64), (5000, 8, 0), (3000, 100, 128)])
def test_tree_identical_to_oracle(n, leaf, cap):
    db = mixed_db(n + 7, n)
    ix = dt.dt_build(to_dev(db), leaf_size=leaf, use_and_image=True, fused_cap=cap)
    g = ix.export(with_and=True)
    o = oracle.build(db, leaf, with_and=True)
    assert_same_tree(g, o, with_and=True)
    info = ix.info()
    assert info["n_nodes"] == o.n_nodes and info["depth"] == int(o.level.max())


@pytest.mark.parametrize("cap", [0, 300])
def test_tree_identical_on_small_workload(cap):
    """100,000 descriptors: single-CTA and multi-CTA split paths."""
    w = synth.workload_small()
    ix = dt.dt_build(to_dev(w["db"]), fused_cap=cap)
    assert_same_tree(ix.export(), oracle.build(w["db"], 32))


@pytest.mark.parametrize("kind", ["identical", "zeros", "ones"])
def test_degenerate_trees(kind):
    rng = np.random.default_rng(1)
    if kind == "identical":
        db = np.repeat(mixed_db(2, 8)[:1], 300, axis=0)
    elif kind == "zeros":
        db = np.zeros((77, 64), np.uint64)
    else:
        db = np.full((90, 64), np.uint64(0xFFFFFFFFFFFFFFFF))
    ix = dt.dt_build(to_dev(db), fused_cap=64)
    assert_same_tree(ix.export(), oracle.build(db, 32))
    q = edge_queries(3, db, 5)
    for path in (1, 2):
        idx, score, ab, _ = dt.dt_search_path(ix, to_dev(q), 5, path, with_ab=True)
        assert_matches_oracle(db, q, 5, idx, score, ab)


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("n,k,use_and", [(1, 1, False), (31, 3, False), (33, 10, True),
                                         (2000, 1, False), (2000, 10, True), (20000, 32, False)])
def test_tree_search_matches_oracle(n, k, use_and, path):
    db = mixed_db(n + 3, n)
    q = edge_queries(n, db, 60)
    ix = dt.dt_build(to_dev(db), use_and_image=use_and)
    idx, score, ab, st = dt.dt_search_path(ix, to_dev(q), k, path, with_ab=True, stats=True)
    assert_matches_oracle(db, q, k, idx, score, ab)
    # the batched path also scans each query's descent leaf (<= 32 rows)
    assert st["descs_scanned"] <= n * q.shape[0] + (32 * q.shape[0] if path == 2 else 0)
    assert st["nodes_visited"] >= q.shape[0]


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("k", [1, 10])
def test_tree_search_small_workload(k, path):
    w = synth.workload_small()
    ix = dt.dt_build(to_dev(w["db"]))
    idx, score, ab, st = dt.dt_search_path(ix, to_dev(w["q"]), k, path, with_ab=True, stats=True)
    assert_matches_oracle(w["db"], w["q"], k, idx, score, ab)
    nq, n = len(w["q"]), w["db"].shape[0]
    if path == 1:
        # visits are within a small factor of the oracle's best-first visits
        o = oracle.build(w["db"], 32)
        _, _, _, ost = oracle.tree_search(w["db"], o, w["q"], k)
        assert st["descs_scanned"] <= 4 * ost[:, 2].sum() + 64 * nq
    else:
        assert 0 < st["descs_scanned"] <= n * nq + 32 * nq
        assert st["bounds_evaluated"] >= nq * ((n + 127) // 128)


def test_ties_at_the_bound_on_gpu():
    """Leaves whose bound equals their distance: no equal-distance loss."""
    rng = np.random.default_rng(21)
    for trial in range(20):
        q = (rng.random(4096) < 0.02).astype(np.uint64).reshape(1, 64, 64)
        q = (q << np.arange(64, dtype=np.uint64)).sum(-1).astype(np.uint64)
        masks = (rng.random((3, 4096)) < 0.7).astype(np.uint64).reshape(3, 64, 64)
        masks = (masks << np.arange(64, dtype=np.uint64)).sum(-1).astype(np.uint64)
        pats = q & masks
        n = int(rng.integers(8, 60))
        db = pats[rng.integers(0, 3, size=n)]
        ix = dt.dt_build(to_dev(db), leaf_size=int(rng.integers(1, 4)))
        for k in (1, 2, 5):
            for path in (1, 2):
                idx, score, ab, _ = dt.dt_search_path(ix, to_dev(q), k, path, with_ab=True)
                assert_matches_oracle(db, q, k, idx, score, ab)


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("k", [1, 10])
def test_seeded_search_is_exact_for_any_seeds(k, path):
    """Warm start: whatever the candidates (exact answers, random, absent,
    repeated, out of range, fewer than k), the result is the oracle's; good
    candidates only remove work."""
    import torch
    db = mixed_db(41, 20000, per_object=500)
    q = edge_queries(42, db, 300)
    d_db, d_q = to_dev(db), to_dev(q)
    ix = dt.dt_build(d_db)
    nq = q.shape[0]
    o_idx, _, _ = oracle.bf_topk(db, q, k)
    rng = np.random.default_rng(5)
    exact = np.where(o_idx < 0, -1, o_idx).astype(np.int64)
    variants = {
        "exact": exact,
        "random": rng.integers(0, db.shape[0], size=(nq, 2 * k)),
        "absent": np.full((nq, 3), -1),
        "repeated": np.repeat(exact[:, :1], 2 * k, axis=1),
        "out_of_range": np.concatenate([exact[:, : max(k - 1, 1)],
                                        np.full((nq, 2), db.shape[0] + 7)], axis=1),
    }
    _, _, _, plain = dt.dt_search_path(ix, d_q, k, path, stats=True)
    for name, seeds in variants.items():
        s = torch.from_numpy(seeds.astype(np.int64).astype(np.uint32).view(np.int32)).cuda()
        idx, score, ab, st = dt.dt_search_path(ix, d_q, k, path, seeds=s.contiguous(),
                                               with_ab=True, stats=True)
        assert_matches_oracle(db, q, k, idx, score, ab)
        if name == "exact":
            assert st["descs_scanned"] <= plain["descs_scanned"], (st, plain)
            assert st["bounds_evaluated"] <= plain["bounds_evaluated"]


def test_seeded_search_with_no_seeds_is_plain_search():
    import torch
    w = synth.workload_small()
    ix = dt.dt_build(to_dev(w["db"]))
    d_q = to_dev(w["q"])
    a = dt.dt_search(ix, d_q, 5, stats=True)
    b = dt.dt_search_seeded(ix, d_q, 5, torch.empty((d_q.shape[0], 0), dtype=torch.int32,
                                                    device=d_q.device), stats=True)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert a[3] == b[3]


# ---------------------------------------------------------------------------
# batched traversal
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,nq,k", [(50_077, 1_037, 1), (50_077, 1_037, 10), (9_000, 300, 32),
                                    (130, 64, 5)])
def test_batched_search_ragged_sizes(n, nq, k):
    """Several scan tiles of 128 rows with a ragged last tile, a ragged last
    query tile (and an odd tile count, so one pair has a single tile), k up
    to 32: the oracle's top-k, and identical to the per-query traversal."""
    db = mixed_db(n + 11, n, per_object=500)
    q = edge_queries(nq, db, nq - 5)
    d_q = to_dev(q)
    ix = dt.dt_build(to_dev(db))
    got = dt.dt_search_path(ix, d_q, k, 2, with_ab=True)
    ref = dt.dt_search_path(ix, d_q, k, 1, with_ab=True)
    for a, b in zip(got[:3], ref[:3]):
        assert torch_equal(a, b)
    pick = np.unique(np.linspace(0, q.shape[0] - 1, 150).astype(np.int64))
    assert_matches_oracle(db, q[pick], k, got[0][pick], got[1][pick], got[2][pick])


def torch_equal(a, b):
    import torch
    return torch.equal(a, b)


def test_batched_search_skips_zero_chunks_and_empty_tiles():
    """Descriptors confined to a band of image rows (most 128-bit K chunks of
    every scan tile are empty and skipped), runs of all-zero descriptors
    (tiles whose image is empty) and a full descriptor: still the oracle's
    top-k."""
    rng = np.random.default_rng(17)
    n = 6_000
    db = np.zeros((n, 64), np.uint64)
    bits = rng.random((n, 64, 64)) < 0.08
    rows = rng.integers(0, 56, size=n)
    for i in range(n):
        lo = rows[i]
        word = (bits[i, lo:lo + 8].astype(np.uint64) << np.arange(64, dtype=np.uint64)).sum(-1)
        db[i, lo:lo + 8] = word
    db[1000:1400] = 0                       # whole tiles of empty descriptors
    db[77] = np.uint64(0xFFFFFFFFFFFFFFFF)
    q = edge_queries(5, db, 200)
    ix = dt.dt_build(to_dev(db))
    for k in (1, 7):
        idx, score, ab, _ = dt.dt_search_path(ix, to_dev(q), k, 2, with_ab=True)
        assert_matches_oracle(db, q, k, idx, score, ab)


def test_batched_search_prunes_tiles():
    """64 objects of 1,024 identical descriptors, object o's bits all in
    word o.  Every bit then has the same popularity, so the construction
    takes bits in index order and splits the objects apart; each object is
    8 scan tiles whose images hold only its word.  Queries are 8 objects'
    patterns with one bit removed: a query's descent ends in its object, its
    cap is one type B error, and every other object's tile has bound |q| Z,
    far above it.  So only the 8 objects' 64 tiles of 512 are scanned, and
    the results — 1,024-way ties broken by lowest index — are the oracle's."""
    rng = np.random.default_rng(23)
    n_obj, per = 64, 1024
    pats = np.zeros((n_obj, 64), np.uint64)
    for o in range(n_obj):
        bits = rng.choice(64, size=40, replace=False)
        pats[o, o] = np.bitwise_or.reduce(np.uint64(1) << bits.astype(np.uint64))
    db = np.repeat(pats, per, axis=0)
    n = db.shape[0]
    objs = rng.choice(n_obj, size=8, replace=False)
    q = np.repeat(pats[objs], 8, axis=0)
    for i in range(q.shape[0]):
        w = int(np.repeat(objs, 8)[i])
        set_bits = [b for b in range(64) if (int(q[i, w]) >> b) & 1]
        q[i, w] &= ~np.uint64(1 << int(rng.choice(set_bits)))
    ix = dt.dt_build(to_dev(db))
    idx, score, ab, st = dt.dt_search_path(ix, to_dev(q), 5, 2, with_ab=True, stats=True)
    assert_matches_oracle(db, q, 5, idx, score, ab)
    assert st["descs_scanned"] <= 64 * 128 * q.shape[0] + 32 * q.shape[0], st


@pytest.mark.parametrize("path", [1, 2])
def test_search_after_insert_and_reload(tmp_path, path):
    """The scan tiles' images follow the rows: after dt_insert (rows move,
    leaves are rebuilt) and after dt_load, both traversals equal the oracle."""
    db = mixed_db(91, 12_000, per_object=400)
    q = edge_queries(92, db, 150)
    ix = dt.dt_build(to_dev(db[:9000]))
    dt.dt_insert(ix, to_dev(db[9000:]))
    idx, score, ab, _ = dt.dt_search_path(ix, to_dev(q), 6, path, with_ab=True)
    assert_matches_oracle(db, q, 6, idx, score, ab)
    ix.save(tmp_path / "t.dtix")
    back = dt.dt_load(tmp_path / "t.dtix", to_dev(db))
    idx, score, ab, _ = dt.dt_search_path(back, to_dev(q), 6, path, with_ab=True)
    assert_matches_oracle(db, q, 6, idx, score, ab)



@pytest.mark.parametrize("n,nq,k", [(50_077, 1_037, 10), (9_000, 300, 32)])
def test_kept_widened_copy_changes_nothing(n, nq, k):
    """dt_keep_widened keeps the tree-ordered rows widened in the index; the
    batched traversal then reads that copy instead of widening per call:
    the same indices, scores and (A, B) as without it, and the oracle's
    top-k; released again, the search still matches."""
    db = mixed_db(n + 3, n, per_object=500)
    q = edge_queries(nq + 3, db, nq - 5)
    d_q = to_dev(q)
    ix = dt.dt_build(to_dev(db))
    ref = dt.dt_search_path(ix, d_q, k, 2, with_ab=True)
    dt.dt_keep_widened(ix, True)
    got = dt.dt_search_path(ix, d_q, k, 2, with_ab=True)
    for a, b in zip(got[:3], ref[:3]):
        assert torch_equal(a, b)
    pick = np.unique(np.linspace(0, q.shape[0] - 1, 100).astype(np.int64))
    assert_matches_oracle(db, q[pick], k, got[0][pick], got[1][pick], got[2][pick])
    dt.dt_keep_widened(ix, False)
    again = dt.dt_search_path(ix, d_q, k, 2, with_ab=True)
    for a, b in zip(again[:3], ref[:3]):
        assert torch_equal(a, b)


def test_kept_widened_copy_follows_insertion():
    """An insertion moves the rows; the kept copy is rebuilt with them."""
    db = mixed_db(95, 14_000, per_object=400)
    q = edge_queries(96, db, 1_100)
    ix = dt.dt_build(to_dev(db[:10_000]))
    dt.dt_keep_widened(ix, True)
    dt.dt_insert(ix, to_dev(db[10_000:]))
    idx, score, ab, _ = dt.dt_search_path(ix, to_dev(q), 7, 2, with_ab=True)
    pick = np.unique(np.linspace(0, q.shape[0] - 1, 120).astype(np.int64))
    assert_matches_oracle(db, q[pick], 7, idx[pick], score[pick], ab[pick])


def test_small_batches_on_a_large_index_take_the_batched_traversal():
    """On an index of 2^17 descriptors or more, dt_search scans batched even
    for a handful of queries (one warp walking most of the rows alone takes
    far longer): its counters are the batched traversal's, and its results
    equal the per-query walk's and the oracle's."""
    db = mixed_db(97, 140_000, per_object=500)
    q = edge_queries(98, db, 10)
    d_q = to_dev(q)
    ix = dt.dt_build(to_dev(db))
    auto = dt.dt_search(ix, d_q, 6, with_ab=True, stats=True)
    batched = dt.dt_search_path(ix, d_q, 6, 2, with_ab=True, stats=True)
    walk = dt.dt_search_path(ix, d_q, 6, 1, with_ab=True)
    for a, b, c in zip(auto[:3], batched[:3], walk[:3]):
        assert torch_equal(a, b) and torch_equal(a, c)
    assert auto[3] == batched[3]
    assert_matches_oracle(db, q, 6, auto[0], auto[1], auto[2])
