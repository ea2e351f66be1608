"""dt_build (§4.1) and dt_search (§4.2) on the GPU against the oracle:
the GPU tree equals the oracle tree node for node; tree search returns the
oracle's exact top-k (bit-exact indices and counts)."""
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
    idx, score, ab, _ = dt.dt_search(ix, to_dev(q), 5, with_ab=True)
    assert_matches_oracle(db, q, 5, idx, score, ab)


@pytest.mark.parametrize("n,k,use_and", [(1, 1, False), (31, 3, False), (33, 10, True),
                                         (2000, 1, False), (2000, 10, True), (20000, 32, False)])
def test_tree_search_matches_oracle(n, k, use_and):
    db = mixed_db(n + 3, n)
    q = edge_queries(n, db, 60)
    ix = dt.dt_build(to_dev(db), use_and_image=use_and)
    idx, score, ab, st = dt.dt_search(ix, to_dev(q), k, with_ab=True, stats=True)
    assert_matches_oracle(db, q, k, idx, score, ab)
    assert st["descs_scanned"] <= n * q.shape[0]
    assert st["nodes_visited"] >= q.shape[0]


@pytest.mark.parametrize("k", [1, 10])
def test_tree_search_small_workload(k):
    w = synth.workload_small()
    ix = dt.dt_build(to_dev(w["db"]))
    idx, score, ab, st = dt.dt_search(ix, to_dev(w["q"]), k, with_ab=True, stats=True)
    assert_matches_oracle(w["db"], w["q"], k, idx, score, ab)
    # visits are within a small factor of the oracle's best-first visits
    o = oracle.build(w["db"], 32)
    _, _, _, ost = oracle.tree_search(w["db"], o, w["q"], k)
    assert st["descs_scanned"] >= 0
    assert st["descs_scanned"] <= 4 * ost[:, 2].sum() + 64 * len(w["q"])


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
            idx, score, ab, _ = dt.dt_search(ix, to_dev(q), k, with_ab=True)
            assert_matches_oracle(db, q, k, idx, score, ab)


@pytest.mark.parametrize("k", [1, 10])
def test_seeded_search_is_exact_for_any_seeds(k):
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
    _, _, _, plain = dt.dt_search(ix, d_q, k, stats=True)
    for name, seeds in variants.items():
        s = torch.from_numpy(seeds.astype(np.int64).astype(np.uint32).view(np.int32)).cuda()
        idx, score, ab, st = dt.dt_search_seeded(ix, d_q, k, s.contiguous(), with_ab=True,
                                                 stats=True)
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
