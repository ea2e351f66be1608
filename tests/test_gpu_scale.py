"""Full-size parity on the GPU.

- Tree search at scale (10,000,000 descriptors, 10,000 queries, top-10, the
  benchmark's configuration): dt_search equals bf_search for every query
  (indices, (A, B) counts, scores), and a spread sample of queries equals the
  oracle's exact top-10; sampled tree nodes satisfy the structural facts.
- Incremental insertion at scale: 100,000 descriptors of new objects go into
  a 10,000,000-descriptor tree; tree search over the grown tree equals the
  tensor-core brute force over all 10,100,000 descriptors for every query
  (old and new objects), sampled queries equal the oracle, and sampled
  nodes (old and rebuilt) cover exactly their members.
- Partial-object retrieval on the 400-object x 25,000-descriptor database:
  votes equal the histogram of the brute-force nearest neighbours' objects
  (a separate GPU path) for a subset of uneven partial queries, and sampled
  nearest neighbours equal the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import SCORE_RTOL, idx_np, to_dev, u16_np
from paper_2107_03368_gb300 import dt, synth

pytestmark = pytest.mark.gpu

SEED = 210703368 + 1


@pytest.fixture(scope="module")
def big():
    db, _ = synth.database(SEED, 10_000_000, per_object=1000)
    q, _ = synth.queries(SEED, db, 10_000)
    d_db, d_q = to_dev(db), to_dev(q)
    ix = dt.dt_build(d_db)
    yield db, q, d_db, d_q, ix
    ix.free()


def test_tree_equals_brute_force_all_queries(big):
    db, q, d_db, d_q, ix = big
    t_idx, t_score, t_ab, _ = dt.dt_search(ix, d_q, 10, with_ab=True)
    b_idx, b_score, b_ab = dt.bf_search(d_db, d_q, 10, with_ab=True, path=1)
    c_idx, c_score, c_ab = dt.bf_search(d_db, d_q, 10, with_ab=True, path=2)
    dt.dt_sync_status()
    for idx, score, ab in ((b_idx, b_score, b_ab), (c_idx, c_score, c_ab)):
        assert torch.equal(t_idx, idx)
        assert torch.equal(t_ab, ab)
        assert torch.equal(t_score, score)


def test_sampled_queries_equal_oracle(big):
    db, q, d_db, d_q, ix = big
    pick = np.linspace(0, q.shape[0] - 1, 12).astype(np.int64)
    t_idx, t_score, t_ab, _ = dt.dt_search(ix, d_q, 10, with_ab=True)
    o_idx, o_score, o_ab = oracle.bf_topk(db, q[pick], 10)
    assert np.array_equal(idx_np(t_idx)[pick], o_idx)
    assert np.array_equal(u16_np(t_ab)[pick], o_ab)
    np.testing.assert_allclose(t_score.cpu().numpy()[pick], o_score, rtol=SCORE_RTOL, atol=0)


def test_sampled_nodes_structure(big):
    db, q, d_db, d_q, ix = big
    t = ix.export()
    m = t["count"].shape[0]
    assert t["count"][0] == db.shape[0]
    assert sorted(t["perm"][:1000].tolist()) == sorted(set(t["perm"][:1000].tolist()))
    rng = np.random.default_rng(0)
    for node in rng.integers(0, m, size=200):
        b, c = t["begin"][node], t["count"][node]
        mem = t["perm"][b:b + c]
        assert np.array_equal(np.bitwise_or.reduce(db[mem], axis=0), t["or_img"][node])
        s, d = t["child"][node]
        if s < 0:
            assert c <= 32 and np.all(np.diff(mem) > 0)
        else:
            assert c > 32
            assert t["begin"][s] == b and t["begin"][d] == b + t["count"][s]
            assert t["count"][s] + t["count"][d] == c and t["count"][s] > 0


def test_insert_at_full_size(big):
    db, q, d_db, d_q, _ = big
    new, _ = synth.database(SEED + 5, 100_000, per_object=1000)
    q_new, _ = synth.queries(SEED + 6, new, 1000)
    ix = dt.dt_build(d_db)
    try:
        n_nodes0 = ix.info()["n_nodes"]
        dt.dt_insert(ix, to_dev(new))
        info = ix.info()
        assert info["n"] == 10_100_000 and info["n_nodes"] > n_nodes0
        all_db = np.concatenate([db, new])
        d_all = torch.cat([d_db, to_dev(new)])
        qq = np.concatenate([q, q_new])
        d_qq = to_dev(qq)
        t_idx, t_score, t_ab, _ = dt.dt_search(ix, d_qq, 10, with_ab=True)
        c_idx, c_score, c_ab = dt.bf_search(d_all, d_qq, 10, with_ab=True, path=2)
        dt.dt_sync_status()
        assert torch.equal(t_idx, c_idx) and torch.equal(t_ab, c_ab) and torch.equal(t_score, c_score)
        hit_new = (idx_np(t_idx)[:, 0] >= 10_000_000).mean()
        assert hit_new > 0.05                    # the new objects' queries find them
        pick = np.concatenate([np.linspace(0, 9999, 6), np.linspace(10000, 10999, 6)]).astype(np.int64)
        o_idx, o_score, o_ab = oracle.bf_topk(all_db, qq[pick], 10)
        assert np.array_equal(idx_np(t_idx)[pick], o_idx)
        assert np.array_equal(u16_np(t_ab)[pick], o_ab)
        np.testing.assert_allclose(t_score.cpu().numpy()[pick], o_score, rtol=SCORE_RTOL, atol=0)
        t = ix.export()
        assert sorted(t["perm"][-1000:].tolist()) == sorted(set(t["perm"][-1000:].tolist()))
        rng = np.random.default_rng(1)
        nodes = np.concatenate([rng.integers(0, n_nodes0, 100),
                                rng.integers(n_nodes0, info["n_nodes"], 100)])
        for node in nodes:
            b, c = t["begin"][node], t["count"][node]
            mem = t["perm"][b:b + c]
            assert np.array_equal(np.bitwise_or.reduce(all_db[mem], axis=0), t["or_img"][node])
            if t["child"][node][0] < 0:
                assert c <= 32 and np.all(np.diff(mem) > 0)
    finally:
        ix.free()


def test_partial_retrieval_on_full_database():
    """Threshold 0 on a subset of uneven queries with every engine; threshold
    10 on all 1,000 queries with the round-based tensor engine; threshold 0
    on 60 queries (about 340,000 query descriptors) with the batched tree
    engine, sampled queries checked against their brute-force neighbours."""
    n_obj, per = 400, 25_000
    db, obj = synth.database(SEED + 2, n_obj * per, per_object=per)
    qd, off, qobj = synth.partial_queries(SEED + 2, db, n_obj, per, 1000)
    sub = 4                                            # first 4 uneven queries
    off_s = off[: sub + 1].copy()
    qd_s = qd[: off_s[-1]]
    sizes = np.diff(off_s)
    assert sizes.min() >= 500 and sizes.max() <= 10_000
    d_db = to_dev(db)
    ix = dt.dt_build(d_db)
    d_obj = torch.from_numpy(obj.view(np.int32)).cuda()
    d_qd = to_dev(qd_s)
    votes, winner, consumed = dt.retrieve_objects(ix, d_obj, n_obj, d_qd,
                                                  torch.from_numpy(off_s).cuda(), 0, SEED, engine=2)
    votes_t, winner_t, consumed_t = dt.retrieve_objects(ix, d_obj, n_obj, d_qd,
                                                        torch.from_numpy(off_s).cuda(), 0, SEED,
                                                        engine=1)
    assert torch.equal(votes, votes_t) and torch.equal(winner, winner_t)
    assert torch.equal(consumed, consumed_t)
    r3 = dt.retrieve_objects(ix, d_obj, n_obj, d_qd, torch.from_numpy(off_s).cuda(), 0, SEED,
                             engine=3)
    for x, y in zip(r3, (votes, winner, consumed)):
        assert torch.equal(x, y)
    b_idx, _, _ = dt.bf_search(d_db, d_qd, 1)
    nn = idx_np(b_idx)[:, 0]
    v = votes.cpu().numpy().view(np.uint32)
    for j in range(sub):
        hist = np.bincount(obj[nn[off_s[j]:off_s[j + 1]]], minlength=n_obj)
        assert np.array_equal(v[j], hist)
        assert winner[j].item() == int(np.argmax(hist))
    assert np.array_equal(consumed.cpu().numpy(), sizes)
    assert np.all(winner.cpu().numpy() == qobj[:sub])
    pick = np.linspace(0, qd_s.shape[0] - 1, 8).astype(np.int64)
    o_idx, _, _ = oracle.bf_topk(db, qd_s[pick], 1)
    assert np.array_equal(nn[pick], o_idx[:, 0])
    # threshold 10, subset: both engines agree
    r2 = dt.retrieve_objects(ix, d_obj, n_obj, d_qd, torch.from_numpy(off_s).cuda(), 10, SEED,
                             engine=2)
    r1 = dt.retrieve_objects(ix, d_obj, n_obj, d_qd, torch.from_numpy(off_s).cuda(), 10, SEED,
                             engine=1)
    r3 = dt.retrieve_objects(ix, d_obj, n_obj, d_qd, torch.from_numpy(off_s).cuda(), 10, SEED,
                             engine=3)
    for x, y, z in zip(r1, r2, r3):
        assert torch.equal(x, y) and torch.equal(x, z)
    # threshold 10 on all 1,000 partial queries: the winner reaches exactly 10
    # votes, every vote is a draw, and the draws replay the oracle's order
    votes10, winner10, used10 = dt.retrieve_objects(ix, d_obj, n_obj, to_dev(qd),
                                                    torch.from_numpy(off).cuda(), 10, SEED,
                                                    engine=2)
    v10 = votes10.cpu().numpy().view(np.uint32)
    w10, u10 = winner10.cpu().numpy(), used10.cpu().numpy()
    assert np.all(v10[np.arange(len(w10)), w10] == 10)
    assert np.array_equal(v10.sum(1), u10) and np.all(u10 <= np.diff(off))
    assert (w10 == qobj).mean() > 0.95
    j = 7                                   # replay one query by hand
    order = oracle.permutation(SEED, j, int(off[j + 1] - off[j]))[: u10[j]]
    o_nn, _, _ = oracle.bf_topk(db, qd[off[j] + order], 1)
    expect = np.bincount(obj[o_nn[:, 0]], minlength=n_obj)
    assert np.array_equal(v10[j], expect)

    # threshold 0 on 60 of the partial queries (about 340,000 descriptors)
    # with the batched tree engine
    m = 60
    off, qobj = off[: m + 1].copy(), qobj[:m]
    d_all, d_off = to_dev(qd[: off[-1]]), torch.from_numpy(off).cuda()
    votes0, winner0, used0 = dt.retrieve_objects(ix, d_obj, n_obj, d_all, d_off, 0, SEED, engine=3)
    v0 = votes0.cpu().numpy().view(np.uint32)
    assert np.array_equal(v0.sum(1), np.diff(off))
    assert np.array_equal(used0.cpu().numpy(), np.diff(off))
    for j in (0, 31, m - 1):
        q_j = to_dev(qd[off[j]:off[j + 1]])
        nn_j = idx_np(dt.bf_search(d_db, q_j, 1, path=2)[0])[:, 0]
        assert np.array_equal(v0[j], np.bincount(obj[nn_j], minlength=n_obj))
        assert winner0[j].item() == int(np.argmax(v0[j]))
    assert (winner0.cpu().numpy() == qobj).mean() > 0.95
    ix.free()


def test_object_scores_on_full_database():
    """Object distance scores of a few query objects against the 400 x
    25,000 database, each checked against the oracle."""
    n_obj, per = 400, 25_000
    db, obj = synth.database(SEED + 2, n_obj * per, per_object=per)
    qd, off, qobj = synth.partial_queries(SEED + 2, db, n_obj, per, 3)
    pick = [np.arange(off[j], off[j] + 4) for j in range(3)]       # 4 descriptors of each
    sub = np.concatenate([qd[p] for p in pick])
    soff = np.array([0, 4, 8, 12], dtype=np.int64)
    got = dt.object_scores(to_dev(db), torch.from_numpy(obj.view(np.int32)).cuda(), n_obj,
                           to_dev(sub), torch.from_numpy(soff).cuda()).cpu().numpy()
    exp = oracle.object_scores(db, obj, n_obj, sub, soff)
    np.testing.assert_allclose(got, exp, rtol=1e-12, atol=0)
    assert np.all(np.argmin(got, axis=1) == qobj[:3])    # the source object scores lowest
