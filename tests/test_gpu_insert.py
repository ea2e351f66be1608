"""dt_insert (incremental insertion, §4.1 suggestion, reading R14) on the GPU
against the oracle: after each batch the GPU tree equals the oracle's node for
node (segments, images, permutation, numbering of rebuilt subtrees); tree
search on it returns the oracle's exact top-k over all descriptors; bad
arguments and failed allocations leave the index as it was."""
import ctypes

import numpy as np
import pytest
import torch

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


def insert_both(db, n_old, ends, leaf, use_and):
    """Build over db[:n_old], then insert db[cur:end] for each end in turn on
    both sides; the trees must agree after every batch."""
    ix = dt.dt_build(to_dev(db[:n_old]), leaf_size=leaf, use_and_image=use_and)
    o = oracle.build(db[:n_old], leaf, with_and=use_and)
    cur = n_old
    for end in ends:
        dt.dt_insert(ix, to_dev(db[cur:end]))
        o = oracle.insert(db[:end], o, cur, leaf_size=leaf)
        cur = end
        assert_same_tree(ix.export(with_and=use_and), o, use_and)
        info = ix.info()
        assert info["n"] == end and info["n_nodes"] == o.n_nodes
        assert info["depth"] == int(o.level.max())
        assert info["n_leaves"] == int((o.child[:, 0] < 0).sum())
    return ix, o


@pytest.mark.parametrize("n_old,ends,leaf,use_and", [
    (1, [70], 32, False),                  # a single leaf overflows
    (20, [25], 32, True),                  # no leaf overflows
    (600, [800], 16, False),
    (3000, [4500], 32, True),
    (400, [2400], 8, False),               # more new than old descriptors
    (2000, [2001], 32, False),             # one descriptor
    (2000, [2300, 2600, 3000], 16, True),  # three batches
])
def test_insert_identical_to_oracle(n_old, ends, leaf, use_and):
    db = mixed_db(n_old + ends[-1], ends[-1])
    insert_both(db, n_old, ends, leaf, use_and)


def test_insert_many_into_one_leaf():
    """5,000 copies of one descriptor: the rebuilt leaf takes the multi-block
    split path and the equal-descriptor fallback of the construction."""
    base = mixed_db(9, 3000)
    rng = np.random.default_rng(9)
    extra = np.concatenate([np.repeat(base[17:18], 5000, axis=0), mixed_db(10, 300)])
    db = np.concatenate([base, extra[rng.permutation(extra.shape[0])]])
    insert_both(db, 3000, [db.shape[0]], 32, False)


def test_insert_on_generated_workload():
    """100,000 generated descriptors, then 20,000 more from new objects."""
    db, _ = synth.database(5, 120000, per_object=2000, pool=8)
    ix, o = insert_both(db, 100000, [120000], 32, False)
    q = edge_queries(6, db, 100)
    for k in (1, 10):
        idx, score, ab, _ = dt.dt_search(ix, to_dev(q), k, with_ab=True)
        assert_matches_oracle(db, q, k, idx, score, ab)


@pytest.mark.parametrize("use_and", [False, True])
def test_search_after_insert_matches_oracle(use_and):
    db = mixed_db(31, 9000)
    ix, _ = insert_both(db, 6000, [7000, 9000], 16, use_and)
    q = edge_queries(32, db, 80)
    for k in (1, 7, 32):
        idx, score, ab, _ = dt.dt_search(ix, to_dev(q), k, with_ab=True)
        assert_matches_oracle(db, q, k, idx, score, ab)


def test_insert_arguments_and_empty_batch():
    db = mixed_db(41, 3000)
    ix = dt.dt_build(to_dev(db[:2000]))
    before = ix.export()
    lib = dt.load()
    new = to_dev(db[2000:])
    assert lib.dt_insert(ix.handle, ctypes.c_void_p(new.data_ptr()), -1, None) == dt.DT_EINVAL
    assert lib.dt_insert(ix.handle, None, 5, None) == dt.DT_EINVAL
    assert lib.dt_insert(None, ctypes.c_void_p(new.data_ptr()), 5, None) == dt.DT_EINVAL
    flat = torch.zeros(65 * 10 + 1, dtype=torch.int64, device="cuda")
    assert lib.dt_insert(ix.handle, ctypes.c_void_p(flat.data_ptr() + 8), 10, None) == dt.DT_EINVAL
    host = np.ascontiguousarray(db[2000:2010])
    assert lib.dt_insert(ix.handle, ctypes.c_void_p(host.ctypes.data), 10, None) == dt.DT_EINVAL
    assert lib.dt_insert(ix.handle, ctypes.c_void_p(new.data_ptr()), 0, None) == dt.DT_OK
    after = ix.export()
    for f in before:
        if before[f] is not None:
            assert np.array_equal(before[f], after[f]), f


def test_failed_allocation_leaves_index_unchanged():
    db = mixed_db(51, 5000)
    ix = dt.dt_build(to_dev(db[:4000]), leaf_size=16)
    before = ix.export()
    new = to_dev(db[4000:])
    failed = 0
    for nth in range(1, 40):
        dt.dt_debug_fail_allocation(nth)
        try:
            dt.dt_insert(ix, new)
        except dt.DtError as e:
            assert e.status == dt.DT_ENOMEM
            failed += 1
            after = ix.export()
            for f in before:
                if before[f] is not None:
                    assert np.array_equal(before[f], after[f]), f
            continue
        finally:
            dt.dt_debug_fail_allocation(0)
        break                           # nth beyond the call's allocations: it succeeded
    else:
        pytest.fail("the insertion never got past the injected failures")
    assert failed >= 5
    o = oracle.insert(db, oracle.build(db[:4000], 16), 4000, leaf_size=16)
    assert_same_tree(ix.export(), o)


def test_other_entry_points_on_a_grown_tree():
    """Voting (tree engine) and the warm-started search on a tree grown by two
    insertions give the same results as on a tree built over everything at
    once (both are exact)."""
    n_obj, per = 12, 400
    db, obj = synth.database(61, n_obj * per, per_object=per, pool=20)
    grown = dt.dt_build(to_dev(db[:3000]), leaf_size=16)
    dt.dt_insert(grown, to_dev(db[3000:4000]))
    dt.dt_insert(grown, to_dev(db[4000:]))
    fresh = dt.dt_build(to_dev(db), leaf_size=16)
    d_obj = torch.from_numpy(obj.view(np.int32)).cuda()
    qd, off = synth.partial_queries(62, db, n_obj, per, 6, n_min=50, n_max=400)[:2]
    d_qd, d_off = to_dev(qd), torch.from_numpy(off).cuda()
    for thr in (0, 5):
        a = dt.retrieve_objects(grown, d_obj, n_obj, d_qd, d_off, thr, 3, engine=1)
        b = dt.retrieve_objects(fresh, d_obj, n_obj, d_qd, d_off, thr, 3, engine=1)
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    q = edge_queries(63, db, 50)
    d_q = to_dev(q)
    idx, score, ab, _ = dt.dt_search(grown, d_q, 5, with_ab=True)
    seeds = torch.flip(idx, dims=[1]).contiguous()
    s_idx, s_score, s_ab, _ = dt.dt_search_seeded(grown, d_q, 5, seeds, with_ab=True)
    assert torch.equal(idx, s_idx) and torch.equal(score, s_score) and torch.equal(ab, s_ab)
    assert_matches_oracle(db, q, 5, idx, score, ab)
    grown.free()
    fresh.free()
