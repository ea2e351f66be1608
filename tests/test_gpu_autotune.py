"""The autotuner (dt_autotune, dt_autotune_retrieve) times launch shapes and
remembers the best; tuned launches give exactly the results of untuned ones
(and, for the votes, the oracle's)."""
import pytest
import torch

from helpers import mixed_db, to_dev
from paper_2107_03368_gb300 import dt, synth

pytestmark = pytest.mark.gpu


def test_autotune_keeps_results(tmp_path):
    db = mixed_db(3, 40_000, per_object=1000)
    q, _ = synth.queries(4, db, 700)
    d_db, d_q = to_dev(db), to_dev(q)
    ix = dt.dt_build(d_db)
    dt.dt_tune_clear()
    before = [dt.dt_search(ix, d_q, 10)[:2], dt.bf_search(d_db, d_q, 10, path=1)[:2],
              dt.bf_search(d_db, d_q, 10, path=2)[:2]]
    rep = dt.dt_autotune(ix, d_db, d_q, 10)
    assert rep["tree_threads"] in (128, 256) and rep["tree_blocks_per_sm"] >= 1
    assert rep["popc_splits"] >= 1 and rep["tc_splits"] >= 1
    assert rep["tc_prewiden"] in (1, 2)
    assert rep["tree_tc_splits"] >= 1 and rep["tree_tc_prewiden"] in (1, 2)
    assert rep["candidates_timed"] >= 12
    after = [dt.dt_search(ix, d_q, 10)[:2], dt.bf_search(d_db, d_q, 10, path=1)[:2],
             dt.bf_search(d_db, d_q, 10, path=2)[:2]]
    for a, b in zip(before, after):
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    p = tmp_path / "tune.txt"
    dt.dt_tune_save(p)
    dt.dt_tune_clear()
    assert dt.dt_tune_load(p) == 4      # per-query tree, batched tree, popcount, tensor
    dt.dt_tune_clear()


@pytest.mark.parametrize("threshold", [0, 3])
def test_autotune_retrieve_keeps_votes(threshold):
    """Engine choice and engine 1's resident blocks tuned on the workload:
    retrieve_objects with engine 0 then gives the untuned votes, winners and
    draw counts, which equal the oracle's voting loop."""
    import numpy as np
    import oracle
    n_obj, per = 6, 1500
    db, obj = synth.database(61, n_obj * per, per_object=per, pool=15)
    qd, off, _ = synth.partial_queries(61, db, n_obj, per, 5)
    d_db, d_obj = to_dev(db), torch.from_numpy(obj.view(np.int32)).cuda()
    d_qd, d_off = to_dev(qd), torch.from_numpy(off).cuda()
    ix = dt.dt_build(d_db)
    dt.dt_tune_clear()
    try:
        before = dt.retrieve_objects(ix, d_obj, n_obj, d_qd, d_off, threshold, 9)
        rep = dt.dt_autotune_retrieve(ix, d_obj, n_obj, d_qd, d_off, threshold)
        assert rep["retrieve_engine"] in (1, 2, 3) and rep["retrieve_ms"] > 0
        after = dt.retrieve_objects(ix, d_obj, n_obj, d_qd, d_off, threshold, 9)
        for x, y in zip(before, after):
            assert torch.equal(x, y)
        o_votes, o_win, o_used = oracle.retrieve(db, obj, n_obj, qd, off, threshold, 9)
        assert np.array_equal(after[0].cpu().numpy().view(np.uint32), o_votes)
        assert np.array_equal(after[1].cpu().numpy(), o_win)
        assert np.array_equal(after[2].cpu().numpy(), o_used)
    finally:
        dt.dt_tune_clear()

