"""The autotuner (dt_autotune) times launch shapes and remembers the best;
tuned launches give exactly the results of untuned ones."""
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
    assert rep["candidates_timed"] >= 12
    after = [dt.dt_search(ix, d_q, 10)[:2], dt.bf_search(d_db, d_q, 10, path=1)[:2],
             dt.bf_search(d_db, d_q, 10, path=2)[:2]]
    for a, b in zip(before, after):
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    p = tmp_path / "tune.txt"
    dt.dt_tune_save(p)
    dt.dt_tune_clear()
    assert dt.dt_tune_load(p) == 3
    dt.dt_tune_clear()
