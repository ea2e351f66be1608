"""retrieve_objects (§3) on the GPU against the oracle's voting pipeline:
votes, winners and descriptors drawn bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from helpers import to_dev
from paper_2107_03368_gb300 import dt, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("engine", [1, 2, 3])
@pytest.mark.parametrize("threshold", [0, 1, 3, 10, 100000])
def test_votes_match_oracle(threshold, engine):
    seed = 77
    n_obj, per = 12, 150
    db, obj = synth.database(seed, n_obj * per, per_object=per, pool=10)
    qd, off, _ = synth.partial_queries(seed, db, n_obj, per, 9, n_min=20, n_max=90)
    off = off.copy()
    off[3] = off[2]                       # an empty query (no vote, winner -1)
    ov, ow, oc = oracle.retrieve(db, obj, n_obj, qd, off, threshold, seed)
    ix = dt.dt_build(to_dev(db))
    votes, winner, consumed = dt.retrieve_objects(
        ix, torch.from_numpy(obj.view(np.int32)).cuda(), n_obj, to_dev(qd),
        torch.from_numpy(off).cuda(), threshold, seed, engine=engine)
    assert np.array_equal(votes.cpu().numpy().view(np.uint32), ov)
    assert np.array_equal(winner.cpu().numpy(), ow)
    assert np.array_equal(consumed.cpu().numpy(), oc)


def test_votes_sum_to_descriptor_counts():
    seed = 9
    n_obj, per = 40, 250
    db, obj = synth.database(seed, n_obj * per, per_object=per, pool=20)
    qd, off, qobj = synth.partial_queries(seed, db, n_obj, per, 30, n_min=50, n_max=200)
    ix = dt.dt_build(to_dev(db))
    votes, winner, consumed = dt.retrieve_objects(
        ix, torch.from_numpy(obj.view(np.int32)).cuda(), n_obj, to_dev(qd),
        torch.from_numpy(off).cuda(), 0, seed)
    v = votes.cpu().numpy().view(np.uint32)
    assert np.array_equal(v.sum(1), np.diff(off))
    assert np.array_equal(consumed.cpu().numpy(), np.diff(off))
    assert (winner.cpu().numpy() == qobj).mean() > 0.8
