"""bf_search (sequential search, §6.2) on the GPU against the oracle:
indices and (A, B) counts bit-exact, FP32 scores within 1e-6 relative of
the FP64 oracle, at sizes that span several tiles and ragged tails."""
import numpy as np
import pytest

from helpers import assert_matches_oracle, edge_queries, mixed_db, to_dev
from paper_2107_03368_gb300 import dt, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,nq,k", [(1, 1, 1), (5, 3, 10), (64, 64, 1), (65, 65, 10),
                                    (1000, 130, 32), (4099, 7, 5), (20000, 70, 10)])
def test_bf_matches_oracle(n, nq, k):
    db = mixed_db(n, n)
    q = edge_queries(n + 1, db, nq)
    idx, score, ab = dt.bf_search(to_dev(db), to_dev(q), k, with_ab=True)
    assert_matches_oracle(db, q, k, idx, score, ab)


@pytest.mark.parametrize("k", [1, 10])
def test_bf_small_workload(k):
    """100,000 descriptors, 100 queries (the small workload) in full."""
    w = synth.workload_small()
    idx, score, ab = dt.bf_search(to_dev(w["db"]), to_dev(w["q"]), k, with_ab=True)
    assert_matches_oracle(w["db"], w["q"], k, idx, score, ab)


def test_bf_twice_same_result_and_status():
    db = mixed_db(3, 3000)
    q = edge_queries(4, db, 40)
    d_db, d_q = to_dev(db), to_dev(q)
    a = dt.bf_search(d_db, d_q, 4)
    b = dt.bf_search(d_db, d_q, 4)
    dt.dt_sync_status()
    assert np.array_equal(a[0].cpu().numpy(), b[0].cpu().numpy())
    assert np.array_equal(a[1].cpu().numpy(), b[1].cpu().numpy())


def test_bf_rejects_host_pointer():
    import torch
    db = torch.zeros((4, 64), dtype=torch.int64)   # host tensor
    with pytest.raises(ValueError):
        dt.bf_search(db, db, 1)
