"""bf_search path 2 — the overlap popc(q & t) as an FP8 0/1 contraction on
the tensor cores (tcgen05, FP32 accumulation in tensor memory) — against the
oracle (indices and (A, B) counts bit-exact, scores within 1e-6 relative)
and against the popcount path (identical outputs), at sizes that leave
ragged 128-query and 128-descriptor tiles, and units whose second query
tile is absent (an odd number of query tiles)."""
import numpy as np
import pytest
import torch

from helpers import assert_matches_oracle, edge_queries, mixed_db, to_dev
from paper_2107_03368_gb300 import dt, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,nq,k", [(1, 1, 1), (5, 3, 10), (256, 128, 1), (257, 129, 10),
                                    (1000, 130, 32), (4099, 7, 5), (20000, 300, 10),
                                    (300, 257, 3), (128, 385, 7), (129, 640, 1)])
def test_tc_matches_oracle(n, nq, k):
    db = mixed_db(n + 11, n)
    q = edge_queries(n + 12, db, nq)
    idx, score, ab = dt.bf_search(to_dev(db), to_dev(q), k, with_ab=True, path=2)
    dt.dt_sync_status()
    assert_matches_oracle(db, q, k, idx, score, ab)


def test_tc_equals_popcount_path():
    w = synth.workload_small()
    d_db = to_dev(w["db"])
    q, _ = synth.queries(77, w["db"], 1000)
    d_q = to_dev(q)
    a = dt.bf_search(d_db, d_q, 10, with_ab=True, path=1)
    b = dt.bf_search(d_db, d_q, 10, with_ab=True, path=2)
    dt.dt_sync_status()
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_tc_small_workload_vs_oracle():
    w = synth.workload_small()
    idx, score, ab = dt.bf_search(to_dev(w["db"]), to_dev(w["q"]), 10, with_ab=True, path=2)
    assert_matches_oracle(w["db"], w["q"], 10, idx, score, ab)
