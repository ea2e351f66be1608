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


def _force(tmp_path, kind, n, nq, k, b):
    """A one-entry tuning table fixing the launch of `kind` (2 = tensor
    brute force, 3 = the batched tree's scan) for this shape: 4 database
    splits, database widened inside the kernel (b = 1) or beforehand (b = 2)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    log2 = lambda v: int(v).bit_length() - 1
    path = tmp_path / ("tune_%d_%d.txt" % (kind, b))
    path.write_text("%d %d %d %d %d 4 %d\n" % (kind, log2(n), log2(nq), k, sms, b))
    dt.dt_tune_clear()
    assert dt.dt_tune_load(path) == 1


@pytest.mark.parametrize("n,nq,k", [(30_011, 1_100, 10), (9_000, 130, 1), (257, 300, 32)])
def test_prewidened_database_equals_in_kernel_widening(tmp_path, n, nq, k):
    """The database widened once into scratch and brought in by bulk copies
    (one copy-issuing thread) gives exactly what the producer warps' own
    widening gives, on the plain brute force and on the batched tree scan
    (ragged database tiles, an odd number of query tiles)."""
    db = mixed_db(n + 5, n, per_object=300)
    q = edge_queries(nq, db, nq - 4)
    d_db, d_q = to_dev(db), to_dev(q)
    ix = dt.dt_build(d_db)
    try:
        out = {}
        for b in (1, 2):
            _force(tmp_path, 2, n, q.shape[0], k, b)
            out[("bf", b)] = dt.bf_search(d_db, d_q, k, with_ab=True, path=2)
            _force(tmp_path, 3, n, q.shape[0], k, b)
            out[("tree", b)] = dt.dt_search_path(ix, d_q, k, 2, with_ab=True)[:3]
            dt.dt_sync_status()
    finally:
        dt.dt_tune_clear()
    for kind in ("bf", "tree"):
        for x, y in zip(out[(kind, 1)], out[(kind, 2)]):
            assert torch.equal(x, y), kind
    assert all(torch.equal(x, y) for x, y in zip(out[("bf", 2)], out[("tree", 2)]))
    pick = np.unique(np.linspace(0, q.shape[0] - 1, 80).astype(np.int64))
    idx, score, ab = out[("tree", 2)]
    assert_matches_oracle(db, q[pick], k, idx[pick], score[pick], ab[pick])
