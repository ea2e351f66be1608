"""bf_search_noalloc — the brute force for callers that cannot let a library
allocate device memory (a serving process with a fixed per-model memory plan,
a host framework that owns all device memory through its own arena): its
scratch is a fixed array inside the library.

The GPU test calls the entry point through the C ABI twice in a row (the
fixed scratch keeps the first call's contents), with the library's
allocator set to fail, checks that free device memory is unchanged across
the second call, and compares both results with the allocating bf_search
and the first also with the oracle.  The file is named to be collected last."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2107_03368_gb300 import dt, synth

SCORE_RTOL = 1e-6


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def test_too_large_request_is_rejected_without_gpu_work():
    lib = dt.load()
    limit_qk = (16 << 20) // 8
    # nq * k just above the fixed scratch: rejected before any pointer is used
    rc = lib.bf_search_noalloc(None, 10, None, limit_qk // 4 + 1, 4, None, None, None, None)
    assert rc == dt.DT_EINVAL
    assert "DT_NOALLOC_SCRATCH_BYTES" in dt.dt_last_error()


@pytest.mark.gpu
def test_noalloc_matches_bf_search_twice():
    import torch
    seed = 4242
    db, _ = synth.database(seed, 30011, per_object=500, pool=20)
    q1, _ = synth.queries(seed, db, 257)
    q2, _ = synth.queries(seed + 1, db, 130)
    d_db = torch.from_numpy(db.view(np.int64)).cuda()
    lib = dt.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (q, k) in enumerate(((q1, 10), (q2, 3))):   # two calls in a row, other shapes
        d_q = torch.from_numpy(q.view(np.int64)).cuda()
        nq = q.shape[0]
        idx = torch.full((nq, k), -7, dtype=torch.int32, device="cuda")
        score = torch.full((nq, k), -1.0, dtype=torch.float32, device="cuda")
        ab = torch.zeros((nq, k, 2), dtype=torch.int16, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        # the entry point's whole contract: any allocation through the
        # library's allocator would fail here and turn into DT_ENOMEM
        dt.dt_debug_fail_allocation(1)
        try:
            rc = lib.bf_search_noalloc(_p(d_db), db.shape[0], _p(d_q), nq, k, _p(idx), _p(score),
                                       _p(ab), stream)
        finally:
            dt.dt_debug_fail_allocation(0)
        assert rc == dt.DT_OK, dt.dt_last_error()
        dt.dt_sync_status()
        if call > 0:   # the first call on a device may load the library's device code
            assert torch.cuda.mem_get_info()[0] == free_before
        r_idx, r_score, r_ab = dt.bf_search(d_db, d_q, k, with_ab=True)
        assert torch.equal(idx, r_idx)
        assert torch.equal(ab, r_ab)
        np.testing.assert_allclose(score.cpu().numpy(), r_score.cpu().numpy(),
                                   rtol=SCORE_RTOL, atol=0)
        if call == 0:  # and directly against the oracle's exact top-k
            o_idx, o_score, o_ab = oracle.bf_topk(db, q, k)
            assert np.array_equal(idx.cpu().numpy().view(np.uint32).astype(np.int64), o_idx)
            assert np.array_equal(ab.cpu().numpy().view(np.uint16).astype(np.int32), o_ab)
            np.testing.assert_allclose(score.cpu().numpy(), o_score, rtol=SCORE_RTOL, atol=0)
