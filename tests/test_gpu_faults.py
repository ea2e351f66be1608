"""Failure handling without a GPU fault (host-injected, both hooks off by
default): a scratch allocation made to fail is reported as DT_ENOMEM, and a
database tile copy that is never issued makes the popcount kernel's bounded
wait give up and report DT_ETIMEOUT.  In both cases nothing faults and the
next calls work and match the oracle."""
import pytest

from helpers import assert_matches_oracle, edge_queries, mixed_db, to_dev
from paper_2107_03368_gb300 import dt

pytestmark = pytest.mark.gpu


@pytest.fixture
def small():
    db = mixed_db(3, 4000, per_object=500)
    q = edge_queries(4, db, 70)
    return db, q, to_dev(db), to_dev(q)


def test_allocation_failure_is_reported_and_recoverable(small):
    db, q, d_db, d_q = small
    ix = dt.dt_build(d_db)
    for nth, call in [(1, lambda: dt.dt_search(ix, d_q, 5)),
                      (2, lambda: dt.bf_search(d_db, d_q, 5, path=2)),
                      (1, lambda: dt.bf_search(d_db, d_q, 5, path=1))]:
        dt.dt_debug_fail_allocation(nth)
        try:
            with pytest.raises(dt.DtError) as e:
                call()
            assert e.value.status == dt.DT_ENOMEM
        finally:
            dt.dt_debug_fail_allocation(0)
    dt.dt_sync_status()
    idx, score, ab, _ = dt.dt_search(ix, d_q, 5, with_ab=True)
    assert_matches_oracle(db, q, 5, idx, score, ab)
    idx, score, ab = dt.bf_search(d_db, d_q, 5, with_ab=True, path=2)
    assert_matches_oracle(db, q, 5, idx, score, ab)


def test_missing_tile_copy_times_out_and_the_context_survives(small):
    db, q, d_db, d_q = small
    dt.dt_debug_inject_missing_copy(True)
    try:
        dt.bf_search(d_db, d_q, 3, path=1)            # enqueued; the wait gives up on the GPU
        with pytest.raises(dt.DtError) as e:
            dt.dt_sync_status()
        assert e.value.status == dt.DT_ETIMEOUT
    finally:
        dt.dt_debug_inject_missing_copy(False)
    dt.dt_sync_status()                                # flag cleared, device fine
    idx, score, ab = dt.bf_search(d_db, d_q, 3, with_ab=True, path=1)
    assert_matches_oracle(db, q, 3, idx, score, ab)
