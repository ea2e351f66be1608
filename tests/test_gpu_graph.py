"""The search entry points can be captured in a CUDA graph and replayed:
all their work is stream-ordered (scratch from the stream-ordered allocator,
no host synchronisation) for dt_search without statistics, bf_search (both
paths) and retrieve_objects with threshold 0.  A replay with new query bits
copied into the captured input gives the same results as a direct call."""
import numpy as np
import pytest
import torch

from helpers import mixed_db, to_dev
from paper_2107_03368_gb300 import dt, synth

pytestmark = pytest.mark.gpu


def _capture(fn):
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()                                  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        out = fn()
    return g, out


def test_graph_replay_matches_direct_calls():
    db = mixed_db(5, 30_000, per_object=1000)
    q1, _ = synth.queries(6, db, 300)
    q2, _ = synth.queries(7, db, 300)
    d_db = to_dev(db)
    ix = dt.dt_build(d_db)
    d_q = to_dev(q1)
    fns = {
        "dt_search": lambda: dt.dt_search(ix, d_q, 10, with_ab=True)[:3],
        "bf_popc": lambda: dt.bf_search(d_db, d_q, 10, with_ab=True, path=1),
        "bf_tc": lambda: dt.bf_search(d_db, d_q, 10, with_ab=True, path=2),
    }
    graphs = {name: _capture(fn) for name, fn in fns.items()}
    d_q.copy_(to_dev(q2))                      # new inputs in the captured buffer
    for name, (g, out) in graphs.items():
        g.replay()
        torch.cuda.synchronize()
        ref = fns[name]()
        for a, b in zip(out, ref):
            assert torch.equal(a, b), name


def test_graph_replay_retrieve():
    seed = 9
    n_obj, per = 40, 250
    db, obj = synth.database(seed, n_obj * per, per_object=per, pool=20)
    qd, off, _ = synth.partial_queries(seed, db, n_obj, per, 30, n_min=50, n_max=200)
    ix = dt.dt_build(to_dev(db))
    d_obj = torch.from_numpy(obj.view(np.int32)).cuda()
    d_qd, d_off = to_dev(qd), torch.from_numpy(off).cuda()
    for engine in (1, 2, 3):
        fn = lambda: dt.retrieve_objects(ix, d_obj, n_obj, d_qd, d_off, 0, seed, engine=engine)
        g, out = _capture(fn)
        g.replay()
        torch.cuda.synchronize()
        ref = fn()
        for a, b in zip(out, ref):
            assert torch.equal(a, b)
