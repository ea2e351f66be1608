"""quicci_generate (§2.2, §5, reading R15) on the GPU against the oracle.

- Closed forms on flat meshes (plane through the axis, parallel plane,
  half-plane, strip limited in height): bit-exact.
- Generated closed meshes and partial views, QUICCI and modified QUICCI:
  the kernel decides in FP32 and the oracle in FP64, so a bit may differ
  only where the geometry sits on a decision boundary; such bits are found
  by the oracle itself (they change when the support radius moves by
  1e-5 relative, which moves every circle and layer by far more than FP32
  rounding).  Every other bit must match, and ambiguous bits must be rare.
- Degenerate inputs: a zero normal and a point out of reach give empty
  images; no points is a no-op; bad vertex ids and radii are rejected.
- The paper's pipeline end to end on synthetic meshes: QUICCI of every
  vertex of complete objects into a tree, modified QUICCI of partial views
  as queries, votes name the source object.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2107_03368_gb300 import dt, synth

pytestmark = pytest.mark.gpu

R = 100.0


def cuda(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def gpu_quicci(v, t, p, n, r=R, modified=False):
    out = dt.quicci(cuda(v, torch.float32), cuda(t, torch.int32), cuda(p, torch.float32),
                    cuda(n, torch.float32), r, modified)
    return out.cpu().numpy().view(np.uint64)


def quad(x0, x1, y, z0, z1):
    v = np.array([[x0, y, z0], [x1, y, z0], [x1, y, z1], [x0, y, z1]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return v, t


P0 = np.zeros((1, 3), np.float32)
NZ = np.array([[0, 0, 1]], np.float32)


@pytest.mark.parametrize("modified", [False, True])
def test_closed_forms(modified):
    v, t = quad(-170.0, 230.0, 0.0, -200.0, 200.0)
    assert np.all(gpu_quicci(v, t, P0, NZ, modified=modified)[0] == np.uint64(1))
    v, t = quad(-170.0, 230.0, 37.0, -200.0, 200.0)
    assert np.all(gpu_quicci(v, t, P0, NZ, modified=modified)[0] == np.uint64(1) << np.uint64(23))
    v, t = quad(0.0, 230.0, 37.0, -200.0, 200.0)
    half = gpu_quicci(v, t, P0, NZ, modified=modified)[0]
    assert np.all(half == (0 if modified else np.uint64(1) << np.uint64(23)))
    v, t = quad(-170.0, 230.0, 0.0, -20.3, 45.1)
    strip = gpu_quicci(v, t, P0, NZ, modified=modified)[0]
    assert np.array_equal(np.flatnonzero(strip), np.arange(26, 46))


def ambiguous(v, t, p, n, modified):
    lo = oracle.quicci(v, t, p, n, R * (1 - 1e-5), modified)
    hi = oracle.quicci(v, t, p, n, R * (1 + 1e-5), modified)
    mid = oracle.quicci(v, t, p, n, R, modified)
    return mid, (lo ^ mid) | (hi ^ mid)


def popcount(a):
    return int(np.unpackbits(np.ascontiguousarray(a).view(np.uint8)).sum())


@pytest.mark.parametrize("modified", [False, True])
@pytest.mark.parametrize("partial", [False, True])
def test_matches_oracle_on_generated_meshes(partial, modified):
    v, t, n = synth.mesh_object(11 + partial, 4)
    if partial:
        v, t, n, _ = synth.mesh_partial(12, v, t)
    pick = np.arange(0, v.shape[0], 3)
    p, pn = v[pick], n[pick]
    g = gpu_quicci(v, t, p, pn, modified=modified)
    o, amb = ambiguous(v, t, p, pn, modified)
    diff = g ^ o
    assert np.all((diff & ~amb) == 0), "bits differ away from a decision boundary"
    total = p.shape[0] * 4096
    assert popcount(amb) < 1e-3 * total
    assert popcount(o) > 20 * p.shape[0]            # descriptors are not empty
    # a few descriptors from points off the surface, with tilted normals
    rng = np.random.default_rng(13)
    q = (v[rng.integers(0, v.shape[0], 64)] + rng.normal(0, 20, (64, 3))).astype(np.float32)
    qn = rng.normal(size=(64, 3)).astype(np.float32)
    g = gpu_quicci(v, t, q, qn, modified=modified)
    o, amb = ambiguous(v, t, q, qn, modified)
    assert np.all(((g ^ o) & ~amb) == 0)


def test_large_mesh_sampled_points():
    """20,480 triangles; 96 sampled vertices of the complete mesh."""
    v, t, n = synth.mesh_object(21, 5)
    pick = np.linspace(0, v.shape[0] - 1, 96).astype(np.int64)
    g = gpu_quicci(v, t, v, n)[pick]
    o, amb = ambiguous(v, t, v[pick], n[pick], False)
    assert np.all(((g ^ o) & ~amb) == 0)


def test_degenerate_inputs():
    v, t, n = synth.mesh_object(31, 3)
    pts = np.array([[5000, 0, 0], v[0]], np.float32)
    nrm = np.array([[0, 0, 1], [0, 0, 0]], np.float32)
    assert np.all(gpu_quicci(v, t, pts, nrm) == 0)
    lib = dt.load()
    dv, dtr = cuda(v, torch.float32), cuda(t, torch.int32)
    dp, dn = cuda(v[:4], torch.float32), cuda(n[:4], torch.float32)
    out = torch.zeros((4, 64), dtype=torch.int64, device="cuda")
    P = lambda x: ctypes.c_void_p(x.data_ptr())
    assert lib.quicci_generate(P(dv), v.shape[0], P(dtr), t.shape[0], P(dp), P(dn), 0, 100.0, 0,
                               P(out), None) == dt.DT_OK
    assert lib.quicci_generate(P(dv), v.shape[0], P(dtr), t.shape[0], P(dp), P(dn), 4, 0.0, 0,
                               P(out), None) == dt.DT_EINVAL
    assert lib.quicci_generate(P(dv), v.shape[0], P(dtr), t.shape[0], P(dp), P(dn), 4,
                               float("inf"), 0, P(out), None) == dt.DT_EINVAL
    bad = t.copy()
    bad[5, 1] = v.shape[0]
    dbad = cuda(bad, torch.int32)
    assert lib.quicci_generate(P(dv), v.shape[0], P(dbad), t.shape[0], P(dp), P(dn), 4, 100.0, 0,
                               P(out), None) == dt.DT_EINVAL
    assert "vertex id" in dt.dt_last_error()
    # no triangles: empty descriptors
    empty = gpu_quicci(v, np.zeros((0, 3), np.int32), v[:4], n[:4])
    assert np.all(empty == 0)


def test_pipeline_on_synthetic_meshes():
    """Complete objects -> QUICCI per vertex -> tree; partial views ->
    modified QUICCI per vertex -> votes (threshold 0: every descriptor)."""
    n_obj = 8
    db, obj = [], []
    parts = []
    for o in range(n_obj):
        v, t, n = synth.mesh_object(100 + o, 4)
        db.append(gpu_quicci(v, t, v, n))
        obj.append(np.full(v.shape[0], o, np.uint32))
        pv, pt, pn, _ = synth.mesh_partial(200 + o, v, t)
        parts.append(gpu_quicci(pv, pt, pv, pn, modified=True))
    db = np.concatenate(db)
    obj = np.concatenate(obj)
    qd = np.concatenate(parts)
    off = np.concatenate([[0], np.cumsum([p.shape[0] for p in parts])]).astype(np.int64)
    d_db = torch.from_numpy(db.view(np.int64)).cuda()
    ix = dt.dt_build(d_db)
    votes, winner, _ = dt.retrieve_objects(ix, torch.from_numpy(obj.view(np.int32)).cuda(), n_obj,
                                           torch.from_numpy(qd.view(np.int64)).cuda(),
                                           torch.from_numpy(off).cuda(), 0, 1)
    w = winner.cpu().numpy()
    assert (w == np.arange(n_obj)).sum() >= n_obj - 1
    ix.free()
