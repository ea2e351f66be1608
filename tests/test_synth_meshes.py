"""The synthetic meshes that stand in for SHREC'16 scans (inputs of QUICCI
generation): a complete object is a closed, consistently oriented surface
(every edge shared by exactly two triangles, traversed once in each
direction), with outward unit vertex normals; a partial view is an open
surface (it has boundary edges) made of the complete mesh's own vertices."""
import numpy as np

from paper_2107_03368_gb300 import synth


def edge_counts(t):
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    directed = {tuple(x) for x in e.tolist()}
    und = np.sort(e, axis=1)
    _, cnt = np.unique(und, axis=0, return_counts=True)
    return directed, e, cnt


def test_complete_mesh_is_closed_and_oriented():
    v, t, n = synth.mesh_object(3, 3)
    assert v.dtype == np.float32 and t.dtype == np.int32 and n.dtype == np.float32
    assert t.min() == 0 and t.max() == v.shape[0] - 1
    directed, e, cnt = edge_counts(t)
    assert np.all(cnt == 2)                           # closed 2-manifold
    assert len(directed) == e.shape[0]                # each directed edge once
    assert all((b, a) in directed for a, b in directed)
    assert v.shape[0] - e.shape[0] // 2 + t.shape[0] == 2   # Euler characteristic of a sphere
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-5)
    c = v.mean(0)
    assert np.mean(np.sum((v - c) * n, axis=1) > 0) > 0.95  # normals point outward


def test_partial_view_is_open_and_reuses_vertices():
    v, t, n = synth.mesh_object(4, 3)
    pv, pt, pn, used = synth.mesh_partial(5, v, t)
    assert 0 < pt.shape[0] < t.shape[0]
    _, _, cnt = edge_counts(pt)
    assert np.any(cnt == 1) and np.all(cnt <= 2)     # boundaries, still a manifold
    assert np.array_equal(pv, v[used])
    np.testing.assert_allclose(np.linalg.norm(pn, axis=1), 1.0, atol=1e-5)


def test_meshes_are_seeded():
    a = synth.mesh_object(7, 2)
    b = synth.mesh_object(7, 2)
    c = synth.mesh_object(8, 2)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0])
