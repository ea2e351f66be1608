"""Pins for the oracle's QUICCI generation (§2.2) and the modified QUICCI of
§5, with the geometry of reading R15 (layer l at height -R + (2l + 1) R / 64
along the normal, circle c of radius (c + 1) R / 64).

Closed forms, on flat meshes placed so that no circle or layer meets a vertex
or a triangle edge exactly:
- a plane containing the axis: every circle meets it twice, so only the
  innermost circle's bit changes (0 -> 2) in every layer;
- a plane parallel to the axis at distance d: circles with r > d meet it
  twice, so the one bit per layer is the first circle larger than d;
- a half-plane whose boundary runs parallel to the axis at distance d: one
  crossing, a change of 1 — set in the QUICCI, dropped by the modification;
- a flat strip limited in height: only the layers whose plane crosses it.
Brute force: on random triangles, counts found by sampling each circle at
4,096 angles and locating where it pierces each triangle (barycentric test,
no layer segments) give the oracle's bits, away from near-tangent circles.
Invariants: a circle meets a closed surface an even number of times, so on a
closed mesh the modified QUICCI equals the QUICCI; the modified QUICCI is a
subset of the QUICCI; rotating the mesh by 90 degrees about the normal,
scaling everything by 2 and mirroring the heights (layers reversed) change
nothing else; a point out of reach and a zero normal give empty images.
"""
import numpy as np
import pytest

import oracle
from paper_2107_03368_gb300 import synth

R = 100.0
N = 64


def quad(x0, x1, y, z0, z1):
    """Rectangle x in [x0, x1], z in [z0, z1] in the plane y = const, as two
    triangles (split along the diagonal (x0, z0) - (x1, z1))."""
    v = np.array([[x0, y, z0], [x1, y, z0], [x1, y, z1], [x0, y, z1]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return v, t


AXIS_P = np.zeros((1, 3), np.float32)
AXIS_N = np.array([[0, 0, 1]], np.float32)


def bits(img):
    return np.unpackbits(np.ascontiguousarray(img).view(np.uint8), bitorder="little").reshape(
        -1, N, N)


@pytest.mark.parametrize("modified", [False, True])
def test_plane_through_axis(modified):
    v, t = quad(-170.0, 230.0, 0.0, -200.0, 200.0)
    img = oracle.quicci(v, t, AXIS_P, AXIS_N, R, modified)
    assert np.all(img[0] == np.uint64(1))           # bit 0 of every layer


@pytest.mark.parametrize("modified", [False, True])
@pytest.mark.parametrize("d", [37.0, 0.7, 99.1])
def test_plane_parallel_to_axis(d, modified):
    v, t = quad(-170.0, 230.0, d, -200.0, 200.0)
    img = oracle.quicci(v, t, AXIS_P, AXIS_N, R, modified)
    c = int(np.floor(d * N / R))                     # first circle with radius > d
    assert (c + 1) * R / N > d >= c * R / N
    assert np.all(img[0] == np.uint64(1) << np.uint64(c))


def test_half_plane_boundary_is_filtered():
    d = 37.0
    v, t = quad(0.0, 230.0, d, -200.0, 200.0)
    full = oracle.quicci(v, t, AXIS_P, AXIS_N, R, False)
    mod = oracle.quicci(v, t, AXIS_P, AXIS_N, R, True)
    assert np.all(full[0] == np.uint64(1) << np.uint64(23))
    assert np.all(mod == 0)


def test_layers_follow_height():
    z0, z1 = -20.3, 45.1
    v, t = quad(-170.0, 230.0, 0.0, z0, z1)
    img = oracle.quicci(v, t, AXIS_P, AXIS_N, R, False)[0]
    zl = -R + (2 * np.arange(N) + 1) * R / N
    expect = (zl > z0) & (zl <= z1)
    # worked by hand: z_26 = -17.1875 is the first above -20.3 (z_25 = -20.3125),
    # z_45 = 43.75 the last at or below 45.1 (z_46 = 46.875)
    assert np.array_equal(np.flatnonzero(expect), np.arange(26, 46))
    assert np.array_equal(img != 0, expect)
    assert np.all(img[expect] == np.uint64(1))
    # the same strip seen with the normal reversed: layers in reverse order
    flip = oracle.quicci(v, t, AXIS_P, -AXIS_N, R, False)[0]
    assert np.array_equal(flip != 0, ((-zl) >= z0) & ((-zl) < z1))


def test_closed_mesh_counts_are_even():
    v, t, n = synth.mesh_object(3, 3)
    pick = np.arange(0, v.shape[0], 7)
    full = oracle.quicci(v, t, v[pick], n[pick], R, False)
    mod = oracle.quicci(v, t, v[pick], n[pick], R, True)
    assert np.array_equal(full, mod)
    assert bits(full).sum(axis=(1, 2)).mean() > 20      # descriptors are not empty


def test_partial_mesh_modified_is_subset():
    v, t, n = synth.mesh_object(4, 3)
    pv, pt, pn, _ = synth.mesh_partial(5, v, t)
    pick = np.arange(0, pv.shape[0], 5)
    full = oracle.quicci(pv, pt, pv[pick], pn[pick], R, False)
    mod = oracle.quicci(pv, pt, pv[pick], pn[pick], R, True)
    assert np.all((mod & ~full) == 0)
    assert bits(mod).sum() < bits(full).sum()            # boundary responses dropped


def test_rotation_scale_and_far_points():
    v, t, _ = synth.mesh_object(6, 3)
    rng = np.random.default_rng(6)
    p = v[rng.integers(0, v.shape[0], 40)] + rng.normal(0, 3, (40, 3)).astype(np.float32)
    p = p.astype(np.float32)
    nz = np.tile(np.array([[0, 0, 1]], np.float32), (40, 1))
    base = oracle.quicci(v, t, p, nz, R, False)
    # 90 degrees about the z axis through each point: (x, y) -> (-y, x)
    for j in range(0, 40, 8):
        rel = v - p[j]
        rot = np.stack([-rel[:, 1], rel[:, 0], rel[:, 2]], 1) + p[j]
        one = oracle.quicci(rot.astype(np.float32), t, p[j:j + 1], nz[:1], R, False)
        assert np.array_equal(one[0], base[j])
    twice = oracle.quicci(2 * v, t, 2 * p, nz, 2 * R, False)
    assert np.array_equal(twice, base)
    far = oracle.quicci(v, t, np.array([[5000, 0, 0]], np.float32), nz[:1], R, False)
    zero_n = oracle.quicci(v, t, p[:1], np.zeros((1, 3), np.float32), R, False)
    assert np.all(far == 0) and np.all(zero_n == 0)
    assert bits(base).sum() > 0


def _sampled_counts(v, t, layers, samples=4096):
    """Intersection counts of every circle of the given layers with the mesh,
    found without layer segments: each circle (axis z through the origin) is
    sampled at `samples` angles, and a point where it passes through a
    triangle's plane, inside the triangle, is one intersection."""
    th = np.linspace(0.0, 2 * np.pi, samples + 1)[:-1]
    cos, sin = np.cos(th), np.sin(th)
    counts = np.zeros((len(layers), N), np.int64)
    tri = v[t].astype(np.float64)
    for li, l in enumerate(layers):
        zl = -R + (2 * l + 1) * R / N
        for c in range(N):
            r = (c + 1) * R / N
            pts = np.stack([r * cos, r * sin, np.full_like(cos, zl)], 1)
            for a, b, cc in tri:
                nrm = np.cross(b - a, cc - a)
                f = (pts - a) @ nrm
                f2 = np.roll(f, -1)
                for i in np.flatnonzero(np.sign(f) != np.sign(f2)):
                    s = f[i] / (f[i] - f2[i])
                    x = pts[i] + s * (pts[(i + 1) % samples] - pts[i])
                    # barycentric inside test
                    v0, v1, v2 = b - a, cc - a, x - a
                    d00, d01, d11 = v0 @ v0, v0 @ v1, v1 @ v1
                    d20, d21 = v2 @ v0, v2 @ v1
                    den = d00 * d11 - d01 * d01
                    bu = (d11 * d20 - d01 * d21) / den
                    bv = (d00 * d21 - d01 * d20) / den
                    if bu >= 0 and bv >= 0 and bu + bv <= 1:
                        counts[li, c] += 1
    return counts


def test_counts_against_sampled_circles():
    """Random triangles crossing the support cylinder: bits from counts found by
    sampling each circle equal the oracle's, away from near-tangent circles."""
    rng = np.random.default_rng(8)
    layers = [5, 20, 31, 32, 44, 60]
    checked = 0
    for trial in range(3):
        cen = rng.uniform(-60, 60, (5, 3))
        v = (cen[:, None, :] + rng.normal(0, 35, (5, 3, 3))).reshape(-1, 3).astype(np.float32)
        t = np.arange(15, dtype=np.int32).reshape(5, 3)
        img = oracle.quicci(v, t, AXIS_P, AXIS_N, R, False)[0]
        lo = oracle.quicci(v, t, AXIS_P, AXIS_N, R * (1 - 1e-4), False)[0]
        hi = oracle.quicci(v, t, AXIS_P, AXIS_N, R * (1 + 1e-4), False)[0]
        cnt = _sampled_counts(v, t, layers)
        for li, l in enumerate(layers):
            d = np.diff(np.concatenate([[0], cnt[li]]))
            word = np.uint64(0)
            for c in np.flatnonzero(d != 0):
                word |= np.uint64(1) << np.uint64(c)
            unsure = (img[l] ^ lo[l]) | (img[l] ^ hi[l])
            assert (word ^ img[l]) & ~unsure == 0, (trial, l)
            checked += int(img[l] != 0)
    assert checked >= 6                      # the triangles reach several layers
