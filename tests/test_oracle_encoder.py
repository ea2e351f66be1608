"""Pins for the encoder oracle (learned proposal; not part of the paper):
its gradient matches central finite differences of its loss, a single lit
pixel through a stride-2 convolution lands where the padding/stride
definition says, and InfoNCE has the closed form of orthonormal batches."""
import numpy as np
import pytest

from oracle import encoder as oe


def _desc(rng, n, density=0.06):
    bits = (rng.random((n, 64, 64)) < density).astype(np.uint64)
    return (bits << np.arange(64, dtype=np.uint64)).sum(-1).astype(np.uint64)


def test_pixel_layout():
    d = np.zeros((1, 64), np.uint64)
    d[0, 5] = np.uint64(1) << np.uint64(9)          # bit 9 of word 5
    img = oe.bits_to_images(d)
    assert img[0, 0, 5, 9] == 1 and img.sum() == 1


def test_conv_impulse_response():
    """One lit input pixel (r, c): output (y, x) sees weight (ky, kx) with
    r = 2y + ky - 1, c = 2x + kx - 1, nothing else (zero bias)."""
    rng = np.random.default_rng(0)
    w = rng.normal(size=(3, 1, 3, 3))
    for r, c in [(0, 0), (7, 12), (63, 63), (30, 1)]:
        x = np.zeros((1, 1, 64, 64))
        x[0, 0, r, c] = 1.0
        out = oe.conv_s2(x, w, np.zeros(3))
        expect = np.zeros_like(out)
        for ky in range(3):
            for kx in range(3):
                if (r + 1 - ky) % 2 == 0 and (c + 1 - kx) % 2 == 0:
                    y, xx = (r + 1 - ky) // 2, (c + 1 - kx) // 2
                    if 0 <= y < 32 and 0 <= xx < 32:
                        expect[0, :, y, xx] += w[:, 0, ky, kx]
        np.testing.assert_allclose(out, expect, atol=1e-12)


def test_infonce_closed_form():
    tau = 0.1
    e = np.eye(4, 128)
    loss, dq, dt = oe.infonce(e, e, tau)
    expect = np.log(np.exp(1 / tau) + 3.0) - 1 / tau
    assert loss == pytest.approx(expect, rel=1e-12)
    # swapping targets raises the loss to log(e^{1/tau} + 3) - 0
    loss2, _, _ = oe.infonce(e, e[[1, 0, 3, 2]], tau)
    assert loss2 == pytest.approx(np.log(np.exp(1 / tau) + 3.0), rel=1e-12)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    flat = oe.init_params(2, scale=0.5)
    q, t = _desc(rng, 3), _desc(rng, 3)
    loss, g = oe.loss_and_grad(flat, q, t, 0.2)
    # coordinates from every layer
    offs, o = [], 0
    for _, shape in oe.SHAPES:
        n = int(np.prod(shape))
        offs += list(o + rng.choice(n, size=min(n, 6), replace=False))
        o += n
    # a step can straddle a ReLU kink; the derivative must match the central
    # difference at one of three step sizes
    for i in offs:
        nums = []
        for eps in (1e-5, 1e-6, 1e-7):
            fp = flat.copy(); fp[i] += eps
            fm = flat.copy(); fm[i] -= eps
            nums.append((oe.loss_and_grad(fp, q, t, 0.2)[0] -
                         oe.loss_and_grad(fm, q, t, 0.2)[0]) / (2 * eps))
        assert any(abs(g[i] - v) <= 1e-5 * abs(v) + 1e-9 for v in nums), (i, g[i], nums)
