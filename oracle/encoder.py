"""Oracle of the learned proposal's encoder and loss — TEST INFRASTRUCTURE.

Plain numpy in FP64, written from the layer definitions (the paper has no
learned component; the network is the one the library's encoder kernels
implement: 3x3 stride-2 convolutions with zero padding 1 and ReLU, 2x2
average pooling, two dense layers, unit-length output; InfoNCE with
in-batch negatives).  Used only by tests to check the GPU forward pass and
the hand-written GPU gradients; pinned by finite differences.
"""
from __future__ import annotations

import numpy as np

SHAPES = [("w1", (32, 1, 3, 3)), ("b1", (32,)), ("w2", (64, 32, 3, 3)), ("b2", (64,)),
          ("w3", (64, 64, 3, 3)), ("b3", (64,)), ("wf1", (256, 1024)), ("bf1", (256,)),
          ("wf2", (128, 256)), ("bf2", (128,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(flat):
    flat = np.asarray(flat, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[o:o + n].reshape(shape)
        o += n
    assert o == flat.size
    return out


def flatten(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bits_to_images(desc):
    """uint64 [n, 64] -> float [n, 1, 64, 64]; pixel (r, c) = bit c of word r."""
    d = np.ascontiguousarray(desc, dtype=np.uint64).reshape(-1, 64)
    bits = (d[:, :, None] >> np.arange(64, dtype=np.uint64)[None, None, :]) & np.uint64(1)
    return bits.astype(np.float64)[:, None, :, :]


def conv_s2(x, w, b):
    """out[n,o,y,x] = b[o] + sum_{c,ky,kx} w[o,c,ky,kx] xpad[n,c,2y+ky,2x+kx]."""
    n, c, h, _ = x.shape
    ho = h // 2
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    out = np.zeros((n, w.shape[0], ho, ho)) + b[None, :, None, None]
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + 2 * ho:2, kx:kx + 2 * ho:2]
            out += np.einsum("nchw,oc->nohw", patch, w[:, :, ky, kx])
    return out


def conv_s2_backward(x, w, dout):
    """Gradients of conv_s2 with respect to x, w and b."""
    n, c, h, _ = x.shape
    ho = h // 2
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + 2 * ho:2, kx:kx + 2 * ho:2]
            dw[:, :, ky, kx] = np.einsum("nohw,nchw->oc", dout, patch)
            dxp[:, :, ky:ky + 2 * ho:2, kx:kx + 2 * ho:2] += np.einsum("nohw,oc->nchw", dout,
                                                                        w[:, :, ky, kx])
    return dxp[:, :, 1:-1, 1:-1], dw, dout.sum(axis=(0, 2, 3))


def pool2(x):
    n, c, h, _ = x.shape
    return x.reshape(n, c, h // 2, 2, h // 2, 2).mean(axis=(3, 5))


def forward(p, desc):
    """Returns (embeddings e [n,128], cache for backward)."""
    x0 = bits_to_images(desc)
    a1 = np.maximum(conv_s2(x0, p["w1"], p["b1"]), 0)
    a2 = np.maximum(conv_s2(a1, p["w2"], p["b2"]), 0)
    a3 = np.maximum(conv_s2(a2, p["w3"], p["b3"]), 0)
    f = pool2(a3).reshape(a3.shape[0], -1)
    h = np.maximum(f @ p["wf1"].T + p["bf1"], 0)
    z = h @ p["wf2"].T + p["bf2"]
    nz = np.linalg.norm(z, axis=1, keepdims=True)
    e = z / np.maximum(nz, 1e-12)
    return e, dict(x0=x0, a1=a1, a2=a2, a3=a3, f=f, h=h, z=z, nz=nz, e=e)


def backward(p, c, de):
    """Gradient of a scalar with d(scalar)/de = de, for every parameter."""
    g = {}
    dz = (de - c["e"] * np.sum(c["e"] * de, axis=1, keepdims=True)) / c["nz"]
    g["wf2"] = dz.T @ c["h"]
    g["bf2"] = dz.sum(0)
    dh = (dz @ p["wf2"]) * (c["h"] > 0)
    g["wf1"] = dh.T @ c["f"]
    g["bf1"] = dh.sum(0)
    df = (dh @ p["wf1"]).reshape(c["a3"].shape[0], 64, 4, 4)
    da3 = np.repeat(np.repeat(df, 2, axis=2), 2, axis=3) / 4.0 * (c["a3"] > 0)
    da2, g["w3"], g["b3"] = conv_s2_backward(c["a2"], p["w3"], da3)
    da2 = da2 * (c["a2"] > 0)
    da1, g["w2"], g["b2"] = conv_s2_backward(c["a1"], p["w2"], da2)
    da1 = da1 * (c["a1"] > 0)
    _, g["w1"], g["b1"] = conv_s2_backward(c["x0"], p["w1"], da1)
    return g


def infonce(eq, et, tau):
    """Mean over i of log sum_j exp(s_ij) - s_ii with s = eq et^T / tau;
    returns (loss, d loss / d eq, d loss / d et)."""
    s = eq @ et.T / tau
    m = s.max(axis=1, keepdims=True)
    pr = np.exp(s - m)
    pr /= pr.sum(axis=1, keepdims=True)
    B = s.shape[0]
    loss = float(np.mean(m[:, 0] + np.log(np.exp(s - m).sum(axis=1)) - np.diag(s)))
    ds = (pr - np.eye(B)) / B
    return loss, ds @ et / tau, ds.T @ eq / tau


def loss_and_grad(flat, qdesc, tdesc, tau):
    """InfoNCE loss of a batch of (query, target) pairs and its gradient."""
    p = unflatten(flat)
    eq, cq = forward(p, qdesc)
    et, ct = forward(p, tdesc)
    loss, deq, det = infonce(eq, et, tau)
    gq, gt = backward(p, cq, deq), backward(p, ct, det)
    return loss, flatten({k: gq[k] + gt[k] for k in gq})


def init_params(seed, scale=1.0):
    """He-uniform-like random parameters for tests (not the library's init)."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SHAPES:
        if name.startswith("b"):
            d[name] = rng.uniform(-0.1, 0.1, size=shape) * scale
        else:
            fan_in = int(np.prod(shape[1:]))
            lim = np.sqrt(6.0 / fan_in)
            d[name] = rng.uniform(-lim, lim, size=shape) * scale
    return flatten(d)
