"""Learned proposal: Python binding of the encoder and inverted-file entry
points of libdt.so (argument marshalling only), and the training loop that
drives them.

Training pairs are (query, exact nearest neighbour) found by the library's
own exact search; the loss is InfoNCE with in-batch negatives.  Every step
runs in the library's kernels (forward, backward and Adam).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import dt

_ready = False


def _lib():
    global _ready
    lib = dt.load()
    if not _ready:
        P, i64, i32, u64, f32 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                 ctypes.c_float)
        sig = {
            "enc_create": ([u64, P], ctypes.c_int),
            "enc_free": ([P], None),
            "enc_param_count": ([], i64),
            "enc_get_params": ([P, P], ctypes.c_int),
            "enc_set_params": ([P, P], ctypes.c_int),
            "enc_get_grads": ([P, P], ctypes.c_int),
            "enc_embed": ([P, P, i64, P, P, i32, P], ctypes.c_int),
            "enc_train_step": ([P, P, P, i32, f32, f32, i32, P, P], ctypes.c_int),
            "ivf_build": ([P, P, i64, i32, i32, P, P], ctypes.c_int),
            "ivf_free": ([P], None),
            "ivf_offsets": ([P, P], ctypes.c_int),
            "ivf_search": ([P, P, P, i64, i32, i32, P, P, P, i32, P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _ready = True
    return lib


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Encoder:
    def __init__(self, seed=1):
        h = ctypes.c_void_p()
        dt._check(_lib().enc_create(seed, ctypes.byref(h)), "enc_create")
        self._h = h
        self.n_params = int(_lib().enc_param_count())

    @property
    def handle(self):
        return self._h

    def get_params(self):
        out = np.empty(self.n_params, np.float32)
        dt._check(_lib().enc_get_params(self._h, ctypes.c_void_p(out.ctypes.data)), "enc_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        dt._check(_lib().enc_set_params(self._h, ctypes.c_void_p(p.ctypes.data)), "enc_set_params")

    def get_grads(self):
        out = np.empty(self.n_params, np.float32)
        dt._check(_lib().enc_get_grads(self._h, ctypes.c_void_p(out.ctypes.data)), "enc_get_grads")
        return out

    def embed(self, bits, bf16=False, path=0, stream=None):
        """path: 0 auto, 1 FP32 on CUDA cores, 2 tensor cores (BF16 operands)."""
        bits = dt._desc(bits, "bits")
        n = bits.shape[0]
        if bf16:
            out = torch.empty((n, 128), dtype=torch.int16, device=bits.device)
            dt._check(_lib().enc_embed(self._h, _p(bits), n, _p(out), None, path,
                                       dt._stream(stream)), "enc_embed")
            return out.view(torch.bfloat16)
        out = torch.empty((n, 128), dtype=torch.float32, device=bits.device)
        dt._check(_lib().enc_embed(self._h, _p(bits), n, None, _p(out), path, dt._stream(stream)),
                  "enc_embed")
        return out

    def train_step(self, q, t, lr=1e-3, tau=0.05, update=True, want_loss=True, stream=None):
        q, t = dt._desc(q, "q"), dt._desc(t, "t")
        loss = ctypes.c_float()
        dt._check(_lib().enc_train_step(self._h, _p(q), _p(t), q.shape[0], lr, tau,
                                        1 if update else 0,
                                        ctypes.byref(loss) if want_loss else None,
                                        dt._stream(stream)), "enc_train_step")
        return loss.value if want_loss else None

    def free(self):
        if self._h is not None:
            _lib().enc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class IVF:
    def __init__(self, enc: Encoder, db, n_lists=4096, iters=4, stream=None):
        db = dt._desc(db, "db")
        h = ctypes.c_void_p()
        dt._check(_lib().ivf_build(enc.handle, _p(db), db.shape[0], n_lists, iters,
                                   dt._stream(stream), ctypes.byref(h)), "ivf_build")
        self._h = h
        self.enc = enc
        self.n_lists = n_lists

    def offsets(self):
        out = np.empty(self.n_lists + 1, np.int64)
        dt._check(_lib().ivf_offsets(self._h, ctypes.c_void_p(out.ctypes.data)), "ivf_offsets")
        return out

    def search(self, q, k, n_probe, with_scanned=False, path=0, stream=None):
        """path: 0 auto, 1 CUDA cores (a block per query), 2 tensor cores
        (list-major); identical results."""
        q = dt._desc(q, "q")
        nq = q.shape[0]
        idx = torch.empty((nq, k), dtype=torch.int32, device=q.device)
        score = torch.empty((nq, k), dtype=torch.float32, device=q.device)
        scanned = torch.empty(nq, dtype=torch.int64, device=q.device) if with_scanned else None
        dt._check(_lib().ivf_search(self._h, self.enc.handle, _p(q), nq, k, n_probe, _p(idx),
                                    _p(score), _p(scanned), path, dt._stream(stream)),
                  "ivf_search")
        return idx, score, scanned

    def free(self):
        if self._h is not None:
            _lib().ivf_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def train(enc: Encoder, d_db, make_queries, steps, batch=256, lr=1e-3, tau=0.05, log=None,
          epochs_per_round=1, seed=0):
    """Train on (query, exact nearest neighbour) pairs.

    make_queries(round) -> uint64 numpy [m, 64] new query descriptors; their
    exact nearest neighbours come from bf_search on d_db, and each round's
    pairs are used for epochs_per_round passes (reshuffled by a generator
    seeded with `seed`, so that the same inputs train the same weights).
    Returns the loss history."""
    losses = []
    step = 0
    rnd = 0
    rng = np.random.default_rng(seed)
    while step < steps:
        q = make_queries(rnd)
        rnd += 1
        d_q = torch.from_numpy(np.ascontiguousarray(q).view(np.int64)).to(d_db.device)
        nn, _, _ = dt.bf_search(d_db, d_q, 1)
        tgt = d_db[nn[:, 0].long()]
        for _ in range(epochs_per_round):
            perm = torch.from_numpy(rng.permutation(d_q.shape[0])).to(d_q.device)
            for b0 in range(0, d_q.shape[0] - batch + 1, batch):
                if step >= steps:
                    break
                sel = perm[b0:b0 + batch]
                want = (step % 20 == 0) or step == steps - 1
                loss = enc.train_step(d_q[sel].contiguous(), tgt[sel].contiguous(), lr=lr,
                                      tau=tau, want_loss=want)
                if want:
                    losses.append((step, loss))
                    if log:
                        log(step, loss)
                step += 1
    return losses
