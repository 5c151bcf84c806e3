"""Warm-start network on the GPU: 3 hidden ReLU layers of 256, masked softmax
over at most 8 actions.

FP32 master weights with BF16 copies; every product (forward and both
backward products), the loss, the ReLU gradients, the bias gradients and the
Adam updates run in libcfr.so's kernels (include/mlp.h). PyTorch only holds
the device memory. Weight layout: W[l] is [fan_in, fan_out] row-major, so a
layer is h_out = relu(h_in @ W + b).
"""
from __future__ import annotations

import ctypes
from typing import List, Optional

import numpy as np

from . import cfr

_lib = cfr._lib
_vp, _l, _i = ctypes.c_void_p, ctypes.c_long, ctypes.c_int
_lib.mlp_gemm.argtypes = [_vp, _i, _l, _l, _vp, _i, _l, _l, _vp, _vp, _l, _i, _i, _i, _vp, _i, _i, _vp]
_lib.mlp_softmax_xent.argtypes = [_vp, _i, _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp]
_lib.mlp_relu_grad.argtypes = [_vp, _vp, _l, _vp]
_lib.mlp_colsum.argtypes = [_vp, _i, _i, _vp, _vp]
_lib.mlp_adam.argtypes = [_vp, _vp, _vp, _vp, _l, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _l,
                          _vp, _vp]
_lib.mlp_to_bf16.argtypes = [_vp, _vp, _l, _vp]
for _f in ("mlp_gemm", "mlp_softmax_xent", "mlp_relu_grad", "mlp_colsum", "mlp_adam", "mlp_to_bf16"):
    getattr(_lib, _f).restype = ctypes.c_int
_lib.mlp_last_error.restype = ctypes.c_char_p

N_OUT = 8


def _ck(rc):
    if rc != 0:
        raise RuntimeError("mlp: " + (_lib.mlp_last_error() or b"").decode())


def _p(t) -> int:
    return 0 if t is None else int(t.data_ptr())


class MLP:
    def __init__(self, in_dim: int, hidden=(256, 256, 256), out: int = N_OUT, seed: int = 0, device="cuda"):
        import torch

        self.torch = torch
        self.dev = torch.device(device)
        self.dims = [in_dim] + list(hidden) + [out]
        rng = np.random.default_rng(seed)
        self.W, self.b, self.Wb = [], [], []
        for fi, fo in zip(self.dims[:-1], self.dims[1:]):
            lim = np.sqrt(6.0 / fi)  # He-uniform for ReLU layers
            w = rng.uniform(-lim, lim, size=(fi, fo)).astype(np.float32)
            self.W.append(torch.tensor(w, device=self.dev))
            self.b.append(torch.zeros(fo, dtype=torch.float32, device=self.dev))
            self.Wb.append(torch.empty((fi, fo), dtype=torch.bfloat16, device=self.dev))
        self.gW = [torch.zeros_like(w) for w in self.W]
        self.gb = [torch.zeros_like(b) for b in self.b]
        self.mW = [torch.zeros_like(w) for w in self.W]
        self.vW = [torch.zeros_like(w) for w in self.W]
        self.mb = [torch.zeros_like(b) for b in self.b]
        self.vb = [torch.zeros_like(b) for b in self.b]
        self.step_no = 0
        self.sync_bf16()

    def _s(self) -> int:
        return int(self.torch.cuda.current_stream(self.dev).cuda_stream)

    def sync_bf16(self):
        for w, wb in zip(self.W, self.Wb):
            _ck(_lib.mlp_to_bf16(_p(w), _p(wb), w.numel(), self._s()))

    # ---------------------------------------------------------------- passes
    def forward(self, X) -> "torch.Tensor":
        """X: [B, in_dim] FP32 on the device. Keeps the activations."""
        torch = self.torch
        B = X.shape[0]
        self.acts = [X]
        h = X
        L = len(self.W)
        for l in range(L):
            fo = self.dims[l + 1]
            out = torch.empty((B, fo), dtype=torch.float32, device=self.dev)
            # A(m, k) = h[m, k]; B(k, n) = Wb[k, n]
            _ck(_lib.mlp_gemm(_p(h), 0, h.shape[1], 1, _p(self.Wb[l]), 1, fo, 1, _p(out), None, fo, B, fo,
                              self.dims[l], _p(self.b[l]), 1 if l < L - 1 else 0, 0, self._s()))
            self.acts.append(out)
            h = out
        return h

    def backward(self, dlogits) -> None:
        """Gradients of every weight and bias given d loss / d logits."""
        torch = self.torch
        B = dlogits.shape[0]
        d = dlogits
        for l in range(len(self.W) - 1, -1, -1):
            fi, fo = self.dims[l], self.dims[l + 1]
            h_in = self.acts[l]
            # gW = h_in^T d : A(m=i, k=b) = h_in[b, i]; B(k=b, n=j) = d[b, j]
            _ck(_lib.mlp_gemm(_p(h_in), 0, 1, fi, _p(d), 0, fo, 1, _p(self.gW[l]), None, fo, fi, fo, B, None, 0, 0,
                              self._s()))
            _ck(_lib.mlp_colsum(_p(d), B, fo, _p(self.gb[l]), self._s()))
            if l > 0:
                dh = torch.empty((B, fi), dtype=torch.float32, device=self.dev)
                # dh = d W^T : A(m=b, k=j) = d[b, j]; B(k=j, n=i) = Wb[i, j]
                _ck(_lib.mlp_gemm(_p(d), 0, fo, 1, _p(self.Wb[l]), 1, 1, fo, _p(dh), None, fi, B, fi, fo, None, 0, 0,
                                  self._s()))
                _ck(_lib.mlp_relu_grad(_p(dh), _p(h_in), dh.numel(), self._s()))
                d = dh

    def loss_and_grad(self, X, nact, target, weight=None) -> float:
        torch = self.torch
        logits = self.forward(X)
        B = X.shape[0]
        dlog = torch.empty_like(logits)
        rows = torch.empty(B, dtype=torch.float32, device=self.dev)
        _ck(_lib.mlp_softmax_xent(_p(logits), N_OUT, _p(nact), _p(target), _p(weight), B, None, _p(dlog), _p(rows),
                                  self._s()))
        self.backward(dlog)
        return float(rows.sum().item()) / B

    def adam_step(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8) -> None:
        self.step_no += 1
        for w, g, m, v, wb in zip(self.W, self.gW, self.mW, self.vW, self.Wb):
            _ck(_lib.mlp_adam(_p(w), _p(g), _p(m), _p(v), w.numel(), lr, b1, b2, eps, self.step_no, _p(wb), self._s()))
        for b, g, m, v in zip(self.b, self.gb, self.mb, self.vb):
            _ck(_lib.mlp_adam(_p(b), _p(g), _p(m), _p(v), b.numel(), lr, b1, b2, eps, self.step_no, None, self._s()))

    def predict(self, X, nact) -> "torch.Tensor":
        torch = self.torch
        logits = self.forward(X)
        prob = torch.empty_like(logits)
        _ck(_lib.mlp_softmax_xent(_p(logits), N_OUT, _p(nact), None, None, X.shape[0], _p(prob), None, None,
                                  self._s()))
        return prob

    # ------------------------------------------------------------ host copies
    def numpy_params(self):
        return ([w.cpu().numpy().astype(np.float64) for w in self.W],
                [b.cpu().numpy().astype(np.float64) for b in self.b])

    def numpy_grads(self):
        return ([g.cpu().numpy().astype(np.float64) for g in self.gW],
                [g.cpu().numpy().astype(np.float64) for g in self.gb])
