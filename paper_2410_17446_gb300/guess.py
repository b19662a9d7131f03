"""Learned GMRES initial guess: the network of include/prop_cnn.h driven from Python.

Argument marshalling and call sequencing only: every convolution, gradient,
loss and optimiser update runs in the library's CUDA kernels.  Buffers are
torch tensors (device memory); the stream is torch's current stream.

Layers: channels[0] -> ... -> channels[-1], each 16 or 32 wide (narrower
inputs and outputs are zero-padded to 16), 3x3 circular convolutions, ReLU
between layers.  Parameters are float32 masters with bfloat16 copies.
"""
from __future__ import annotations

import ctypes as ct
from typing import List, Optional, Sequence

import numpy as np

from . import prop as P

C_OK = 0


def _chk(rc, where):
    if rc != C_OK:
        raise RuntimeError(f"{where}: status {rc}")


class GuessNet:
    def __init__(self, channels: Sequence[int], seed: int = 0, device: str = "cuda",
                 weights: Optional[List[np.ndarray]] = None, biases: Optional[List[np.ndarray]] = None):
        import torch
        self.torch = torch
        self.channels = list(channels)
        for c in self.channels:
            if c not in (16, 32):
                raise ValueError("channel widths must be 16 or 32")
        self.L = len(self.channels) - 1
        rng = np.random.default_rng(seed)
        self.w32, self.b32, self.wbf, self.m, self.v = [], [], [], [], []
        for l, (ci, co) in enumerate(zip(self.channels[:-1], self.channels[1:])):
            if weights is not None:
                w = np.asarray(weights[l], np.float32)
                b = np.asarray(biases[l], np.float32)
            else:
                w = (rng.standard_normal((9, co, ci)) * np.sqrt(2.0 / (9 * ci))).astype(np.float32)
                b = np.zeros(co, np.float32)
            self.w32.append(torch.tensor(w, device=device))
            self.b32.append(torch.tensor(b, device=device))
            self.wbf.append(self.w32[-1].to(torch.bfloat16))
            self.m.append((torch.zeros_like(self.w32[-1]), torch.zeros_like(self.b32[-1])))
            self.v.append((torch.zeros_like(self.w32[-1]), torch.zeros_like(self.b32[-1])))
        self.step_count = 0

    def _stream(self):
        return self.torch.cuda.current_stream().cuda_stream

    # ---- forward ----------------------------------------------------------
    def forward(self, x, keep: bool = False, active=None, active_stride: int = 1, active_want: int = 1):
        """x: bf16 [N, H, W, channels[0]] -> float32 [N, H, W, channels[-1]] (and the activations)."""
        torch = self.torch
        N, H, W, _ = x.shape
        acts = [x]
        a = x
        for l in range(self.L):
            ci, co = self.channels[l], self.channels[l + 1]
            last = l == self.L - 1
            out = torch.empty((N, H, W, co), dtype=torch.float32 if last else torch.bfloat16, device=x.device)
            if active is not None:
                out.zero_()
            mode = 2 if last else 0
            _chk(P.lib().prop_cnn_conv(ci, co, mode, a.data_ptr(), self.wbf[l].data_ptr(), self.b32[l].data_ptr(),
                                       out.data_ptr(), N, H, W, active.data_ptr() if active is not None else None,
                                       active_stride, active_want, self._stream()), "prop_cnn_conv")
            acts.append(out)
            a = out
        return (a, acts) if keep else a

    # ---- backward ---------------------------------------------------------
    def backward(self, acts, grad_out_bf16):
        """Gradients of every layer for dloss/d(output) = grad_out (bf16 [N,H,W,C_L])."""
        torch = self.torch
        N, H, W, _ = acts[0].shape
        dws, dbs = [None] * self.L, [None] * self.L
        g = grad_out_bf16
        for l in range(self.L - 1, -1, -1):
            ci, co = self.channels[l], self.channels[l + 1]
            if l < self.L - 1:   # ReLU derivative from the stored activation a_{l+1}
                _chk(P.lib().prop_cnn_relu_mask(g.data_ptr(), acts[l + 1].data_ptr(), g.numel(), self._stream()),
                     "prop_cnn_relu_mask")
            n = ct.c_size_t()
            _chk(P.lib().prop_cnn_wgrad_workspace(ci, co, N, H, W, ct.byref(n)), "prop_cnn_wgrad_workspace")
            work = torch.empty(n.value, dtype=torch.uint8, device=g.device)
            dw = torch.empty((9, co, ci), dtype=torch.float32, device=g.device)
            db = torch.empty((co,), dtype=torch.float32, device=g.device)
            _chk(P.lib().prop_cnn_wgrad(ci, co, g.data_ptr(), acts[l].data_ptr(), N, H, W, dw.data_ptr(),
                                        db.data_ptr(), work.data_ptr(), n.value, self._stream()), "prop_cnn_wgrad")
            dws[l], dbs[l] = dw, db
            if l > 0:
                wt = torch.empty((9, ci, co), dtype=torch.bfloat16, device=g.device)
                _chk(P.lib().prop_cnn_flip_transpose(self.wbf[l].data_ptr(), wt.data_ptr(), co, ci, self._stream()),
                     "prop_cnn_flip_transpose")
                gi = torch.empty((N, H, W, ci), dtype=torch.bfloat16, device=g.device)
                _chk(P.lib().prop_cnn_conv(co, ci, 1, g.data_ptr(), wt.data_ptr(), None, gi.data_ptr(), N, H, W,
                                           None, 1, 1, self._stream()), "prop_cnn_conv(data grad)")
                g = gi
        return dws, dbs

    def mse(self, out, target, valid: int):
        """(loss tensor[1] float64, bf16 gradient) of 0.5 sum_valid (out - target)^2 / npix."""
        torch = self.torch
        N, H, W, C = out.shape
        grad = torch.empty(out.shape, dtype=torch.bfloat16, device=out.device)
        loss = torch.zeros(1, dtype=torch.float64, device=out.device)
        _chk(P.lib().prop_cnn_mse(out.data_ptr(), target.data_ptr(), grad.data_ptr(), N * H * W, C, valid,
                                  loss.data_ptr(), self._stream()), "prop_cnn_mse")
        return loss, grad

    def adam(self, dws, dbs, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        for l in range(self.L):
            for p, gr, m, v, pb in ((self.w32[l], dws[l], self.m[l][0], self.v[l][0], self.wbf[l]),
                                    (self.b32[l], dbs[l], self.m[l][1], self.v[l][1], None)):
                _chk(P.lib().prop_cnn_adam(p.data_ptr(), gr.data_ptr(), m.data_ptr(), v.data_ptr(), p.numel(),
                                           lr, b1, b2, eps, self.step_count, pb.data_ptr() if pb is not None else None,
                                           self._stream()), "prop_cnn_adam")

    def state(self):
        return {"channels": self.channels,
                "weights": [w.cpu().numpy() for w in self.w32], "biases": [b.cpu().numpy() for b in self.b32]}
