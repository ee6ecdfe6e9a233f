"""Python binding of the learned warm start (3-D conv net + warm-started CG).

Argument marshalling around the mrcm_net_* and mrcm_pcg_mbf entry points of
libmrcm; PyTorch only provides the device buffers and the stream.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L
from .solver import _ptr, _stream


class WarmStartNet:
    """Network of `layers` 3x3x3 convolutions on D x H x W boxes (4 input channels)."""

    def __init__(self, D, H, W, hidden=32, layers=4, in_channels=4, batch=256, device="cuda", seed=0):
        self.lib = L.load()
        h = C.c_void_p()
        L.check(self.lib.mrcm_net_create(in_channels, hidden, layers, D, H, W, C.byref(h)))
        self.net = h
        self.shape = (D, H, W)
        self.S = D * H * W
        self.in_channels = in_channels
        self.batch = batch
        self.device = torch.device(device)
        p, sf, wsb = C.c_size_t(), C.c_size_t(), C.c_size_t()
        L.check(self.lib.mrcm_net_query(self.net, batch, C.byref(p), C.byref(sf), C.byref(wsb)))
        self.n_params = int(p.value)
        self.state = torch.zeros(int(sf.value), dtype=torch.float32, device=self.device)
        self.ws = torch.empty(int(wsb.value), dtype=torch.uint8, device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.step = 0
        L.check(self.lib.mrcm_net_init(self.net, _ptr(self.state), C.c_ulonglong(seed), _stream()))

    def __del__(self):
        try:
            self.lib.mrcm_net_destroy(self.net)
        except Exception:
            pass

    @property
    def master(self):
        return self.state[: self.n_params]

    def forward(self, x):
        n = x.shape[0]
        assert n <= self.batch and x.is_contiguous() and x.dtype == torch.float32
        y = torch.empty((n, 1) + self.shape, dtype=torch.float32, device=self.device)
        L.check(self.lib.mrcm_net_forward(self.net, _ptr(self.state), _ptr(x), _ptr(y), n, _ptr(self.ws), _stream()))
        return y

    def gradient(self, x, target, weight=None):
        n = x.shape[0]
        grad = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        L.check(self.lib.mrcm_net_gradient(self.net, _ptr(self.state), _ptr(x), _ptr(target),
                                           _ptr(weight) if weight is not None else None, n, _ptr(grad),
                                           _ptr(self.loss), _ptr(self.ws), _stream()))
        return grad, self.loss

    def train_step(self, x, target, lr=1e-3, weight=None):
        self.step += 1
        L.check(self.lib.mrcm_net_train_step(self.net, _ptr(self.state), _ptr(x), _ptr(target),
                                             _ptr(weight) if weight is not None else None, x.shape[0],
                                             C.c_float(lr), self.step, _ptr(self.loss), _ptr(self.ws), _stream()))
        return self.loss

    def flux_weights(self, solver, n_samples):
        """Face-flux loss weights (sum of T_R^2 over each cell's Robin faces) of the first n samples."""
        w = torch.empty((n_samples, 1) + self.shape, dtype=torch.float32, device=self.device)
        L.check(self.lib.mrcm_net_flux_weights(solver.handle, self.net, solver.ws_ptr, _ptr(w), n_samples,
                                               _stream()), solver.handle)
        return w

    def set_output_bias(self, mean_target):
        """Start the logistic output at the training targets' mean."""
        import math
        m = min(max(float(mean_target), 1e-4), 1 - 1e-4)
        self.master[self.n_params - 1] = math.log(m / (1.0 - m))
        self.sync_weights()

    def sync_weights(self):
        L.check(self.lib.mrcm_net_sync_weights(self.net, _ptr(self.state), _stream()))

    def bf16_weights(self):
        """The BF16 copy the convolutions use, as FP32 values."""
        off = 3 * self.n_params
        raw = self.state[off: off + (self.n_params + 1) // 2].view(torch.bfloat16)
        return raw[: self.n_params].float()

    # ---- MRCM side
    def samples(self, solver, max_samples=None, targets=True):
        """(x, target) of every P-MBF of the solver's subdomains with this box shape
        (target None with targets=False: inputs only, after factor_local)."""
        n = C.c_int()
        L.check(self.lib.mrcm_net_samples(solver.handle, self.net, solver.ws_ptr, None, None, 1 << 30, C.byref(n),
                                          _stream()), solver.handle)
        cnt = n.value if max_samples is None else min(n.value, max_samples)
        x = torch.empty((cnt, self.in_channels) + self.shape, dtype=torch.float32, device=self.device)
        t = torch.empty((cnt, 1) + self.shape, dtype=torch.float32, device=self.device) if targets else None
        L.check(self.lib.mrcm_net_samples(solver.handle, self.net, solver.ws_ptr, _ptr(x),
                                          _ptr(t) if t is not None else None, cnt, C.byref(n), _stream()),
                solver.handle)
        return x, t

    def predict(self, x):
        """Network output for any number of samples (in batches of the network's batch size)."""
        return torch.cat([self.forward(x[i:i + self.batch].contiguous()) for i in range(0, x.shape[0], self.batch)])

    def pcg(self, solver, x0, n_samples, maxit=500, tol=1e-6):
        """Warm-started FP32 CG of the first n_samples P-MBFs; returns per-sample iterations."""
        iters = torch.empty(n_samples, dtype=torch.int32, device=self.device)
        L.check(self.lib.mrcm_pcg_mbf(solver.handle, self.net, solver.ws_ptr, _ptr(x0) if x0 is not None else None,
                                      n_samples, maxit, C.c_double(tol), _ptr(iters), _stream()), solver.handle)
        return iters
