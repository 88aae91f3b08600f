"""Learned warm start for the EM loop (not part of the paper).

For a fixed template X (one setup: Gram matrix, eigendecomposition, top-K
basis U), a point-set network maps a scene Y to the K x 3 eigen-coefficients
c = U^T (T* - X) of the registration's end point T* and to log sigma2*; the
next registration then starts at T = X + U c with a variance calibrated on
held-out scenes, instead of at W = 0 with the data variance.  Training pairs
are produced by the method itself (registrations from W = 0).  Every step
runs in libfcpd.so kernels (EM, coefficients, network forward/backward,
Adam); this module only moves arrays and keeps the target normalisation.
A start from W = 0 stays the fallback (Context.reset()).
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import cpd


NET_FP32, NET_BF16 = 0, 1    # cpd_net_create_ex precisions


class Net:
    """The network (cpd_net_*): n_out outputs, scenes of n_points points.
    precision NET_BF16 runs the wide per-point layers and their gradients on
    the BF16 tensor cores (FP32 accumulation and master weights)."""

    def __init__(self, n_out, n_points, max_batch=32, seed=0, stream=None, precision=NET_FP32):
        lib = cpd.load()
        self.n_out, self.n_points, self.max_batch = int(n_out), int(n_points), int(max_batch)
        h = C.c_void_p()
        cpd._check(lib.cpd_net_create_ex(self.n_out, self.max_batch, self.n_points, int(seed), int(precision),
                                         cpd._stream_handle(stream, True), C.byref(h)))
        self.precision = int(lib.cpd_net_precision(h))
        self._h = h
        self.n_params = int(lib.cpd_net_num_params(h))

    def _check_batch(self, Y):
        import torch
        if not (isinstance(Y, torch.Tensor) and Y.is_cuda and Y.dtype == torch.float32 and Y.is_contiguous()):
            raise TypeError("Y must be a contiguous float32 CUDA tensor")
        if Y.dim() != 3 or Y.shape[1] != self.n_points or Y.shape[2] != 3 or not 1 <= Y.shape[0] <= self.max_batch:
            raise ValueError(f"Y must be (B <= {self.max_batch}, {self.n_points}, 3), got {tuple(Y.shape)}")
        return int(Y.shape[0])

    def params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        cpd._check(cpd.load().cpd_net_get_params(self._h, out.ctypes.data))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        cpd._check(cpd.load().cpd_net_set_params(self._h, p.ctypes.data))

    def forward(self, Y):
        """Y: CUDA tensor (B, n_points, 3) float32 -> (B, n_out) numpy."""
        B = self._check_batch(Y)
        out = np.empty((B, self.n_out), dtype=np.float32)
        cpd._check(cpd.load().cpd_net_forward(self._h, Y.data_ptr(), B, out.ctypes.data))
        return out

    def gradients(self, Y, target):
        B = self._check_batch(Y)
        t = np.ascontiguousarray(target, dtype=np.float32).reshape(B, self.n_out)
        g = np.empty(self.n_params, dtype=np.float32)
        loss = C.c_float()
        cpd._check(cpd.load().cpd_net_gradients(self._h, Y.data_ptr(), t.ctypes.data, B, g.ctypes.data,
                                                C.byref(loss)))
        return g, loss.value

    def train_step(self, Y, target, lr):
        B = self._check_batch(Y)
        t = np.ascontiguousarray(target, dtype=np.float32).reshape(B, self.n_out)
        loss = C.c_float()
        cpd._check(cpd.load().cpd_net_train_step(self._h, Y.data_ptr(), t.ctypes.data, B, float(lr),
                                                 C.byref(loss)))
        return loss.value

    def close(self):
        if getattr(self, "_h", None):
            cpd.load().cpd_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def registration_targets(ctx, scenes, n_coef, iters, group=8):
    """End points of registrations from W = 0: (n, 3 n_coef + 1) float32 rows
    [c = U^T (T - X) (row-major n_coef x 3), log sigma2].  The scenes are
    registered `group` at a time against the context's model
    (cpd_iterate_shared: one pass over the basis per group and iteration);
    group = 1 registers them one at a time on the context itself."""
    import torch
    out = np.empty((len(scenes), 3 * n_coef + 1), dtype=np.float32)
    if group <= 1:
        for i, Y in enumerate(scenes):
            ctx.reset()
            _, s2, _ = ctx.iterate(torch.as_tensor(Y, device="cuda"), iters, want_T=False)
            out[i, :-1] = ctx.coefficients(n_coef).ravel()
            out[i, -1] = math.log(max(s2, 1e-30))
        return out
    for g0 in range(0, len(scenes), group):
        Ys = [torch.as_tensor(Y, device="cuda") for Y in scenes[g0:g0 + group]]
        for j, (T, s2) in enumerate(ctx.iterate_shared(Ys, iters)):
            out[g0 + j, :-1] = ctx.coefficients_of(T, n_coef).ravel()
            out[g0 + j, -1] = math.log(max(s2, 1e-30))
    return out


class WarmStart:
    """Network + target normalisation + start-variance calibration."""

    def __init__(self, n_coef, n_points, max_batch=32, seed=0, precision=NET_FP32):
        self.n_coef = int(n_coef)
        self.net = Net(3 * self.n_coef + 1, n_points, max_batch, seed, precision=precision)
        self.mean = np.zeros(3 * self.n_coef + 1, dtype=np.float32)
        self.std = np.ones(3 * self.n_coef + 1, dtype=np.float32)
        self.sigma2_floor = 0.0

    def fit(self, scenes, targets, steps, batch, lr, seed=0, log_every=0):
        """Adam on the normalised targets; scenes: (n, N, 3) float32.  The
        coefficient outputs share one scale (their RMS deviation), so the
        loss weighs them by their size -- the displacement error |U dc| =
        |dc| -- instead of giving the many small, hard-to-predict high-order
        coefficients equal weight; log sigma2 has its own scale."""
        import torch
        targets = np.asarray(targets, dtype=np.float32)
        self.mean = targets.mean(0)
        dev = targets - self.mean
        self.std = np.full(targets.shape[1], float(np.sqrt((dev[:, :-1] ** 2).mean())) + 1e-6, dtype=np.float32)
        self.std[-1] = float(dev[:, -1].std()) + 1e-6
        z = (targets - self.mean) / self.std
        Yd = torch.as_tensor(np.asarray(scenes, dtype=np.float32), device="cuda")
        rng = np.random.default_rng(seed)
        losses = []
        n = len(targets)
        for s in range(int(steps)):
            idx = rng.choice(n, size=min(batch, n), replace=False)
            ix = torch.as_tensor(idx, device="cuda")
            losses.append(self.net.train_step(Yd.index_select(0, ix).contiguous(), z[idx], lr))
            if log_every and s % log_every == 0:
                print(f"step {s}: loss {losses[-1]:.4f}", flush=True)
        return losses

    def predict(self, scenes):
        """(coefficients (B, n_coef, 3), predicted final sigma2 (B,))."""
        import torch
        Y = torch.as_tensor(np.asarray(scenes, dtype=np.float32), device="cuda")
        out = []
        for b in range(0, Y.shape[0], self.net.max_batch):
            out.append(self.net.forward(Y[b:b + self.net.max_batch].contiguous()))
        p = np.concatenate(out) * self.std + self.mean
        return p[:, :-1].reshape(-1, self.n_coef, 3), np.exp(p[:, -1])

    def calibrate(self, scenes, targets, M):
        """Start variance from held-out scenes: twice the mean squared error of
        the predicted end point per coordinate (U is orthonormal, so
        |U dc|^2 = |dc|^2): sigma2_0 = 2 |c_pred - c|^2 / (3 M)."""
        c, _ = self.predict(scenes)
        ct = np.asarray(targets)[:, :-1].reshape(-1, self.n_coef, 3)
        mse = float(((c - ct) ** 2).sum(axis=(1, 2)).mean())
        self.sigma2_floor = 2.0 * mse / (3.0 * M)
        return self.sigma2_floor

    def start(self, ctx, scene):
        """Next registration of ctx starts at the prediction for `scene`."""
        c, s2 = self.predict(np.asarray(scene, dtype=np.float32)[None])
        ctx.warm_start(c[0], max(float(s2[0]), self.sigma2_floor))
        return c[0], max(float(s2[0]), self.sigma2_floor)
