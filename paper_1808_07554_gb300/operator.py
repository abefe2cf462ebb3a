"""Learned warm start of the pressure solves: a five-layer convolutional operator.

The operator predicts the correction to the linear extrapolation in time of the converged
pressure, d = (P^{n+1} - (2 P^n - P^{n-1})) / dp_scale, from four channels (ln K, S^n,
S^n - S^{n-1}, P^n - P^{n-1}, each normalised).  Its prediction enters the solver through
``lbm2p_warm_start`` (the equilibrium part of f moves to it, Eq. 3-3) and the pressure solve
still runs to the same residual, so the prediction changes the number of sweeps, never the
converged field.  Training pairs come from the solver itself: quarter five-spot realisations
stepped to r <= 1e-8, their converged P and S recorded every step.

Every computation runs in the library's kernels (``include/lbm2p_operator.h``): the 3x3
convolutions and their gradients on the tensor cores (tcgen05, BF16 in, FP32 accumulate),
features, loss gradient, Adam, prediction on CUDA cores.  This module allocates device
buffers through PyTorch and sequences the calls; it does no arithmetic on field data.
"""
from __future__ import annotations

import numpy as np

from . import (LBM2PError, lbm2p_op_adam, lbm2p_op_conv3x3, lbm2p_op_conv3x3_wgrad,
               lbm2p_op_diff_stats, lbm2p_op_features, lbm2p_op_flip_weights,
               lbm2p_op_mse_grad, lbm2p_op_predict, lbm2p_op_target)

# (C_in, C_out) of the five 3x3 convolutions: 16 input channels (4 used), 32 hidden, and an
# output layer of 16 channels of which channel 0 is the prediction
LAYERS = [(16, 32), (32, 32), (32, 32), (32, 32), (32, 16)]
IN_CHANNELS = 4


class PressureOperator:
    """Weights (FP32 master copy, BF16 working copy, Adam moments) of the five convolutions
    and the calls of one forward pass, one training step and one prediction."""

    def __init__(self, seed: int = 0, device: str = "cuda"):
        import torch
        self.torch = torch
        self.device = device
        rng = np.random.default_rng(seed)
        chunks, self.offsets = [], []
        off = 0
        for li, (ci, co) in enumerate(LAYERS):
            fan_in = 9 * (IN_CHANNELS if li == 0 else ci)
            w = rng.standard_normal((9, co, ci)) * np.sqrt(2.0 / fan_in)
            if li == 0:
                w[:, :, IN_CHANNELS:] = 0.0
            if li == len(LAYERS) - 1:
                w *= 0.1                                # a small first prediction
                w[:, 1:, :] = 0.0                      # only channel 0 is read
            b = np.zeros(co)
            self.offsets.append((off, off + w.size, off + w.size + co))
            chunks += [w.ravel(), b]
            off += w.size + co
        self.n = off
        flat = np.concatenate(chunks).astype(np.float32)
        f32 = dict(dtype=torch.float32, device=device)
        self.p = torch.from_numpy(flat).to(device)
        self.pb = self.p.to(torch.bfloat16)
        self.g = torch.zeros(self.n, **f32)
        self.m = torch.zeros(self.n, **f32)
        self.v = torch.zeros(self.n, **f32)
        self.t = 0
        self.wt = [torch.empty(9 * ci * co, dtype=torch.bfloat16, device=device)
                   for ci, co in LAYERS]
        self.err = torch.zeros(1, dtype=torch.int32, device=device)
        self._acts = {}
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)

    # ---- parameter views (device pointers) -------------------------------------------------
    def _w(self, li):
        a, b, _ = self.offsets[li]
        return self.pb[a:b].data_ptr()

    def _b(self, li):
        _, b, c = self.offsets[li]
        return self.p[b:c].data_ptr()

    def _gw(self, li):
        a, b, _ = self.offsets[li]
        return self.g[a:b].data_ptr()

    def _gb(self, li):
        _, b, c = self.offsets[li]
        return self.g[b:c].data_ptr()

    def _stream(self):
        return self.torch.cuda.current_stream().cuda_stream

    def _buffers(self, n, H, W):
        key = (n, H, W)
        if key not in self._acts:
            torch = self.torch
            bf = dict(dtype=torch.bfloat16, device=self.device)
            acts = [None] + [torch.empty((n, H, W, co), **bf) for _, co in LAYERS[:-1]]
            grads = [torch.empty((n, H, W, co), **bf) for _, co in LAYERS]
            y0 = torch.empty((n, H, W), dtype=torch.float32, device=self.device)
            self._acts = {key: (acts, grads, y0)}
        return self._acts[key]

    def check(self):
        if int(self.err.item()) != 0:
            raise LBM2PError(3, "an operator kernel gave up waiting on its tensor-core work")

    # ---- passes ------------------------------------------------------------------------
    def forward(self, feat, n, H, W):
        """feat: BF16 [n, H, W, 16] device tensor; returns the FP32 [n, H, W] output (a view
        of an internal buffer, valid until the next call with the same shape)."""
        acts, _, y0 = self._buffers(n, H, W)
        s = self._stream()
        x = feat.data_ptr()
        last = len(LAYERS) - 1
        for li, (ci, co) in enumerate(LAYERS):
            if li < last:
                lbm2p_op_conv3x3(x, self._w(li), self._b(li), 0, acts[li + 1].data_ptr(), 0, n,
                                 H, W, ci, co, 1, self.err.data_ptr(), s)
                x = acts[li + 1].data_ptr()
            else:
                lbm2p_op_conv3x3(x, self._w(li), self._b(li), 0, 0, y0.data_ptr(), n, H, W, ci,
                                 co, 0, self.err.data_ptr(), s)
        return y0

    def train_step(self, feat, target, n, H, W, lr=1e-3):
        """One Adam step on the mean-squared error of the output against target (FP32
        [n, H, W]); returns the loss of this batch as a device scalar (FP64)."""
        acts, grads, y0 = self._buffers(n, H, W)
        s = self._stream()
        self.forward(feat, n, H, W)
        self.loss.zero_()
        last = len(LAYERS) - 1
        lbm2p_op_mse_grad(y0.data_ptr(), target.data_ptr(), grads[last].data_ptr(),
                          self.loss.data_ptr(), n * H * W, LAYERS[last][1], s)
        for li in range(last, -1, -1):
            ci, co = LAYERS[li]
            x = feat.data_ptr() if li == 0 else acts[li].data_ptr()
            lbm2p_op_conv3x3_wgrad(x, grads[li].data_ptr(), self._gw(li), self._gb(li), n, H, W,
                                   ci, co, 0, self.err.data_ptr(), s)
            if li > 0:
                # input gradient through the flipped weights, times the ReLU derivative
                lbm2p_op_flip_weights(self._w(li), self.wt[li].data_ptr(), ci, co, s)
                lbm2p_op_conv3x3(grads[li].data_ptr(), self.wt[li].data_ptr(), 0,
                                 acts[li].data_ptr(), grads[li - 1].data_ptr(), 0, n, H, W, co,
                                 ci, 0, self.err.data_ptr(), s)
        self.t += 1
        lbm2p_op_adam(self.p.data_ptr(), self.g.data_ptr(), self.m.data_ptr(),
                      self.v.data_ptr(), self.pb.data_ptr(), self.n, lr, 0.9, 0.999, 1e-8,
                      self.t, s)
        return self.loss


# ---- training data from the solver, training, and the learned warm-start loop -------------
def _planes(torch, shape, count, device):
    return torch.empty((count,) + tuple(shape), dtype=torch.float32, device=device)


def record_snapshots(pkg, problems, steps, device="cuda", solver_kw=None, log=None):
    """Step each problem `steps` physical steps to r <= its tolerance (the t = 0 pressure from
    the coarse-lattice guess, each step warm-started by the linear extrapolation, which does
    not change the converged fields) and keep, on the device, ln K and the converged P^n, S^n
    of every time level n = 0 .. steps.  Returns [(lnK [H, W], P [steps + 1, H, W],
    S [steps + 1, H, W])]."""
    import torch
    from .initial_guess import coarse_initial_pressure
    kw = dict(tol=1e-8, check_every=8, warm_start=1, fuse_sweeps=1, sweep_kernel=2)
    kw.update(solver_kw or {})
    out = []
    for prob in problems:
        P0 = coarse_initial_pressure(prob, pkg, fuse_sweeps=1, sweep_kernel=2)
        if P0 is not None:
            prob.P0 = P0
        s = pkg.Solver.from_problem(prob, **kw)
        H, W = prob.ny, prob.nx
        lnK = torch.from_numpy(np.log(prob.K).astype(np.float32)).to(device)
        P = _planes(torch, (H, W), steps + 1, device)
        S = _planes(torch, (H, W), steps + 1, device)
        s.fields_device(P[0], S[0])
        sweeps = 0
        for n in range(steps):
            st, stats = s.step(1)
            if st not in (pkg.OK, pkg.ENOTCONVERGED):
                raise LBM2PError(st, "a training run failed")
            sweeps += stats[0].sub_iters
            s.fields_device(P[n + 1], S[n + 1])
        torch.cuda.synchronize()
        s.close()
        if log is not None:
            log.append({"n": H, "steps": steps, "sweeps": sweeps})
        out.append((lnK, P, S))
    return out


def train(op: PressureOperator, runs, epochs=1, batch=16, lr=1e-3, s_mean=0.2, s_scale=0.1,
          seed=0, max_seconds=None, log=None):
    """Train on every (run, n) with 1 <= n < steps: features of time level n (ln K, S^n,
    S^n - S^{n-1}, P^n - P^{n-1}), target the correction to the extrapolation of P^{n+1}.
    Returns the mean loss of each epoch."""
    import time
    torch = op.torch
    H, W = runs[0][1].shape[1:]
    items = [(r, n) for r in range(len(runs)) for n in range(1, runs[r][1].shape[0] - 1)]
    rng = np.random.default_rng(seed)
    feat = torch.empty((batch, H, W, 16), dtype=torch.bfloat16, device=op.device)
    tgt = torch.empty((batch, H, W), dtype=torch.float32, device=op.device)
    stats = torch.zeros((batch, 2, 2), dtype=torch.float64, device=op.device)
    s = op._stream()
    t0 = time.perf_counter()

    def fill(idx):
        stats.zero_()
        for i, k in enumerate(idx):
            r, n = items[k]
            lnK, P, S = runs[r]
            ds, dp = stats[i, 0], stats[i, 1]
            lbm2p_op_diff_stats(S[n].data_ptr(), S[n - 1].data_ptr(), H * W, ds.data_ptr(), s)
            lbm2p_op_diff_stats(P[n].data_ptr(), P[n - 1].data_ptr(), H * W, dp.data_ptr(), s)
            lbm2p_op_features(lnK.data_ptr(), S[n].data_ptr(), S[n - 1].data_ptr(),
                              P[n].data_ptr(), P[n - 1].data_ptr(), ds.data_ptr(),
                              dp.data_ptr(), feat[i].data_ptr(), H, W, s_mean, s_scale, s)
            lbm2p_op_target(P[n + 1].data_ptr(), P[n].data_ptr(), P[n - 1].data_ptr(),
                            dp.data_ptr(), tgt[i].data_ptr(), H, W, s)

    # the loss of the zero prediction (the plain extrapolation) on a sample of batches: the
    # share of the target's mean square that the operator removes is what it learned
    zero = torch.zeros((batch, H, W), dtype=torch.float32, device=op.device)
    gbuf = torch.empty((batch, H, W, 16), dtype=torch.bfloat16, device=op.device)
    zl = torch.zeros(1, dtype=torch.float64, device=op.device)
    sample = rng.permutation(len(items))[:batch * 16]
    for b0 in range(0, len(sample) - batch + 1, batch):
        fill(sample[b0:b0 + batch])
        lbm2p_op_mse_grad(zero.data_ptr(), tgt.data_ptr(), gbuf.data_ptr(), zl.data_ptr(),
                          batch * H * W, 16, s)
    zero_loss = float(zl.item()) / max(1, len(sample) // batch)
    if log is not None:
        log.append({"zero_prediction_loss": zero_loss})
    losses = []
    for ep in range(epochs):
        order = rng.permutation(len(items))
        total, count = 0.0, 0
        for b0 in range(0, len(order) - batch + 1, batch):
            fill(order[b0:b0 + batch])
            loss = op.train_step(feat, tgt, batch, H, W, lr=lr)
            total += float(loss.item())
            count += 1
            if max_seconds is not None and time.perf_counter() - t0 > max_seconds:
                break
        op.check()
        losses.append(total / max(1, count))
        if log is not None:
            log.append({"epoch": ep, "batches": count, "loss": losses[-1],
                        "seconds": round(time.perf_counter() - t0, 2)})
        if max_seconds is not None and time.perf_counter() - t0 > max_seconds:
            break
    return losses


class LearnedWarmStart:
    """Steps a Solver whose every pressure solve starts from the operator's prediction:
    before each step the solver's P^n, S^n (and the previous level's) give the features, the
    operator predicts P^{n+1}, and lbm2p_warm_start moves the populations' equilibrium part
    to it.  The solve then runs to the solver's own tolerance."""

    def __init__(self, op: PressureOperator, solver, lnK, s_mean=0.2, s_scale=0.1):
        torch = op.torch
        self.op, self.s = op, solver
        self.H, self.W = solver.ny, solver.nx
        shape = (self.H, self.W)
        f32 = dict(dtype=torch.float32, device=op.device)
        self.lnK = torch.from_numpy(np.ascontiguousarray(lnK, dtype=np.float32)).to(op.device)
        self.P, self.Pp = torch.empty(shape, **f32), torch.empty(shape, **f32)
        self.S, self.Sp = torch.empty(shape, **f32), torch.empty(shape, **f32)
        self.Ppred = torch.empty(shape, **f32)
        self.feat = torch.empty((1, self.H, self.W, 16), dtype=torch.bfloat16, device=op.device)
        self.stats = torch.zeros((2, 2), dtype=torch.float64, device=op.device)
        self.s_mean, self.s_scale = s_mean, s_scale

    def prime(self):
        """Record the solver's current time level; called after each of two steps the solver
        takes on its own before the learned steps start (the features need two levels)."""
        self.Pp, self.P = self.P, self.Pp
        self.Sp, self.S = self.S, self.Sp
        self.s.fields_device(self.P, self.S)

    def step(self):
        """One physical step from the learned prediction; returns (status, stats)."""
        op = self.op
        s = op._stream()
        H, W = self.H, self.W
        self.stats.zero_()
        lbm2p_op_diff_stats(self.S.data_ptr(), self.Sp.data_ptr(), H * W,
                            self.stats[0].data_ptr(), s)
        lbm2p_op_diff_stats(self.P.data_ptr(), self.Pp.data_ptr(), H * W,
                            self.stats[1].data_ptr(), s)
        lbm2p_op_features(self.lnK.data_ptr(), self.S.data_ptr(), self.Sp.data_ptr(),
                          self.P.data_ptr(), self.Pp.data_ptr(), self.stats[0].data_ptr(),
                          self.stats[1].data_ptr(), self.feat.data_ptr(), H, W, self.s_mean,
                          self.s_scale, s)
        d = op.forward(self.feat, 1, H, W)
        lbm2p_op_predict(self.P.data_ptr(), self.Pp.data_ptr(), d.data_ptr(),
                         self.stats[1].data_ptr(), self.Ppred.data_ptr(), H, W, s)
        self.s.warm_start_device(self.Ppred)
        st, stats = self.s.step(1)
        # the new time level becomes the current one
        self.Pp, self.P = self.P, self.Pp
        self.Sp, self.S = self.S, self.Sp
        self.s.fields_device(self.P, self.S)
        return st, stats
