"""torch.autograd.Function wrappers of the library's forward sweep and its adjoint.

TeukWaveformFn.apply(amps, r0, solver, n_steps) returns the waveform records
W_1 .. W_n (float64 [n][n_theta][2]) of a run that starts from zero data at step 0
with source amplitudes amps (A_0 .. A_{n-1}) and orbit radius r0.  Its backward
calls teuk_adjoint_n with the incoming cotangent dL/dW, which runs the transposed
stencil on the GPU and returns dL/dA_n and dL/dr0.

TeukPsiLossFn.apply(amps, r0, solver, n_steps, ckpt_every) returns the built-in loss
L = sum_{k=1..n} sum_j |r_ext^3 W_k[j]|^2 (psi = r^3 Phi, Eq. 4) of the same run.  Its
forward is one teuk_adjoint_n call in built-in-loss mode; the gradients it returns are
kept for backward, which scales them by the incoming gradient of L.  The step is linear
in the state, so the reverse sweep needs only the loss's cotangent on the records, never
a forward state: with ckpt_every = 0 the forward sweep keeps every
record's cotangent (n_steps x n_theta x 16 B) and the reverse sweep follows at once;
with ckpt_every = K > 0 (the default, K = 100) the forward sweep keeps a state
checkpoint every K steps and the reverse sweep recomputes each segment's records from
its checkpoint (one more forward sweep of work).  A checkpoint is a whole state, so
this saves memory only where a segment's records outweigh a state, i.e. for K above
about 4 n_rstar (FP32-Kahan)."""
from __future__ import annotations

import numpy as np
import torch


def _source_args(amps, r0):
    a = amps.detach().to("cpu", torch.float64).numpy().copy()
    r = float(r0.detach()) if torch.is_tensor(r0) else float(r0)
    dev_r = r0.device if torch.is_tensor(r0) else torch.device("cpu")
    return a, r, dev_r


class TeukWaveformFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, amps, r0, solver, n_steps):
        a, r, dev_r = _source_args(amps, r0)
        solver.set_source(r, a)
        solver.set_state(np.zeros(solver.shape()), 0)
        solver.step(n_steps)
        w, first = solver.extract(cap=n_steps + 1)
        if first != 0 or w.shape[0] != n_steps + 1:
            raise RuntimeError("waveform ring too small: create the solver with "
                               "wave_capacity >= n_steps + 1")
        # the source of this call: another apply on the same solver, or a set_source,
        # may come before backward, which must differentiate this problem
        ctx.solver, ctx.n, ctx.amps, ctx.r0 = solver, n_steps, a, r
        ctx.devices = (amps.device, dev_r)
        return torch.from_numpy(np.ascontiguousarray(w[1:])).to(amps.device)

    @staticmethod
    def backward(ctx, gw):
        g = gw.detach().to("cpu", torch.float64).contiguous().numpy()
        # cotangent mode leaves the state alone and uses the solver's source
        ctx.solver.set_source(ctx.r0, ctx.amps)
        ga, gr, _ = ctx.solver.adjoint(ctx.n, step0=0, grad_wave=g)
        return (torch.from_numpy(ga).to(ctx.devices[0]),
                torch.tensor(gr, dtype=torch.float64, device=ctx.devices[1]), None, None)


class TeukPsiLossFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, amps, r0, solver, n_steps, ckpt_every=100):
        a, r, dev_r = _source_args(amps, r0)
        solver.set_source(r, a)
        solver.set_state(np.zeros(solver.shape()), 0)
        ga, gr, loss = solver.adjoint(n_steps, step0=0, ckpt_every=ckpt_every)
        ctx.ga, ctx.gr = ga, gr
        ctx.devices = (amps.device, dev_r)
        return torch.tensor(loss, dtype=torch.float64, device=amps.device)

    @staticmethod
    def backward(ctx, gl):
        s = float(gl.detach())
        return (torch.from_numpy(s * ctx.ga).to(ctx.devices[0]),
                torch.tensor(s * ctx.gr, dtype=torch.float64, device=ctx.devices[1]),
                None, None, None)


def psi_loss(solver, w):
    """L = sum |r_ext^3 W|^2 (psi = r^3 Phi, Eq. 4) of waveform records w."""
    r = solver.geometry()["r_ext"]
    return (r ** 6) * (w ** 2).sum()
