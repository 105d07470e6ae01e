"""torch.autograd.Function over the library's forward sweep and its adjoint.

TeukWaveformFn.apply(amps, r0, solver, n_steps) returns the waveform records
W_1 .. W_n (float64 [n][n_theta][2]) of a run that starts from zero data at step 0
with source amplitudes amps (A_0 .. A_{n-1}) and orbit radius r0.  Its backward
calls teuk_adjoint_n with the incoming cotangent dL/dW, which runs the transposed
stencil on the GPU and returns dL/dA_n and dL/dr0."""
from __future__ import annotations

import numpy as np
import torch


class TeukWaveformFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, amps, r0, solver, n_steps):
        a = amps.detach().to("cpu", torch.float64).numpy()
        solver.set_source(float(r0), a)
        solver.set_state(np.zeros(solver.shape()), 0)
        solver.step(n_steps)
        w, first = solver.extract(cap=n_steps + 1)
        if first != 0 or w.shape[0] != n_steps + 1:
            raise RuntimeError("waveform ring too small: create the solver with "
                               "wave_capacity >= n_steps + 1")
        ctx.solver, ctx.n = solver, n_steps
        ctx.devices = (amps.device, r0.device if torch.is_tensor(r0) else torch.device("cpu"))
        return torch.from_numpy(np.ascontiguousarray(w[1:])).to(amps.device)

    @staticmethod
    def backward(ctx, gw):
        g = gw.detach().to("cpu", torch.float64).contiguous().numpy()
        ga, gr, _ = ctx.solver.adjoint(ctx.n, step0=0, grad_wave=g)
        return (torch.from_numpy(ga).to(ctx.devices[0]),
                torch.tensor(gr, dtype=torch.float64, device=ctx.devices[1]), None, None)


def psi_loss(solver, w):
    """L = sum |r_ext^3 W|^2 (psi = r^3 Phi, Eq. 4) of waveform records w."""
    r = solver.geometry()["r_ext"]
    return (r ** 6) * (w ** 2).sum()
