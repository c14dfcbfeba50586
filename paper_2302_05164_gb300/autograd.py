"""The hand-written adjoint of the explicit stepper as a torch.autograd.Function.

`ThermalObjective.apply(P, s, ...)` returns, per instance of a batch, the melt-pool objective
J = (1/N) sum_n (M_n - T_target)^2 of N forward-Euler steps (M_n the p-norm of the
top-surface temperature, Eq. forward_euler for the steps) as a function of the per-segment
laser powers P [batch, n_seg] and the conductivity scales s [batch]. Forward and reverse
sweeps both run in the library's `pbf_adjoint_sweep` (binomial checkpointing of the state):
the forward pass of this Function computes J and dJ/d(P, s) in that one call, and its
backward pass only scales the stored gradient by the incoming one. Nothing is differentiated
by torch itself; the binding marshals arguments and tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import pbf


class ThermalObjective(torch.autograd.Function):
    """J(P, s) [batch] with gradients from the library's adjoint sweep.

    Arguments of `apply`: P [batch, n_seg] and s [batch] (float64 tensors, any device; the
    gradients come back on theirs), then the context handle of a `pbf.Context` created with
    that batch, the initial state T0 (float64 CUDA tensor [n_dofs][batch], not modified), the
    laser dict whose segments are used (its powers are replaced by P), t0, dt, the number of
    steps, the number of stored states for the binomial schedule, and optionally T_target
    (2300 K) and the p-norm exponent (16).
    """

    @staticmethod
    def forward(fctx, P, s, ctx_handle, T0, laser, t0, dt, nsteps, n_checkpoints, T_target=2300.0, p_exp=16.0):
        batch = int(s.shape[0])
        if P.dim() != 2 or P.shape[0] != batch:
            raise ValueError("P must be [batch, n_seg] with the batch of s")
        ls = dict(laser, power=P.detach().to("cpu", torch.float64).numpy())
        pbf.pbf_ctx_set_k_scale(ctx_handle, s.detach().to("cpu", torch.float64).numpy())
        J, grad, _ = pbf.pbf_adjoint_sweep(ctx_handle, T0, ls, t0, dt, nsteps, n_checkpoints, T_target=T_target,
                                           p_exp=p_exp, batch=batch)
        g = torch.from_numpy(np.ascontiguousarray(grad))
        fctx.save_for_backward(g)
        fctx.devices = (P.device, s.device)
        return torch.from_numpy(J).to(s.device)

    @staticmethod
    def backward(fctx, gJ):
        (g,) = fctx.saved_tensors
        gJ = gJ.detach().to("cpu", torch.float64)
        gP = (gJ[:, None] * g[:, :-1]).to(fctx.devices[0])
        gs = (gJ * g[:, -1]).to(fctx.devices[1])
        return gP, gs, None, None, None, None, None, None, None, None, None
