"""torch.autograd.Function around the discrete adjoint of liblbm.

Argument marshalling only: the forward steps and the reverse sweep run in
liblbm's CUDA kernels (lbm_step / lbm_adjoint).  Gradients are those of the
objective after n_coarse coarse steps from a fixed initial state, with
respect to the body-force field, the coarsest relaxation rate and the inlet
velocity.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm


class MultilevelLBM(torch.autograd.Function):
    """J = objective(state after n_coarse steps) as a differentiable function of
    (force [n, d] float64 tensor, omega_c 0-d tensor, u_in [3] tensor).

    sim: a bound lbm.Sim built with use_force=True; init: (rho, u, S, df)
    host arrays giving the initial state (re-applied before every evaluation);
    objective: 0 kinetic energy, k = 1..d obstacle force component k."""

    @staticmethod
    def forward(ctx, force, omega_c, u_in, sim, init, n_coarse, K, objective):
        sim.set_params(float(omega_c), [float(x) for x in u_in.detach().cpu().tolist()])
        sim.init(*init)
        sim.set_force(force.detach().cpu().numpy())
        needs = any(ctx.needs_input_grad[:3])
        if needs:
            J, dF, dw, du = sim.adjoint(n_coarse, K, objective)
            ctx.save_for_backward(torch.from_numpy(dF), torch.tensor(dw, dtype=torch.float64),
                                  torch.from_numpy(du[: u_in.numel()].copy()))
        else:
            sim.step(n_coarse)
            red = sim.reduce()
            J = float(red[7] if objective == 0 else red[3 + objective])
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        dF, dw, du = ctx.saved_tensors
        return gJ * dF, gJ * dw, gJ * du, None, None, None, None, None


def objective(force, omega_c, u_in, sim, init, n_coarse, K=20, objective=0):
    return MultilevelLBM.apply(force, omega_c, u_in, sim, init, n_coarse, K, objective)
