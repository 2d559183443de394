"""torch.autograd.Function around pq_survival_grad: the survival probability
P(theta) = |<Psi(0)|Psi(T)>|^2 of the pruned Henon-Heiles propagation as a
differentiable function of theta = (lambda, omega_1..omega_D, q0_1..q0_D).

The forward call runs the propagation and the adjoint sweep on the GPU (the
sets of active functions recorded and held fixed); backward returns the
stored gradient times the incoming gradient."""
from __future__ import annotations

import numpy as np
import torch

from . import FP64, State, build_model, henon_heiles_param_derivs


class SurvivalProbability(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, cfg, precision, ckpt_every):
        D = cfg["D"]
        th = theta.detach().cpu().double().numpy()
        lam, om, q0 = float(th[0]), th[1:1 + D], th[1 + D:1 + 2 * D]
        b = build_model(cfg, omegas=om, lam=lam)
        s = State(b, q0, cfg["p0"], cfg["width"], cfg["theta"], precision=precision)
        grids = [b.grid(k)[0] for k in range(D)]
        P, g = s.survival_grad(cfg["K"], cfg["dt"], cfg["theta"], cfg["nsteps"], ckpt_every,
                               henon_heiles_param_derivs(grids, lam, om))
        ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype))
        return torch.as_tensor(P, dtype=theta.dtype)

    @staticmethod
    def backward(ctx, gP):
        (g,) = ctx.saved_tensors
        return gP * g, None, None, None


def survival_probability(theta, cfg, precision=FP64, ckpt_every=25):
    """P(theta) with an autograd backward through the GPU adjoint."""
    return SurvivalProbability.apply(theta, cfg, precision, ckpt_every)
