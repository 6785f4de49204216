"""PyTorch autograd wrapper of the likelihood-ratio adjoint.

``kappa(log_tau_scale, p_pore, ...)`` is a Monte Carlo estimate of kappa_eff
of one steady geometry in which relaxation time tau_i of bin i is scaled by
exp(log_tau_scale_i) and the pore-wall specularity is p_pore.  Its backward
is the library's score-function estimate (``mcbte_grad``) of the gradient of
the expected kappa_eff, computed in the same pass as the forward estimate:
an unbiased gradient of E[kappa], not the derivative of the sampled value.
The pore-specularity derivative is NaN at p_pore = 0 or 1, where the
likelihood-ratio estimator is undefined.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np
import torch

from . import _lib as L
from . import api


class KappaFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_tau_scale, p_pore, material, geometry, n_particles, cfg):
        s = log_tau_scale.detach().to("cpu", torch.float64).numpy()
        mat = material.scaled_tau(s)
        geo = replace(geometry, pore_p=float(p_pore.detach().item()))
        M = api.Material(mat)
        G = api.Geometry(geo)
        fwd, go = api.grad(M, G, int(n_particles), cfg)
        torch.cuda.current_stream().synchronize()
        ctx.save_for_backward(go.dkappa_dlogtau.clone(), go.dkappa_dp[0:1].clone())
        ctx.meta = (log_tau_scale.dtype, log_tau_scale.device, p_pore.dtype, p_pore.device)
        ctx.stats = fwd.stats[0].clone()
        return fwd.stats[0, L.STAT_KAPPA].clone().to(log_tau_scale.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        dk, dp = ctx.saved_tensors
        dt, dev, pdt, pdev = ctx.meta
        g_tau = (grad_out.to(torch.float64) * dk).to(dt).to(dev)
        g_p = (grad_out.to(torch.float64) * dp[0]).to(pdt).to(pdev)
        return g_tau, g_p, None, None, None, None


def kappa(log_tau_scale: torch.Tensor, p_pore: torch.Tensor, material, geometry, n_particles: int,
          cfg: api.SteadyConfig) -> torch.Tensor:
    """kappa_eff estimate with a likelihood-ratio backward (see module doc)."""
    return KappaFunction.apply(log_tau_scale, p_pore, material, geometry, n_particles, cfg)
