"""torch.autograd binding of the VMC energy and the stochastic-reconfiguration
step (Sec. 3.2, Eqs. 7-12).  Argument marshalling only: the energy, the
log-derivatives O_k, the gradient F and the CG solve run in the CUDA library.

Parameters are a float64 CUDA tensor of shape [P, 2] holding (Re alpha_k,
Im alpha_k) in the layout of include/nnqs.h.
"""
from __future__ import annotations

import torch

from . import nnqs


class VMCEnergy(torch.autograd.Function):
    """E(alpha) = mean_s Re E_loc(s) over configurations s drawn from
    |psi_alpha|^2.  backward: dE/dRe alpha_k = 2 Re F_k, dE/dIm alpha_k =
    2 Im F_k with F_k = <conj(O_k)(E_loc - <E_loc>)> from the hand-written
    O_k kernels (nnqs_grad_logpsi, nnqs_energy_grad)."""

    @staticmethod
    def forward(ctx, params, model: nnqs.Model, cfg):
        model.set_params(params.detach())
        sums = torch.empty(4, dtype=torch.float64, device=params.device)
        eloc = model.local_energy(cfg, sums=sums)
        ctx.model, ctx.cfg = model, cfg
        ctx.save_for_backward(eloc)
        return sums[0] / sums[3]

    @staticmethod
    def backward(ctx, grad_e):
        (eloc,) = ctx.saved_tensors
        O = ctx.model.grad_logpsi(ctx.cfg)
        F = ctx.model.energy_grad(O, eloc)
        return 2.0 * grad_e * F, None, None


def sr_step(model: nnqs.Model, params, cfg, lam=1e-6, dtau=0.01, max_iter=200, tol=1e-10, weights=None):
    """One SR update (Eq. 12): params += delta with (S + lam) delta = -dtau F,
    in place on the device; returns (delta, info = [iterations, |r|/|b|])."""
    model.set_params(params)
    eloc = model.local_energy(cfg)
    O = model.grad_logpsi(cfg)
    F = model.energy_grad(O, eloc, weights=weights)
    delta, info = model.sr_solve(O, F, lam=lam, dtau=dtau, max_iter=max_iter, tol=tol, weights=weights,
                                 params_inout=params)
    model.set_params(params)
    return delta, info
