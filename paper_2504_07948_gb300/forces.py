"""Ionic forces through ``torch.autograd``.

``ForceFn.apply(R_nuc, qmc)`` evaluates, at the current walkers of ``qmc``
and nuclear positions ``R_nuc`` ([n_nuc, 3] float64), the per-walker local
energy E_L and ln|Psi_T|.  Its backward pass calls the adjoint kernel of
libqmc (``qmc_force_vjp``) with the incoming per-walker weights, so
``torch.autograd.grad`` of any loss linear in (E_L, ln|Psi_T|) returns
sum_w g_E dE_L/dR + g_psi d ln|Psi_T|/dR without storing intermediates.

``zvzb_force`` returns the zero-variance zero-bias estimator the paper's
force formalism uses (Sec. "Single Determinant QMC Forces"),
F = -<dE_L/dR> - 2 (<E_L d ln|Psi|/dR> - <E_L><d ln|Psi|/dR>),
computed by the library (qmc_force_estimate) at the given nuclear positions.
"""
from __future__ import annotations

import numpy as np
import torch

from . import qmc as Q


class ForceFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, R_nuc: torch.Tensor, qmc: "Q.QMC"):
        Q.qmc_set_nuclei(qmc.h, R_nuc.detach().to("cpu", torch.float64).numpy())
        out = qmc.evaluate()
        ctx.qmc = qmc
        ctx.dev = R_nuc.device
        eloc = torch.from_numpy(out["eloc"]).to(R_nuc.device)
        logpsi = torch.from_numpy(out["logpsi"]).to(R_nuc.device)
        return eloc, logpsi

    @staticmethod
    def backward(ctx, g_eloc, g_logpsi):
        qmc = ctx.qmc
        gE = None if g_eloc is None else g_eloc.detach().to("cpu", torch.float64).contiguous().numpy()
        gL = None if g_logpsi is None else g_logpsi.detach().to("cpu", torch.float64).contiguous().numpy()
        dR = np.zeros((qmc.sys.n_nuc, 3))
        Q.qmc_force_vjp(qmc.h, gE, gL, dR, None)
        return torch.from_numpy(dR).to(ctx.dev), None


def zvzb_force(R_nuc: torch.Tensor, qmc: "Q.QMC", weights=None) -> torch.Tensor:
    """Force estimator over the current walkers (weights [W] or None = equal)
    at nuclear positions R_nuc [n_nuc, 3]."""
    Q.qmc_set_nuclei(qmc.h, R_nuc.detach().to("cpu", torch.float64).contiguous().numpy())
    F = np.zeros((qmc.sys.n_nuc, 3))
    w = None if weights is None else np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    Q.qmc_force_estimate(qmc.h, w, F)
    return torch.from_numpy(F).to(R_nuc.device)
