"""torch.autograd.Function over dcm_forces / dcm_forces_backward.

Forward: forces F (n x 3) and total energy E of cell-sorted positions for
per-type LJ parameters eps, sigma (cutoffs fixed).  Backward: the
hand-written adjoint kernel gives dL/dpos and dL/deps, dL/dsigma for any
upstream dL/dF, dL/dE.  Only the inputs are kept for the backward pass; the
adjoint needs no stored forces.
"""
from __future__ import annotations

import torch

from . import dcm as D


class LJForces(torch.autograd.Function):
    @staticmethod
    def forward(fctx, pos4, eps, sigma, rc, cell_start, ctx):
        n = pos4.shape[0]
        D.dcm_set_lj(ctx, eps.detach().cpu().tolist(), sigma.detach().cpu().tolist())
        force = torch.empty_like(pos4)
        totals = torch.zeros(3, dtype=torch.float64, device=pos4.device)
        D.dcm_forces(ctx, n, pos4.detach().contiguous(), rc, cell_start, force, totals)
        fctx.save_for_backward(pos4, rc, cell_start)
        fctx.dcm = ctx
        fctx.nt = eps.shape[0]
        return force[:, :3], totals[0].to(pos4.dtype)

    @staticmethod
    def backward(fctx, gF, gE):
        pos4, rc, cell_start = fctx.saved_tensors
        n = pos4.shape[0]
        A = torch.zeros_like(pos4)
        if gF is not None:
            A[:, :3] = gF
        dE = 0.0 if gE is None else float(gE)
        G = torch.empty_like(pos4)
        dpar = torch.zeros(2 * fctx.nt, dtype=torch.float64, device=pos4.device)
        D.dcm_forces_backward(fctx.dcm, n, pos4.detach().contiguous(), rc, cell_start, A, dE, G, dpar)
        G[:, 3] = 0
        nt = fctx.nt
        return G, dpar[:nt].to(pos4.dtype), dpar[nt:].to(pos4.dtype), None, None, None


def lj_forces(pos4, eps, sigma, rc, cell_start, ctx):
    """(F, E) with autograd support for pos4, eps and sigma."""
    return LJForces.apply(pos4, eps, sigma, rc, cell_start, ctx)
