"""The projection as a differentiable PyTorch op with a hand-written adjoint.

``project(u_star, phi)`` returns the divergence-free velocity u = u* - dt beta grad p
(Eq. runge1) and the pressure p.  Its backward is the adjoint projection of the C ABI
(mg_project_adjoint: one more solve with the same self-adjoint operator) followed by
the chain rule to phi (mg_phi_grad).  Saved for backward: phi (an input), the solid
mask (an input) and p; the face coefficients and the multigrid hierarchy are rebuilt
in backward from phi (into a cached context, see ``clear_cache``).
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import mgproj

# One multigrid context per (grid, spacing, precision, device), reused across calls:
# mg_update rebuilds its hierarchy for each new phi without reallocating.
_CONTEXTS = {}


def _context(beta, h, prec):
    key = (tuple(beta[0].shape), float(h), int(prec), beta[0].device.index, torch.cuda.current_stream().cuda_stream)
    mg = _CONTEXTS.get(key)
    if mg is None:
        if len(_CONTEXTS) >= 4:
            _CONTEXTS.pop(next(iter(_CONTEXTS))).close()
        # CG preconditioned by V-cycles: 2 cycles per application with FP32 cycles, 1 with FP64
        mg = _CONTEXTS[key] = mgproj.Context(beta, h, prec=prec, krylov=1,
                                             inner_cycles=2 if prec == mgproj.MG_MIXED else 1)
    else:
        mg.update(beta)
    return mg


def clear_cache():
    """Free the cached multigrid contexts."""
    while _CONTEXTS:
        _CONTEXTS.popitem()[1].close()


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ux, uy, uz, phi, solid, h, dt, rho_air, rho_water, tol, prec):
        beta = mgproj.face_coeffs(phi, h, solid, rho_air, rho_water)
        mg = _context(beta, h, prec)
        p = torch.zeros_like(phi)
        u, p, st = mg.project((ux, uy, uz), p=p, dt=dt, tol=tol)
        ctx.save_for_backward(phi, p, solid if solid is not None else torch.empty(0, device=phi.device))
        ctx.has_solid = solid is not None
        ctx.cfg = (h, dt, rho_air, rho_water, tol, prec)
        ctx.mark_non_differentiable(p)
        return u[0], u[1], u[2], p

    @staticmethod
    def backward(ctx, gux, guy, guz, gp):
        phi, p, solid = ctx.saved_tensors
        solid = solid if ctx.has_solid else None
        h, dt, rho_air, rho_water, tol, prec = ctx.cfg
        w = tuple((g if g is not None else torch.zeros_like(phi)).contiguous() for g in (gux, guy, guz))
        beta = mgproj.face_coeffs(phi, h, solid, rho_air, rho_water)
        mg = _context(beta, h, prec)
        grad_u, grad_beta, _ = mg.project_adjoint(w, p, dt=dt, tol=tol, q=torch.zeros_like(phi))
        gphi = mgproj.phi_grad(beta, grad_beta, h, rho_air, rho_water) if ctx.needs_input_grad[3] else None
        return grad_u[0], grad_u[1], grad_u[2], gphi, None, None, None, None, None, None, None


def project(u_star: Sequence[torch.Tensor], phi: torch.Tensor, h: float, solid: Optional[torch.Tensor] = None,
            dt: float = 1.0, rho_air: float = 1e-3, rho_water: float = 1.0, tol: float = 1e-10,
            precision: str = "fp64"):
    """Differentiable pressure projection.  Returns ((ux, uy, uz), p); gradients flow to u* and phi."""
    prec = {"fp64": mgproj.MG_FP64, "mixed": mgproj.MG_MIXED}[precision]
    ux, uy, uz, p = _Project.apply(u_star[0], u_star[1], u_star[2], phi, solid, h, dt, rho_air, rho_water, tol, prec)
    return (ux, uy, uz), p
