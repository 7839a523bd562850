"""The projection as a differentiable PyTorch op with a hand-written adjoint.

``project(u_star, phi)`` returns the divergence-free velocity u = u* - dt beta grad p
(Eq. runge1) and the pressure p.  Its backward is the adjoint projection of the C ABI
(mg_project_adjoint: one more solve with the same self-adjoint operator) followed by
the chain rule to phi (mg_phi_grad).  Saved for backward: p, the one array the forward
creates, and references to its inputs phi and the solid mask; the face coefficients are
formed again from them in backward (mg_face_coeffs) unless the cached context still
holds this forward's.  The multigrid hierarchy lives in that cached context (see
``clear_cache``); backward rebuilds it only when another forward has rebuilt the
context since this one.
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import mgproj

# One multigrid context per (grid, spacing, precision, device), reused across calls:
# mg_update rebuilds its hierarchy for each new phi without reallocating.
_CONTEXTS = {}


def _context(beta, h, prec, token):
    """The cached context for this grid, its hierarchy built from ``beta``.  ``token`` names
    the forward call that ``beta`` belongs to: a context whose hierarchy was last built for
    the same token is returned as it is."""
    key = (tuple(beta[0].shape), float(h), int(prec), beta[0].device.index, torch.cuda.current_stream().cuda_stream)
    mg = _CONTEXTS.get(key)
    if mg is None:
        if len(_CONTEXTS) >= 4:
            _CONTEXTS.pop(next(iter(_CONTEXTS))).close()
        # CG preconditioned by V-cycles: 2 cycles per application with FP32 cycles, 1 with FP64
        mg = _CONTEXTS[key] = mgproj.Context(beta, h, prec=prec, krylov=1,
                                             inner_cycles=2 if prec == mgproj.MG_MIXED else 1)
    elif getattr(mg, "built_for", None) is not token:
        mg.update(beta)
    mg.built_for = token
    mg.beta = beta  # this forward's face coefficients, for a backward that finds the context unchanged
    return mg


def _cached_beta(h, prec, shape, device, token):
    """The face coefficients of the forward named by token, if its context still holds them."""
    key = (tuple(shape), float(h), int(prec), device.index, torch.cuda.current_stream().cuda_stream)
    mg = _CONTEXTS.get(key)
    if mg is not None and getattr(mg, "built_for", None) is token:
        return mg.beta
    return None


def clear_cache():
    """Free the cached multigrid contexts."""
    while _CONTEXTS:
        _CONTEXTS.popitem()[1].close()


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ux, uy, uz, phi, solid, h, dt, rho_air, rho_water, tol, prec):
        beta = mgproj.face_coeffs(phi, h, solid, rho_air, rho_water)
        ctx.token = object()
        mg = _context(beta, h, prec, ctx.token)
        p = torch.zeros_like(phi)
        u, p, st = mg.project((ux, uy, uz), p=p, dt=dt, tol=tol)
        ctx.save_for_backward(phi, solid, p)
        ctx.cfg = (h, dt, rho_air, rho_water, tol, prec)
        ctx.mark_non_differentiable(p)
        return u[0], u[1], u[2], p

    @staticmethod
    def backward(ctx, gux, guy, guz, gp):
        phi, solid, p = ctx.saved_tensors
        h, dt, rho_air, rho_water, tol, prec = ctx.cfg
        beta = _cached_beta(h, prec, p.shape, p.device, ctx.token)
        if beta is None:
            beta = mgproj.face_coeffs(phi.detach(), h, solid, rho_air, rho_water)
        w = tuple((g if g is not None else torch.zeros_like(p)).contiguous() for g in (gux, guy, guz))
        mg = _context(beta, h, prec, ctx.token)
        grad_u, grad_beta, _ = mg.project_adjoint(w, p, dt=dt, tol=tol, q=torch.zeros_like(p))
        gphi = mgproj.phi_grad(beta, grad_beta, h, rho_air, rho_water) if ctx.needs_input_grad[3] else None
        return grad_u[0], grad_u[1], grad_u[2], gphi, None, None, None, None, None, None, None


def project(u_star: Sequence[torch.Tensor], phi: torch.Tensor, h: float, solid: Optional[torch.Tensor] = None,
            dt: float = 1.0, rho_air: float = 1e-3, rho_water: float = 1.0, tol: float = 1e-10,
            precision: str = "fp64"):
    """Differentiable pressure projection.  Returns ((ux, uy, uz), p); gradients flow to u* and phi."""
    prec = {"fp64": mgproj.MG_FP64, "mixed": mgproj.MG_MIXED}[precision]
    ux, uy, uz, p = _Project.apply(u_star[0], u_star[1], u_star[2], phi, solid, h, dt, rho_air, rho_water, tol, prec)
    return (ux, uy, uz), p
