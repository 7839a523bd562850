"""Solves from a nonzero initial guess (the CG's first true residual tests its guess for zero
and, only if every value is a zero of either sign, takes r = b without the stencil).

A guess with one nonzero cell must be seen as nonzero: the solve then converges to the
zero-start solution (a guess taken for zero would leave its spike in the result).  The
converged solution as the guess needs no CG iteration.  A guess of negative zeros takes the
same path as one of positive zeros, so the two results are bitwise equal.
"""
import numpy as np
import pytest
import torch

import oracle as O

from _gpu_util import case_rhs, cases_small, dev, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_2240_gb300 import mgproj
    return mgproj


SMALL = cases_small()
NAME = "c2_64" if "c2_64" in SMALL else next(iter(SMALL))


def _setup(mgp, prec):
    case = SMALL[NAME]
    solid = None if case.solid is None else dev(case.solid, dtype=torch.uint8)
    beta = mgp.face_coeffs(dev(case.phi), case.h, solid, rho_air=case.lam, rho_water=1.0)
    ctx = mgp.Context(beta, case.h, prec=prec, krylov=1, inner_cycles=2 if prec == "mixed" else 1,
                      coarse_max_cells=2048)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    rhs = case_rhs(case, beta_o)
    return case, ctx, beta_o, rhs


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_single_nonzero_cell_guess_is_not_taken_for_zero(mgp, prec):
    case, ctx, beta_o, rhs = _setup(mgp, prec)
    p_zero, _ = ctx.solve(dev(rhs), tol=1e-10)
    bx, by, bz = beta_o
    live = (bx > 0) | (by > 0) | (bz > 0)  # any open face, low or high
    live[:, :, :-1] |= bx[:, :, 1:] > 0
    live[:, :-1, :] |= by[:, 1:, :] > 0
    live[:-1, :, :] |= bz[1:, :, :] > 0
    guess = torch.zeros_like(p_zero)
    flat = guess.view(-1)
    flat[int(np.flatnonzero(live.ravel())[-1])] = 1.0e3  # one spike in the last live cell
    p_warm, st = ctx.solve(dev(rhs), p=guess, tol=1e-10)
    lab, nc = O.components(beta_o)
    b = O.remove_mean(rhs, lab, nc)
    pw = host(p_warm)
    assert np.linalg.norm(O.residual(beta_o, b, pw, case.h)) / np.linalg.norm(b) <= 1.0001e-10
    assert rel(pw, host(p_zero)) <= 1e-8
    assert st.cycles >= 1


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_converged_guess_needs_no_iteration(mgp, prec):
    case, ctx, beta_o, rhs = _setup(mgp, prec)
    p_tight, _ = ctx.solve(dev(rhs), tol=1e-12)
    guess = p_tight.clone()
    p, st = ctx.solve(dev(rhs), p=guess, tol=1e-10)
    assert st.cycles == 0
    assert rel(host(p), host(p_tight)) <= 1e-12


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_negative_zero_guess_matches_positive_zero(mgp, prec):
    case, ctx, beta_o, rhs = _setup(mgp, prec)
    p_pos, st_pos = ctx.solve(dev(rhs), p=torch.zeros(case.shape, dtype=torch.float64, device="cuda"), tol=1e-10)
    neg = torch.full(case.shape, -0.0, dtype=torch.float64, device="cuda")
    assert bool(torch.signbit(neg).all())
    p_neg, st_neg = ctx.solve(dev(rhs), p=neg, tol=1e-10)
    assert st_pos.cycles == st_neg.cycles
    assert np.array_equal(host(p_pos), host(p_neg))
