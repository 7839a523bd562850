"""Pins of the oracle's stretched-grid form (cell widths per axis; Eq. integral2 times the cell
volume on the index grid): uniform widths reproduce the uniform projection, a linear pressure's
face gradients are exact under any stretching, the projection is divergence-free, and a layered
problem matches an independently assembled one-dimensional finite-volume system; CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_1410_2240_gb300 import synth


def _widths(n, ratio, seed=0):
    """smoothly varying widths summing to 1, largest / smallest = ratio"""
    t = (np.arange(n) + 0.5) / n
    w = 1.0 + (ratio - 1.0) * (0.5 - 0.5 * np.cos(2 * np.pi * (t + 0.1 * seed)))
    return w / w.sum()


def test_uniform_widths_reproduce_uniform_projection():
    case = synth.small_case(16, 12, 8, seed=2, solid="none", interface="wave")
    nz, ny, nx = case.shape
    h = case.h
    hx, hy, hz = np.full(nx, h), np.full(ny, h), np.full(nz, h)
    u_s, p_s, bi, area, rhs_s = O.project_stretched(case.phi, hx, hy, hz, case.u_star, lam=case.lam, tol=1e-13)
    u_u, p_u, beta, rhs_u = O.project(case.phi, None, case.u_star, h, lam=case.lam, tol=1e-13)
    assert np.allclose(rhs_s, rhs_u * h ** 3, rtol=1e-13, atol=1e-13 * np.abs(rhs_u * h ** 3).max())
    assert np.linalg.norm(p_s - p_u) <= 1e-10 * np.linalg.norm(p_u)
    for a, b in zip(u_s, u_u):
        assert np.abs(a - b).max() <= 1e-10 * max(np.abs(b).max(), 1.0)


def test_linear_pressure_face_gradients_exact():
    """p = z at the cell centres: every open z-face's (p_R - p_L) / d is 1, so the correction
    subtracts dt * beta exactly; x and y faces see no gradient."""
    nx, ny, nz = 6, 5, 9
    hx, hy, hz = _widths(nx, 2.0), _widths(ny, 1.5, 1), _widths(nz, 3.5, 2)
    zc = np.cumsum(hz) - hz / 2
    p = np.broadcast_to(zc[:, None, None], (nz, ny, nx)).copy()
    beta = tuple(np.full((nz, ny, nx), 0.7) for _ in range(3))
    bi, area = O.stretched_metrics(hx, hy, hz, beta)
    zero = tuple(np.zeros((nz, ny, nx)) for _ in range(3))
    u = O.correct(bi, p, zero, 1.0, 0.5)
    assert np.allclose(u[2][1:], -0.5 * 0.7, rtol=1e-14, atol=0)
    assert np.all(u[2][0] == 0) and np.all(u[0] == 0) and np.all(u[1] == 0)
    # areas: the face's two widths
    assert np.allclose(area[2][1:], (hx[None, :] * hy[:, None])[None], rtol=1e-15)
    assert np.allclose(area[0][:, :, 1:], (hy[None, :, None] * hz[:, None, None]), rtol=1e-15)


def test_stretched_projection_divergence_free():
    case = synth.small_case(16, 16, 16, seed=3, solid="none", interface="wave")
    nz, ny, nx = case.shape
    hx, hy, hz = _widths(nx, 1.5), _widths(ny, 2.0, 1), _widths(nz, 3.5, 2)
    u, p, bi, area, rhs = O.project_stretched(case.phi, hx, hy, hz, case.u_star, lam=case.lam, tol=1e-12)
    d = O.divergence_area(area, u, 1.0, 1.0)
    assert np.linalg.norm(d) <= 1e-9 * np.linalg.norm(rhs)


def test_layered_problem_matches_1d_finite_volumes():
    """phi(z) and u* = (0, 0, w(z)) on a grid stretched in z: p depends on z only and solves the
    one-dimensional finite-volume system sum over the cell's z-faces of beta_f (p_nb - p_c) / d_f
    = sum +-w_f (per unit area), assembled here from the widths alone."""
    nx = ny = 4
    nz = 24
    hz = _widths(nz, 3.5, 1)
    hx = np.full(nx, 0.05)   # columns about as wide as the z-cells (the face area cancels in p)
    hy = np.full(ny, 0.05)
    zc = np.cumsum(hz) - hz / 2
    zf = np.concatenate([[0.0], np.cumsum(hz)])
    phi1 = 0.5 * (1 - np.tanh((zc - 0.55) / 0.05))
    phi = np.ascontiguousarray(np.broadcast_to(phi1[:, None, None], (nz, ny, nx)))
    w1 = np.sin(3 * zf[:-1]) * (np.arange(nz) > 0)      # low z-faces; the wall face carries 0
    us = (np.zeros((nz, ny, nx)), np.zeros((nz, ny, nx)),
          np.ascontiguousarray(np.broadcast_to(w1[:, None, None], (nz, ny, nx))))
    # one level (nx = 4 does not coarsen): the exact solve's residual floor is ~5e-12 for this
    # 384-cell operator, so solve to 1e-11
    lam = 0.1
    u, p, bi, area, rhs = O.project_stretched(phi, hx, hy, hz, us, lam=lam, tol=1e-11)
    # 1-D system: unknowns p_k; face k (between k-1 and k), k = 1..nz-1
    rho = lam + (1 - lam) * phi1
    A = np.zeros((nz, nz))
    b = np.zeros(nz)
    for k in range(1, nz):
        beta = 2.0 / (rho[k - 1] + rho[k])
        dk = 0.5 * (hz[k - 1] + hz[k])
        g = beta / dk
        A[k, k] -= g
        A[k - 1, k - 1] -= g
        A[k, k - 1] += g
        A[k - 1, k] += g
        b[k - 1] += w1[k]
        b[k] -= w1[k]
    b -= b.mean()
    p1 = np.linalg.lstsq(A, b, rcond=1e-13)[0]
    p1 -= p1.mean()
    col = p[:, 0, 0] - p[:, 0, 0].mean()
    assert np.allclose(col, p1, rtol=0, atol=1e-9 * np.abs(p1).max())
    assert np.allclose(p, p[:, :1, :1], rtol=0, atol=1e-10 * np.abs(p1).max())
