"""Pins of the oracle's time step (Numerical Time Integration section): the VOF operator (upwind
fluxes) against a hand-worked example, exact mass conservation and free-stream preservation under a
divergence-free flow, boundedness; the Runge-Kutta step keeps a hydrostatic column at rest, leaves a
divergence-free velocity unchanged without forces, and returns a divergence-free velocity; CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_1410_2240_gb300 import synth


def _stream_flow(nx, ny, nz, h, amp=1.0):
    """u = curl of (0, psi, 0), psi = amp sin(pi x/Lx) sin(pi z/Lz) at the x-z edges: discretely
    divergence-free, no flow through the walls, uniform in y."""
    Lx, Lz = nx * h, nz * h
    xe = np.arange(nx + 1) * h
    ze = np.arange(nz + 1) * h
    psi = amp * np.sin(np.pi * xe[None, :] / Lx) * np.sin(np.pi * ze[:, None] / Lz)   # (nz+1, nx+1)
    ux = (psi[1:, :nx] - psi[:-1, :nx]) / h           # x-face (i, k): edges (i, k) and (i, k+1)
    uz = -(psi[:nz, 1:nx + 1] - psi[:nz, :nx]) / h     # z-face (i, k): edges (i, k) and (i+1, k)
    ux = np.broadcast_to(ux[:, None, :], (nz, ny, nx)).copy()
    uz = np.broadcast_to(uz[:, None, :], (nz, ny, nx)).copy()
    ux[:, :, 0] = 0.0
    uz[0] = 0.0
    return ux, np.zeros((nz, ny, nx)), uz


def test_vof_upwind_hand_example():
    """Three cells in x, flow +1 through both interior faces: the first cell loses u phi_0 through
    its high face, the middle gains it and loses u phi_1, the last gains u phi_1 (times dt/h)."""
    phi = np.array([0.9, 0.4, 0.1]).reshape(1, 1, 3)
    beta = (np.array([0.0, 1.0, 1.0]).reshape(1, 1, 3), np.zeros((1, 1, 3)), np.zeros((1, 1, 3)))
    u = (np.array([0.0, 1.0, 1.0]).reshape(1, 1, 3), np.zeros((1, 1, 3)), np.zeros((1, 1, 3)))
    v = O.vof_upwind(beta, u, phi, 0.5, 0.1)[0, 0]
    s = 0.1 / 0.5
    assert np.allclose(v, [s * 0.9, s * (0.4 - 0.9), s * (-0.4)], rtol=1e-15, atol=0)
    # reversed flow takes the other cells' values
    u2 = (np.array([0.0, -1.0, -1.0]).reshape(1, 1, 3), np.zeros((1, 1, 3)), np.zeros((1, 1, 3)))
    v2 = O.vof_upwind(beta, u2, phi, 0.5, 0.1)[0, 0]
    assert np.allclose(v2, [-s * 0.4, s * (0.4 - 0.1), s * 0.1], rtol=1e-15, atol=0)


def test_vof_conserves_mass_and_constants():
    n = 24
    case = synth.small_case(n, 8, n, seed=2, solid="none", interface="wave")
    beta = O.face_coeffs(case.phi, None, case.lam)
    u = _stream_flow(n, 8, n, case.h)
    d = O.divergence(beta, u, case.h)
    assert np.abs(d).max() <= 1e-12 * np.abs(u[0]).max() / case.h
    dt = 0.2 * case.h / np.abs(u[0]).max()
    v = O.vof_upwind(beta, u, case.phi, case.h, dt)
    assert abs(v.sum()) <= 1e-13 * np.abs(v).sum()
    const = O.vof_upwind(beta, u, np.full(case.shape, 0.37), case.h, dt)
    assert np.abs(const).max() <= 1e-13
    new = case.phi - v
    assert new.min() >= -1e-14 and new.max() <= 1 + 1e-14


def test_rk2_hydrostatic_column_stays_at_rest():
    """Flat interface, fluid at rest, gravity: the pressure balances the body force in both
    stages, so the velocity stays zero and the volume fraction does not move."""
    case = synth.small_case(16, 16, 16, seed=1, solid="none", interface="flat")
    zero = tuple(np.zeros(case.shape) for _ in range(3))
    dt, g = 0.01, 1.0
    u1, phi1, P = O.rk2_step(case.phi, None, zero, case.h, dt, g, lam=case.lam, tol=1e-12)
    assert max(np.abs(x).max() for x in u1) <= 1e-9 * dt * g
    assert np.abs(phi1 - case.phi).max() <= 1e-9
    # the pressure is hydrostatic: at rest the correction cancels the body force face by face,
    # so on every interior z-face (P_k - P_{k-1}) / h = -g / beta_z = -g (rho_{k-1} + rho_k) / 2
    rho = case.lam + (1.0 - case.lam) * case.phi
    slope = (P[1:] - P[:-1]) / case.h
    expect = -g * 0.5 * (rho[1:] + rho[:-1])
    assert np.abs(slope - expect).max() <= 1e-8 * g


def test_rk2_keeps_divergence_free_velocity_without_forces():
    n = 16
    case = synth.small_case(n, 8, n, seed=4, solid="none", interface="wave")
    u = _stream_flow(n, 8, n, case.h, amp=0.05)
    u1, phi1, P = O.rk2_step(case.phi, None, u, case.h, 0.5 * case.h, 0.0, lam=case.lam, tol=1e-12)
    for a, b in zip(u1, u):
        assert np.abs(a - b).max() <= 1e-10 * np.abs(u[0]).max()


def test_rk2_returns_divergence_free_velocity():
    case = synth.small_case(16, 16, 16, seed=5, solid="ellipsoid", interface="wave")
    u1, phi1, P = O.rk2_step(case.phi, case.solid, case.u_star, case.h, 0.2 * case.h, 1.0, lam=case.lam, tol=1e-12)
    beta = O.face_coeffs(phi1, case.solid, case.lam)  # the mask only depends on the solid
    d = O.divergence(beta, u1, case.h)
    assert np.abs(d).max() <= 1e-9 * np.abs(O.divergence(beta, case.u_star, case.h)).max()
