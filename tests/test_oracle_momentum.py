"""Pins of the oracle's momentum right-hand side R_i (Eq. navi without the pressure and sub-grid
terms: convective, viscous with mu(phi) of Eq. density, and body force) and of the time step that
uses it (Numerical Time Integration section); CPU only.

* Exactness: the central conservative MAC forms are exact, at faces whose stencils stay clear of
  the walls, for a linear velocity (convective term: (div u) u_i + (u . grad) u_i) and for a
  quadratic velocity with a linear viscosity (viscous term: d_j (mu (d_j u_i + d_i u_j)), here in
  closed form), times 1/rho on the face.
* Walls (free-slip): closed forms of a shear u_x(y) and of a flux v(y) u_x(y) next to the y-walls.
* Mirror symmetry about each axis (any index slip on one side of a stencil breaks it).
* Body force alone, closed faces zero.
* The Runge-Kutta step is second order in time (Heun's method on the projected equations): the
  error falls ~4x when dt halves, for a viscous flow with convection.
"""
import numpy as np
import pytest

import oracle as O
from paper_1410_2240_gb300 import synth

MU_AIR = 1.8e-2


def _face_positions(n, h):
    """Positions of the x-, y- and z-faces (low-face layout), each a tuple (x, y, z) of arrays of
    shape (nz, ny, nx)."""
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy, cz = (i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h
    return ((i * h, cy, cz), (cx, j * h, cz), (cx, cy, k * h))


def _poly_field(n, h, c, B, H):
    """u_a(x) = c_a + B_a . x + x^T H_a x / 2 sampled at the a-faces; wall faces 0."""
    pos = _face_positions(n, h)
    u = []
    for a in range(3):
        x = np.stack(pos[a])  # (3, nz, ny, nx)
        v = c[a] + np.einsum("j,jzyx->zyx", B[a], x) + 0.5 * np.einsum("jl,jzyx,lzyx->zyx", H[a], x, x)
        v = v.copy()
        if a == 0:
            v[:, :, 0] = 0.0
        elif a == 1:
            v[:, 0, :] = 0.0
        else:
            v[0] = 0.0
        u.append(v)
    return tuple(u), pos


def _open_beta(n, rng=None):
    """1/rho on the faces: 1 (or random in [0.5, 2]) on every face but the walls."""
    nx, ny, nz = n
    b = [np.ones((nz, ny, nx)) if rng is None else rng.uniform(0.5, 2.0, (nz, ny, nx)) for _ in range(3)]
    b[0][:, :, 0] = 0.0
    b[1][:, 0, :] = 0.0
    b[2][0] = 0.0
    return tuple(b)


def _interior(n, a):
    """Faces of axis a whose stencils use no wall face and no mirrored value: index along a in
    [2, n_a - 2], along the others in [1, n - 2]."""
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    idx = (i, j, k)
    m = np.ones((nz, ny, nx), bool)
    for b in range(3):
        lo, hi = (2, n[b] - 2) if b == a else (1, n[b] - 2)
        m &= (idx[b] >= lo) & (idx[b] <= hi)
    return m


N = (10, 9, 8)
H = 0.1


def test_convective_term_exact_for_linear_velocity():
    rng = np.random.default_rng(1)
    c = rng.standard_normal(3)
    B = rng.standard_normal((3, 3))
    u, pos = _poly_field(N, H, c, B, np.zeros((3, 3, 3)))
    phi = np.ones((N[2], N[1], N[0]))
    R = O.momentum_rhs(phi, _open_beta(N), u, H, g=0.0, inv_re=0.0, mu_air=MU_AIR, convect=True)
    div = np.trace(B)
    for a in range(3):
        x = np.stack(pos[a])
        ua = c[a] + np.einsum("j,jzyx->zyx", B[a], x)
        uvec = [c[b] + np.einsum("j,jzyx->zyx", B[b], x) for b in range(3)]
        exact = -(div * ua + sum(uvec[b] * B[a, b] for b in range(3)))
        m = _interior(N, a)
        assert np.abs(R[a][m] - exact[m]).max() <= 1e-12 * np.abs(exact[m]).max(), a


@pytest.mark.parametrize("variable_mu", [False, True])
def test_viscous_term_exact_for_quadratic_velocity(variable_mu):
    """d_j (mu (d_j u_i + d_i u_j)) for a quadratic u, mu constant or linear (from a linear phi),
    times inv_re / rho_face (random 1/rho on the faces)."""
    rng = np.random.default_rng(2)
    c = rng.standard_normal(3)
    B = rng.standard_normal((3, 3))
    Hq = rng.standard_normal((3, 3, 3))
    Hq = 0.5 * (Hq + Hq.transpose(0, 2, 1))
    u, pos = _poly_field(N, H, c, B, Hq)
    nx, ny, nz = N
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    if variable_mu:
        p0, pv = 0.4, np.array([0.3, -0.2, 0.5])
    else:
        p0, pv = 1.0, np.zeros(3)
    phi = p0 + pv[0] * (i + 0.5) * H + pv[1] * (j + 0.5) * H + pv[2] * (k + 0.5) * H
    dmu = 1.0 - MU_AIR
    beta = _open_beta(N, rng)
    inv_re = 0.7
    R = O.momentum_rhs(phi, beta, u, H, g=0.0, inv_re=inv_re, mu_air=MU_AIR, convect=False)
    for a in range(3):
        x = np.stack(pos[a])
        mu = MU_AIR + dmu * (p0 + np.einsum("j,jzyx->zyx", pv, x))
        gmu = dmu * pv
        # grad u_b at the face: B_b + H_b x
        grad = [B[b][:, None, None, None] + np.einsum("jl,lzyx->jzyx", Hq[b], x) for b in range(3)]
        lap = np.trace(Hq[a]) + sum(Hq[b][a, b] for b in range(3))
        term = mu * lap + sum(gmu[b] * (grad[a][b] + grad[b][a]) for b in range(3))
        exact = inv_re * beta[a] * term
        m = _interior(N, a)
        assert np.abs(R[a][m] - exact[m]).max() <= 1e-10 * np.abs(exact[m]).max(), a


def test_free_slip_walls_shear_closed_form():
    """u_x = f(y) on every interior x-face, no other velocity, mu = 1, rho = 1: away from the
    x-walls R_x = (f_{j+1} - 2 f_j + f_{j-1}) / h^2 with the mirror values f_{-1} = f_0 and
    f_{ny} = f_{ny-1} (no shear at the y-walls), and R_y = 0."""
    nx, ny, nz = N
    f = np.random.default_rng(3).standard_normal(ny)
    ux = np.broadcast_to(f[None, :, None], (nz, ny, nx)).copy()
    ux[:, :, 0] = 0.0
    u = (ux, np.zeros_like(ux), np.zeros_like(ux))
    R = O.momentum_rhs(np.ones_like(ux), _open_beta(N), u, H, inv_re=1.0, mu_air=MU_AIR, convect=False)
    fe = np.concatenate([[f[0]], f, [f[-1]]])
    lap = (fe[2:] - 2 * fe[1:-1] + fe[:-2]) / H ** 2
    assert np.allclose(R[0][:, :, 2:nx - 1], lap[None, :, None], rtol=1e-12, atol=1e-12 * np.abs(lap).max())
    assert np.abs(R[1][:, 1:, 1:nx - 1]).max() <= 1e-12 * np.abs(lap).max()


def test_free_slip_walls_flux_closed_form():
    """u_x = f(y), v = g(y) (zero on the y-walls), both uniform in x and z: away from the x-walls
    R_x = -(F_{j+1} - F_j)/h with F_j = g_j (f_{j-1} + f_j)/2 at the edge of rows j-1, j, no flux
    through the walls (g_0 = g_ny = 0) and the mirror value f_{-1} = f_0."""
    nx, ny, nz = N
    rng = np.random.default_rng(4)
    f = rng.standard_normal(ny)
    gv = np.concatenate([[0.0], rng.standard_normal(ny - 1)])
    ux = np.broadcast_to(f[None, :, None], (nz, ny, nx)).copy()
    ux[:, :, 0] = 0.0
    uy = np.broadcast_to(gv[None, :, None], (nz, ny, nx)).copy()
    R = O.momentum_rhs(np.ones_like(ux), _open_beta(N), (ux, uy, np.zeros_like(ux)), H, inv_re=0.0,
                       mu_air=MU_AIR, convect=True)
    fm = np.concatenate([[f[0]], f[:-1]])       # f_{j-1} for j = 0..ny-1, mirrored at j = 0
    F = np.concatenate([gv * 0.5 * (fm + f), [0.0]])   # edges j = 0..ny
    exact = -(F[1:] - F[:-1]) / H
    assert np.allclose(R[0][:, :, 2:nx - 1], exact[None, :, None], rtol=1e-12, atol=1e-12 * np.abs(exact).max())


def _mirror(a, n, fields_faces, fields_cells):
    """Reflect the domain about the mid-plane of axis a: face arrays of axis a map face m to
    n_a - m with a sign change, every other array flips its cells along a."""
    ax = 2 - a  # numpy axis of grid axis a

    def flip_faces(v, own, sign):
        if not own:
            return np.flip(v, ax).copy()
        out = np.zeros_like(v)
        sl = [slice(None)] * 3
        sl[ax] = slice(1, None)
        src = np.flip(np.take(v, np.arange(1, n[a]), axis=ax), ax)
        out[tuple(sl)] = sign * src
        return out

    faces = [tuple(flip_faces(f[b], b == a, s) for b in range(3)) for f, s in fields_faces]
    cells = [np.flip(c, ax).copy() for c in fields_cells]
    return faces, cells


@pytest.mark.parametrize("a", [0, 1, 2])
def test_mirror_symmetry(a):
    """R of the reflected state is the reflected R (velocity component along the axis changes
    sign): a random velocity, density and viscosity, a body, every term but gravity."""
    case = synth.small_case(12, 10, 8, seed=5, solid="ellipsoid", interface="random")
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    u = case.u_star
    R = O.momentum_rhs(case.phi, beta, u, case.h, g=0.0, inv_re=0.3, mu_air=MU_AIR, convect=True)
    (um, bm, Rm), (phim,) = _mirror(a, (12, 10, 8), [(u, -1.0), (beta, 1.0), (R, -1.0)], [case.phi])
    R2 = O.momentum_rhs(phim, bm, um, case.h, g=0.0, inv_re=0.3, mu_air=MU_AIR, convect=True)
    scale = max(np.abs(x).max() for x in R)
    for b in range(3):
        assert np.abs(R2[b] - Rm[b]).max() <= 1e-12 * scale, b


def test_body_force_alone_and_closed_faces():
    case = synth.small_case(12, seed=6, solid="ellipsoid")
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    zero = tuple(np.zeros_like(b) for b in beta)
    R = O.momentum_rhs(case.phi, beta, zero, case.h, g=2.5, inv_re=0.1, mu_air=MU_AIR, convect=True)
    assert np.array_equal(R[0], np.zeros_like(R[0])) and np.array_equal(R[1], np.zeros_like(R[1]))
    assert np.array_equal(R[2], np.where(beta[2] > 0, -2.5, 0.0))
    R = O.momentum_rhs(case.phi, beta, case.u_star, case.h, g=2.5, inv_re=0.1, mu_air=MU_AIR, convect=True)
    for b in range(3):
        assert np.all(R[b][beta[b] == 0] == 0.0)
        assert np.any(R[b][beta[b] > 0] != 0.0)


def _tg_flow(n, h, amp=1.0):
    """A discretely divergence-free flow in the x-z plane: u = curl (0, psi, 0) with psi at the
    x-z edges, no flux through the walls, plus a y-dependence through the amplitude."""
    nx, ny, nz = n
    Lx, Lz = nx * h, nz * h
    xe = np.arange(nx + 1) * h
    ze = np.arange(nz + 1) * h
    psi = amp * np.sin(np.pi * xe[None, :] / Lx) ** 2 * np.sin(np.pi * ze[:, None] / Lz) ** 2
    ux = (psi[1:, :nx] - psi[:-1, :nx]) / h
    uz = -(psi[:nz, 1:nx + 1] - psi[:nz, :nx]) / h
    ux = np.broadcast_to(ux[:, None, :], (nz, ny, nx)).copy()
    uz = np.broadcast_to(uz[:, None, :], (nz, ny, nx)).copy()
    ux[:, :, 0] = 0.0
    uz[0] = 0.0
    return ux, np.zeros((nz, ny, nx)), uz


def _run(u0, phi, h, T, nsteps, inv_re):
    u = u0
    for _ in range(nsteps):
        u, phi, _ = O.rk2_step(phi, None, u, h, T / nsteps, 0.0, lam=1.0, tol=1e-13, inv_re=inv_re,
                               mu_air=MU_AIR, convect=True)
    return u


def test_rk2_second_order_in_time():
    """Uniform density (lam = 1), viscous flow with convection from a divergence-free start: the
    error against a 128-step solution falls by ~4 (3.4 to 4.8) from 8 to 16 steps, as Heun's method
    does (measured 4.3); a second stage that took R from u^k instead of u* is first order (2.2)."""
    n, h = (16, 16, 16), 1.0 / 16
    u0 = _tg_flow(n, h, amp=0.2)
    phi = np.ones((n[2], n[1], n[0]))
    T, inv_re = 0.04, 0.05
    ref = _run(u0, phi, h, T, 128, inv_re)
    err = []
    for m in (8, 16):
        u = _run(u0, phi, h, T, m, inv_re)
        err.append(np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(u, ref))))
    ratio = err[0] / err[1]
    assert 3.4 <= ratio <= 4.8, (err, ratio)
