"""Pins of the oracle's solvers, projection and adjoint (CPU only)."""
import math
import numpy as np
import pytest

import oracle as O
from paper_1410_2240_gb300 import synth


def _compat(beta, b):
    lab, nc = O.components(beta)
    return O.remove_mean(b, lab, nc), lab, nc


@pytest.mark.parametrize("solid", ["none", "ellipsoid"])
def test_mg_matches_dense_pseudoinverse_8cubed(solid):
    """Brute force: dense least-squares minimum-norm solution on 8^3, density ratio 1000."""
    case = synth.small_case(8, solid=solid, seed=11)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    lab, nc = O.components(beta)
    p_dense, _ = O.dense_solve(beta, case.rhs, case.h, lab, nc)
    p, cyc, _ = O.MG(beta, case.h).solve(case.rhs, tol=1e-13, max_cycles=200)
    assert cyc > 0
    assert np.linalg.norm(p - p_dense) <= 1e-11 * np.linalg.norm(p_dense)


def test_mg_matches_dense_two_chambers():
    """A solid wall splits the box: p is mean-zero in each chamber, solid cells hold 0."""
    case = synth.small_case(8, solid="wall", seed=12)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    lab, nc = O.components(beta)
    p_dense, _ = O.dense_solve(beta, case.rhs, case.h, lab, nc)
    p, cyc, _ = O.MG(beta, case.h).solve(case.rhs, tol=1e-13, max_cycles=300)
    assert cyc > 0
    assert np.linalg.norm(p - p_dense) <= 1e-11 * np.linalg.norm(p_dense)
    assert np.all(p[case.solid.astype(bool)] == 0)
    for m in range(nc):
        assert abs(p[lab == m].mean()) <= 1e-13 * np.abs(p).max()


def test_layered_density_reduces_to_thomas():
    """phi = phi(z), b = b(z): the solution is z-only and equals the tridiagonal (Thomas) solve.

    Tolerance: the 1-D operator with a 1000:1 coefficient jump has condition number
    ~1e6 here, so two backward-stable FP64 solves may differ by ~cond * eps ~ 1e-10."""
    nx, ny, nz = 16, 16, 64
    case = synth.small_case(nx, ny, nz, interface="flat", seed=13)
    beta = O.face_coeffs(case.phi, None, case.lam)
    bcol = np.random.default_rng(3).standard_normal(nz)
    b = np.broadcast_to(bcol[:, None, None], (nz, ny, nx)).copy()
    p, cyc, _ = O.MG(beta, case.h).solve(b, tol=1e-12, max_cycles=200)
    assert cyc > 0
    pz = O.thomas_layered(beta[2][:, 0, 0], bcol, case.h)
    # z-only
    assert np.abs(p - p[:, :1, :1]).max() <= 1e-12 * np.abs(pz).max()
    np.testing.assert_allclose(p, np.broadcast_to(pz[:, None, None], p.shape), rtol=0,
                               atol=1e-10 * np.abs(pz).max())


@pytest.mark.parametrize("name", ["c1", "c2_64"])
def test_cg_and_mg_agree(name):
    """Two algorithms (Jacobi-PCG, the paper's earlier solver family, and multigrid) reach one answer."""
    case = synth.case_c1() if name == "c1" else synth.case_c2(64)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    rhs = case.rhs if case.rhs is not None else O.divergence(beta, case.u_star, case.h)
    p_mg, cyc, _ = O.MG(beta, case.h).solve(rhs, tol=1e-13, max_cycles=200)
    p_cg, it = O.cg_solve(beta, rhs, case.h, tol=1e-13, max_it=50000)
    assert cyc > 0 and it > 0
    assert np.linalg.norm(p_mg - p_cg) <= 1e-11 * np.linalg.norm(p_cg)
    p_mg10, cyc10, _ = O.MG(beta, case.h).solve(rhs, tol=1e-10)
    assert np.linalg.norm(p_mg10 - p_cg) <= 1e-9 * np.linalg.norm(p_cg)


@pytest.mark.parametrize("name", ["c1", "c2_64"])
def test_residual_decreases_monotonically(name):
    case = synth.case_c1() if name == "c1" else synth.case_c2(64)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    rhs = case.rhs if case.rhs is not None else O.divergence(beta, case.u_star, case.h)
    p, cyc, hist = O.MG(beta, case.h).solve(rhs, tol=1e-12)
    assert cyc > 0
    assert np.all(np.diff(hist) < 0)
    assert hist[-1] <= 1e-12


def test_vcycle_error_energy_norm_decreases():
    case = synth.case_c2(32)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    b, lab, nc = _compat(beta, O.divergence(beta, case.u_star, case.h))
    mg = O.MG(beta, case.h)
    p_ex, _, _ = mg.solve(b, tol=1e-14, max_cycles=300)
    p = np.zeros_like(b)
    prev = None
    for _ in range(6):
        p = O.remove_mean(mg.vcycle(b, p), lab, nc)
        e = p - p_ex
        en = -np.vdot(e, O.apply_A(beta, e, case.h))
        if prev is not None:
            assert en < prev
        prev = en


def test_vcycle_commutes_with_constant_shift():
    """V(p + c) = V(p) + c on every non-isolated cell (A annihilates constants)."""
    case = synth.small_case(16, solid="ellipsoid", seed=14)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    b, lab, nc = _compat(beta, case.rhs)
    mg = O.MG(beta, case.h)
    p = np.random.default_rng(0).standard_normal(case.shape)
    live = O.diag_inv(beta) > 0
    a = mg.vcycle(b, p)
    c = mg.vcycle(b, p + 3.0)
    np.testing.assert_allclose(c[live] - a[live], 3.0, rtol=0, atol=1e-9)


# --- projection --------------------------------------------------------------

def _proj_case(n=12, solid="ellipsoid", seed=15):
    return synth.small_case(n, solid=solid, seed=seed)


def test_projection_is_divergence_free_and_idempotent():
    case = _proj_case()
    u, p, beta, rhs = O.project(case.phi, case.solid, case.u_star, case.h, dt=2.5e-4, lam=case.lam, tol=1e-13)
    du = O.divergence(beta, u, case.h)
    assert np.linalg.norm(du) <= 1e-11 * np.linalg.norm(rhs * 2.5e-4)
    u2, p2, _, _ = O.project(case.phi, case.solid, u, case.h, dt=2.5e-4, lam=case.lam, tol=1e-13)
    for a, b in zip(u, u2):
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-12 * max(np.abs(x).max() for x in u))
    assert np.abs(p2).max() <= 1e-10 * np.abs(p).max()


def test_projection_dt_invariance():
    """u does not depend on dt; p scales as 1/dt."""
    case = _proj_case(seed=16)
    u1, p1, _, _ = O.project(case.phi, case.solid, case.u_star, case.h, dt=1.0, lam=case.lam, tol=1e-13)
    u2, p2, _, _ = O.project(case.phi, case.solid, case.u_star, case.h, dt=0.25, lam=case.lam, tol=1e-13)
    for a, b in zip(u1, u2):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
    np.testing.assert_allclose(p2, 4.0 * p1, rtol=0, atol=1e-10 * np.abs(p2).max())


def test_projection_dot_product_test():
    """<P a, b> = <a, P^T b>: forward projection against the adjoint's grad_u."""
    case = _proj_case(seed=17)
    rng = np.random.default_rng(5)
    a = synth.random_face_field(rng, case.shape, 1.0, case.solid)
    bw = synth.random_face_field(rng, case.shape, 1.0, case.solid)
    Pa, p, beta, _ = O.project(case.phi, case.solid, a, case.h, lam=case.lam, tol=1e-13)
    gu, _, _ = O.project_adjoint(beta, p, bw, case.h, lam=case.lam, tol=1e-13)
    lhs = sum(np.vdot(x, y) for x, y in zip(Pa, bw))
    rhs = sum(np.vdot(x, y) for x, y in zip(a, gu))
    # each side carries the error of a solve stopped at relative residual 1e-13, amplified by
    # the conditioning of A (density ratio 1000); a wrong sign or transpose gives O(1)
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs))


def test_projection_is_orthogonal_in_beta_inverse_inner_product():
    """P is the B^-1-orthogonal projector onto div-free fields: <P a, B^-1 (a - P a)> = 0 on open faces."""
    case = _proj_case(seed=18)
    Pa, p, beta, _ = O.project(case.phi, case.solid, case.u_star, case.h, lam=case.lam, tol=1e-13)
    s = 0.0
    norm = 0.0
    for x, y, b in zip(Pa, case.u_star, beta):
        m = b > 0
        s += np.sum(x[m] * (y[m] - x[m]) / b[m])
        norm += np.sum(y[m] * y[m] / b[m])
    assert abs(s) <= 1e-11 * norm


def test_adjoint_phi_gradient_central_differences():
    """grad_phi against FP64 central differences of L = sum(w * u) (solves to 1e-13), at the
    paper's production step dt = 2.5e-4 (u and L do not depend on dt; p and the adjoint's dt G p
    terms do, so a dropped dt shows)."""
    case = synth.small_case(12, solid="ellipsoid", interface="wave", seed=19)
    lam, h, dt = case.lam, case.h, 2.5e-4

    def loss(phi):
        u, _, _, _ = O.project(phi, case.solid, case.u_star, h, dt=dt, lam=lam, tol=1e-13)
        return sum(np.vdot(a, b) for a, b in zip(u, case.w))

    u, p, beta, _ = O.project(case.phi, case.solid, case.u_star, h, dt=dt, lam=lam, tol=1e-13)
    _, _, gphi = O.project_adjoint(beta, p, case.w, h, dt=dt, lam=lam, tol=1e-13)
    # cells in the interface band where the gradient is largest
    band = np.argwhere((case.phi > 0.05) & (case.phi < 0.95) & (case.solid == 0))
    rng = np.random.default_rng(6)
    picks = band[rng.choice(len(band), size=8, replace=False)]
    for k, j, i in picks:
        # central differences at eps and eps/2, Richardson-extrapolated (error O(eps^4));
        # a bare central difference at small eps is dominated by the solves' residual noise
        def cd(eps):
            pp = case.phi.copy()
            pp[k, j, i] += eps
            pm = case.phi.copy()
            pm[k, j, i] -= eps
            return (loss(pp) - loss(pm)) / (2 * eps)
        eps = 1e-3
        fd = (4 * cd(eps / 2) - cd(eps)) / 3
        assert abs(fd - gphi[k, j, i]) <= 1e-6 * max(abs(fd), 1e-6 * np.abs(gphi).max()), (k, j, i, fd, gphi[k, j, i])


def test_adjoint_u_gradient_is_exact_for_linear_loss():
    """L = sum(w * P u*) is linear in u*: directional derivative = <grad_u*, d>."""
    case = _proj_case(seed=20)
    rng = np.random.default_rng(7)
    d = synth.random_face_field(rng, case.shape, 1.0, case.solid)
    u, p, beta, _ = O.project(case.phi, case.solid, case.u_star, case.h, lam=case.lam, tol=1e-13)
    gu, _, _ = O.project_adjoint(beta, p, case.w, case.h, lam=case.lam, tol=1e-13)
    up = [a + b for a, b in zip(case.u_star, d)]
    u2, _, _, _ = O.project(case.phi, case.solid, up, case.h, lam=case.lam, tol=1e-13)
    dl = sum(np.vdot(a - b, w) for a, b, w in zip(u2, u, case.w))
    pred = sum(np.vdot(g, x) for g, x in zip(gu, d))
    assert abs(dl - pred) <= 1e-11 * (abs(dl) + abs(pred))


# --- multigrid-preconditioned CG (the next solver row) ------------------------

@pytest.mark.parametrize("vcycles", [1, 2])
def test_pcg_matches_dense_pseudoinverse(vcycles):
    case = synth.small_case(8, solid="ellipsoid", seed=21)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    lab, nc = O.components(beta)
    p_dense, _ = O.dense_solve(beta, case.rhs, case.h, lab, nc)
    p, it, _ = O.MG(beta, case.h).pcg(case.rhs, tol=1e-13, vcycles=vcycles)
    assert it > 0
    assert np.linalg.norm(p - p_dense) <= 1e-11 * np.linalg.norm(p_dense)


@pytest.mark.parametrize("name", ["c1", "c2_64"])
def test_pcg_and_stationary_cycles_agree(name):
    case = synth.case_c1() if name == "c1" else synth.case_c2(64)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    rhs = case.rhs if case.rhs is not None else O.divergence(beta, case.u_star, case.h)
    mg = O.MG(beta, case.h)
    p_mg, c1, _ = mg.solve(rhs, tol=1e-13, max_cycles=200)
    for k in (1, 2):
        p, it, hist = mg.pcg(rhs, tol=1e-13, vcycles=k)
        assert it > 0
        assert np.linalg.norm(p - p_mg) <= 1e-10 * np.linalg.norm(p_mg)
        assert it < c1  # Krylov acceleration of the same cycle needs fewer iterations
    lab, nc = O.components(beta)
    b = O.remove_mean(rhs, lab, nc)
    p, it, _ = mg.pcg(rhs, tol=1e-10, vcycles=2)
    assert np.linalg.norm(O.residual(beta, b, p, case.h)) <= 1e-10 * np.linalg.norm(b)


def test_pcg_closed_form_eigenmode():
    nx, ny, nz = 16, 12, 8
    h = 1.0 / nx
    beta = O.face_coeffs(np.ones((nz, ny, nx)), None, 1e-3)
    k = (3, 2, 1)
    v = synth.fourier_mode(nx, ny, nz, *k)
    lam = -(4 / h ** 2) * sum(math.sin(math.pi * kd / (2 * n)) ** 2 for kd, n in zip(k, (nx, ny, nz)))
    p, it, _ = O.MG(beta, h).pcg(v, tol=1e-13, vcycles=1)
    np.testing.assert_allclose(p, v / lam, rtol=0, atol=1e-12 * np.abs(v / lam).max())
