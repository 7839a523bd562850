"""Pins of the oracle's elementary operators against what the paper and mathematics fix.

CPU only.  Every test here checks the oracle against something other than itself:
hand-derived values (tests/golden), closed forms, invariants, textbook/library
special cases, or brute force.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.stats

import oracle as O
from paper_1410_2240_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _beta_random(nx, ny, nz, seed, solid=None, lo=0.5, hi=2.0):
    """Random positive coefficients on interior faces (walls zero)."""
    rng = np.random.default_rng(seed)
    bx = rng.uniform(lo, hi, (nz, ny, nx))
    by = rng.uniform(lo, hi, (nz, ny, nx))
    bz = rng.uniform(lo, hi, (nz, ny, nx))
    bx[:, :, 0] = 0
    by[:, 0, :] = 0
    bz[0, :, :] = 0
    if solid is not None:
        cx, cy, cz = synth.closed_face_masks(solid, solid.shape)
        bx[cx] = 0
        by[cy] = 0
        bz[cz] = 0
    return bx, by, bz


# --- face coefficients (Eq. density; Poisson-solver section) ----------------

def test_face_coeffs_golden_pairs():
    g = json.load(open(os.path.join(GOLD, "face_coeffs.json")))
    for pr in g["pairs"]:
        phi = np.array([[[pr["phiL"], pr["phiR"]]]])
        bx, by, bz = O.face_coeffs(phi, None, g["lam"])
        assert bx[0, 0, 0] == 0.0  # low wall
        assert bx[0, 0, 1] == pytest.approx(pr["beta"], rel=1e-15)
        assert np.all(by == 0) and np.all(bz == 0)


def test_face_coeffs_is_harmonic_mean_of_inverse_density():
    case = synth.small_case(6, interface="random", seed=3)
    lam = case.lam
    bx, by, bz = O.face_coeffs(case.phi, None, lam)
    rho = lam + (1 - lam) * case.phi
    inv = 1.0 / rho
    hx = scipy.stats.hmean(np.stack([inv[:, :, :-1], inv[:, :, 1:]]), axis=0)
    hy = scipy.stats.hmean(np.stack([inv[:, :-1, :], inv[:, 1:, :]]), axis=0)
    hz = scipy.stats.hmean(np.stack([inv[:-1], inv[1:]]), axis=0)
    np.testing.assert_allclose(bx[:, :, 1:], hx, rtol=1e-14)
    np.testing.assert_allclose(by[:, 1:, :], hy, rtol=1e-14)
    np.testing.assert_allclose(bz[1:], hz, rtol=1e-14)
    assert np.all(bx[:, :, 0] == 0) and np.all(by[:, 0, :] == 0) and np.all(bz[0] == 0)


def test_face_coeffs_solid_faces_closed():
    case = synth.small_case(10, solid="ellipsoid", seed=1)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    closed = synth.closed_face_masks(case.solid, case.solid.shape)
    for b, c in zip(beta, closed):
        assert np.all(b[c] == 0)
        assert np.all(b[~c] > 0)


# --- operator A (Eq. pois, finite-volume form of Eq. integral2) -------------

def test_stencil_golden_3x3x3():
    g = json.load(open(os.path.join(GOLD, "stencil_3x3x3.json")))
    n = 3
    bx = np.ones((n, n, n))
    by = np.ones((n, n, n))
    bz = np.ones((n, n, n))
    bx[:, :, 0] = 0
    by[:, 0, :] = 0
    bz[0] = 0
    sf = g["special_face"]
    bx[sf["k"], sf["j"], sf["i"]] = sf["beta"]
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    p = (i + 10 * j + 100 * k).astype(float)
    Ap = O.apply_A((bx, by, bz), p, g["h"])
    for v in g["values"]:
        ii, jj, kk = v["ijk"]
        assert Ap[kk, jj, ii] == v["Ap"]


def test_constant_coefficient_operator_is_neumann_laplacian():
    """beta = 1: A must be the 7-point Neumann Laplacian built as a Kronecker sum (scipy)."""
    nx, ny, nz, h = 5, 4, 3, 0.25
    beta = O.face_coeffs(np.ones((nz, ny, nx)), None, 1e-3)

    def lap1(n):
        main = -2.0 * np.ones(n)
        main[0] = main[-1] = -1.0
        return sp.diags([np.ones(n - 1), main, np.ones(n - 1)], [-1, 0, 1])

    L = (sp.kron(sp.kron(sp.eye(nz), sp.eye(ny)), lap1(nx)) + sp.kron(sp.kron(sp.eye(nz), lap1(ny)), sp.eye(nx))
         + sp.kron(sp.kron(lap1(nz), sp.eye(ny)), sp.eye(nx))) / h ** 2
    A = O.dense_A(beta, h)
    np.testing.assert_allclose(A, L.toarray(), rtol=0, atol=1e-12)


def test_dense_operator_matches_independent_assembly():
    case = synth.small_case(6, ny=5, nz=4, solid="ellipsoid", seed=2)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    _, A_py = O.dense_solve(beta, np.zeros(case.shape), case.h)
    A_c = O.dense_A(beta, case.h)
    np.testing.assert_allclose(A_c, A_py, rtol=1e-15, atol=0)


@pytest.mark.parametrize("solid", ["none", "ellipsoid", "wall"])
def test_operator_invariants(solid):
    case = synth.small_case(10, ny=8, nz=6, solid=solid, seed=4)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(case.shape)
    y = rng.standard_normal(case.shape)
    Ax = O.apply_A(beta, x, case.h)
    Ay = O.apply_A(beta, y, case.h)
    scale = np.linalg.norm(Ax) * np.linalg.norm(y)
    # symmetry
    assert abs(np.vdot(Ax, y) - np.vdot(x, Ay)) <= 1e-14 * scale
    # negative semi-definite
    assert np.vdot(Ax, x) <= 0
    # flux conservation: sum of A x over all cells vanishes
    assert abs(Ax.sum()) <= 1e-13 * np.abs(Ax).sum()
    # null space: constants per component
    lab, nc = O.components(beta)
    v = np.zeros(case.shape)
    for m in range(nc):
        v[lab == m] = rng.standard_normal()
    assert np.abs(O.apply_A(beta, v, case.h)).max() <= 1e-10 * np.abs(v).max() * np.max(beta[0]) / case.h ** 2


def test_components_counts():
    c = synth.small_case(8, solid="wall", seed=0)
    beta = O.face_coeffs(c.phi, c.solid, c.lam)
    lab, nc = O.components(beta)
    nsolid = int(c.solid.sum())
    assert nc == 2 + nsolid
    c = synth.small_case(10, solid="ellipsoid", seed=0)
    beta = O.face_coeffs(c.phi, c.solid, c.lam)
    lab, nc = O.components(beta)
    assert nc == 1 + int(c.solid.sum())


def test_diag_inv_is_inverse_of_minus_h2_diagonal():
    case = synth.small_case(6, solid="ellipsoid", seed=5)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    A = O.dense_A(beta, case.h)
    d = -np.diag(A) * case.h ** 2
    dinv = O.diag_inv(beta).ravel()
    expect = np.where(d > 0, 1.0 / np.where(d > 0, d, 1), 0.0)
    np.testing.assert_allclose(dinv, expect, rtol=1e-15)


# --- smoother ----------------------------------------------------------------

@pytest.mark.parametrize("colour", [0, 1])
def test_colour_sweep_zeroes_that_colours_residual(colour):
    """Gauss-Seidel on one colour solves each of that colour's rows exactly."""
    case = synth.small_case(8, ny=6, nz=10, solid="ellipsoid", seed=6)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    lab, nc = O.components(beta)
    b = O.remove_mean(case.rhs, lab, nc)
    dinv = O.diag_inv(beta)
    p0 = np.random.default_rng(1).standard_normal(case.shape)
    p1 = O.smooth_colour(beta, dinv, b, p0, case.h, colour)
    k, j, i = np.meshgrid(*[np.arange(n) for n in case.shape], indexing="ij")
    mine = ((i + j + k) % 2 == colour) & (dinv > 0)
    r = O.residual(beta, b, p1, case.h)
    assert np.abs(r[mine]).max() <= 1e-11 * np.abs(b).max()
    # the other colour is untouched
    assert np.array_equal(p1[~mine & (dinv > 0)], p0[~mine & (dinv > 0)])


def test_gauss_seidel_fixed_point():
    case = synth.small_case(8, seed=7)
    beta = O.face_coeffs(case.phi, None, case.lam)
    lab, nc = O.components(beta)
    b = O.remove_mean(case.rhs, lab, nc)
    p, _ = O.cg_solve(beta, b, case.h, tol=1e-14)
    dinv = O.diag_inv(beta)
    q = O.smooth_colour(beta, dinv, b, p, case.h, 0)
    q = O.smooth_colour(beta, dinv, b, q, case.h, 1)
    assert np.abs(q - p).max() <= 1e-10 * np.abs(p).max()


# --- transfers ---------------------------------------------------------------

def test_coefficient_restriction_invariants():
    nx, ny, nz = 8, 6, 4
    beta = O.face_coeffs(np.ones((nz, ny, nx)), None, 1e-3)
    cb = O.restrict_coeffs(beta)
    # constant beta = 1 stays 1 on interior coarse faces; coarse walls are 0
    assert np.all(cb[0][:, :, 1:] == 1) and np.all(cb[0][:, :, 0] == 0)
    assert np.all(cb[1][:, 1:, :] == 1) and np.all(cb[1][:, 0, :] == 0)
    assert np.all(cb[2][1:] == 1) and np.all(cb[2][0] == 0)
    # total conductance of a coarse face plane = 1/4 of the fine plane's
    beta = _beta_random(nx, ny, nz, 3)
    cb = O.restrict_coeffs(beta)
    for I in range(nx // 2):
        assert cb[0][:, :, I].sum() == pytest.approx(0.25 * beta[0][:, :, 2 * I].sum(), rel=1e-14)
    for J in range(ny // 2):
        assert cb[1][:, J, :].sum() == pytest.approx(0.25 * beta[1][:, 2 * J, :].sum(), rel=1e-14)
    for K in range(nz // 2):
        assert cb[2][K].sum() == pytest.approx(0.25 * beta[2][2 * K].sum(), rel=1e-14)
    # a coarse face is closed iff its 4 fine faces are closed
    sol = np.zeros((nz, ny, nx), np.uint8)
    sol[:, :, 3:5] = 1
    beta = _beta_random(nx, ny, nz, 4, solid=sol)
    cb = O.restrict_coeffs(beta)
    fine_closed = (beta[0][0::2, 0::2, 0::2] == 0) & (beta[0][1::2, 0::2, 0::2] == 0) & \
                  (beta[0][0::2, 1::2, 0::2] == 0) & (beta[0][1::2, 1::2, 0::2] == 0)
    assert np.array_equal(cb[0] == 0, fine_closed)


def test_restriction_is_child_average():
    rng = np.random.default_rng(2)
    r = rng.standard_normal((6, 8, 10))
    rc = O.restrict(r)
    ref = r.reshape(3, 2, 4, 2, 5, 2).mean(axis=(1, 3, 5))
    np.testing.assert_allclose(rc, ref, rtol=1e-14)
    assert O.restrict(np.full((4, 4, 4), 3.5)).tolist() == np.full((2, 2, 2), 3.5).tolist()


def test_prolongation_reproduces_linear_fields_and_constants():
    nx, ny, nz = 12, 8, 16
    dinv = np.ones((nz, ny, nx))
    NX, NY, NZ = nx // 2, ny // 2, nz // 2
    # coarse centres in fine-cell units: X = 2I + 1 (fine centre i + 1/2 -> position i + 0.5)
    K, J, I = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
    a, b, c, d = 0.3, -1.7, 2.1, 0.9
    ec = a * (2 * I + 1) + b * (2 * J + 1) + c * (2 * K + 1) + d
    p = O.prolong_add(ec, dinv, np.zeros((nz, ny, nx)))
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lin = a * (i + 0.5) + b * (j + 0.5) + c * (k + 0.5) + d
    interior = (i >= 1) & (i <= nx - 2) & (j >= 1) & (j <= ny - 2) & (k >= 1) & (k <= nz - 2)
    np.testing.assert_allclose(p[interior], lin[interior], rtol=0, atol=1e-12)
    # constants are reproduced everywhere (clamping keeps the weights' sum at 1)
    p = O.prolong_add(np.full((NZ, NY, NX), 2.5), dinv, np.zeros((nz, ny, nx)))
    np.testing.assert_allclose(p, 2.5, rtol=1e-15)
    # cells with dinv = 0 are not touched
    dinv[0, 0, 0] = 0
    p = O.prolong_add(np.full((NZ, NY, NX), 2.5), dinv, np.zeros((nz, ny, nx)))
    assert p[0, 0, 0] == 0 and p[0, 0, 1] == 2.5


def test_prolongation_weights_at_a_wall_corner():
    """Fine cell (0,0,0): parent (0,0,0), the other neighbour clamps onto the parent: value e(0,0,0).
    Fine cell (1,1,1): 27/64 e000 + 9/64 (e100 + e010 + e001) + 3/64 (e110 + e101 + e011) + 1/64 e111."""
    ec = np.arange(8, dtype=float).reshape(2, 2, 2) ** 2 + 1.0
    p = O.prolong_add(ec, np.ones((4, 4, 4)), np.zeros((4, 4, 4)))
    assert p[0, 0, 0] == pytest.approx(ec[0, 0, 0], rel=1e-15)
    e = lambda i, j, k: ec[k, j, i]
    expect = (27 * e(0, 0, 0) + 9 * (e(1, 0, 0) + e(0, 1, 0) + e(0, 0, 1)) + 3 * (e(1, 1, 0) + e(1, 0, 1) + e(0, 1, 1))
              + e(1, 1, 1)) / 64
    assert p[1, 1, 1] == pytest.approx(expect, rel=1e-15)


# --- dense pseudo-inverse ----------------------------------------------------

def test_pinv_matches_numpy_and_penrose_conditions():
    case = synth.small_case(4, seed=8)
    beta = O.face_coeffs(case.phi, None, case.lam)
    A = O.dense_A(beta, case.h)
    X = O.pinv_sym(A)
    Xn = np.linalg.pinv(A, rcond=1e-10)
    np.testing.assert_allclose(X, Xn, rtol=0, atol=1e-11 * np.abs(Xn).max())
    np.testing.assert_allclose(A @ X @ A, A, atol=1e-10 * np.abs(A).max())
    np.testing.assert_allclose(X @ A @ X, X, atol=1e-10 * np.abs(X).max())
    np.testing.assert_allclose(A @ X, (A @ X).T, atol=1e-10)
    # with isolated cells (zero rows) and two components
    c = synth.small_case(4, solid="wall", seed=1)
    beta = O.face_coeffs(c.phi, c.solid, c.lam)
    A = O.dense_A(beta, c.h)
    X = O.pinv_sym(A)
    np.testing.assert_allclose(X, np.linalg.pinv(A, rcond=1e-10), atol=1e-11 * np.abs(X).max())


# --- closed forms ------------------------------------------------------------

@pytest.mark.parametrize("k", [(1, 0, 0), (2, 3, 1), (5, 1, 4)])
def test_eigenmodes_of_constant_density_operator(k):
    nx, ny, nz = 16, 12, 8
    h = 1.0 / nx
    beta = O.face_coeffs(np.ones((nz, ny, nx)), None, 1e-3)
    v = synth.fourier_mode(nx, ny, nz, *k)
    lam = -(4 / h ** 2) * sum(math.sin(math.pi * kd / (2 * n)) ** 2 for kd, n in zip(k, (nx, ny, nz)))
    np.testing.assert_allclose(O.apply_A(beta, v, h), lam * v, rtol=0, atol=1e-10 * abs(lam))
    p, cyc, _ = O.MG(beta, h).solve(v, tol=1e-13)
    assert cyc > 0
    np.testing.assert_allclose(p, v / lam, rtol=0, atol=1e-12 * np.abs(v / lam).max())
