"""Pins of the oracle's fractional face areas and of the projection on them (Body Boundary
Conditions section, Eq. integral2), checked against closed forms, brute-force integration,
analytic cross-sections and the projection's own invariants; CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_1410_2240_gb300 import synth


def _brute_open(f00, f10, f01, f11, m=400):
    """Fraction of the unit square where the piecewise-linear interpolant of the four corners
    over the four triangles about the centre (centre value = corner mean) is > 0, by sampling
    the m x m cell midpoints.  Coded independently of the closed form."""
    s = (np.arange(m) + 0.5) / m
    S, T = np.meshgrid(s, s, indexing="xy")
    fc = (f00 + f10 + f01 + f11) / 4.0
    # corners: (0,0) f00, (1,0) f10, (0,1) f01, (1,1) f11; triangles share the centre (.5,.5)
    below = T < S          # under the diagonal t = s
    above_anti = T > 1 - S  # over the anti-diagonal t = 1 - s
    val = np.empty_like(S)
    # bottom triangle (00, 10, c): t < s and t < 1 - s
    m0 = below & ~above_anti
    # right triangle (10, 11, c): t < s and t > 1 - s
    m1 = below & above_anti
    # top triangle (11, 01, c): t > s and t > 1 - s
    m2 = ~below & above_anti
    m3 = ~below & ~above_anti  # left (01, 00, c)

    def bary(P, A, B, C, fa, fb, fc_):
        (px, py), (ax, ay), (bx, by), (cx, cy) = P, A, B, C
        det = (by - cy) * (ax - cx) + (cx - bx) * (ay - cy)
        l1 = ((by - cy) * (px - cx) + (cx - bx) * (py - cy)) / det
        l2 = ((cy - ay) * (px - cx) + (ax - cx) * (py - cy)) / det
        return l1 * fa + l2 * fb + (1 - l1 - l2) * fc_

    P = (S, T)
    val = np.where(m0, bary(P, (0, 0), (1, 0), (.5, .5), f00, f10, fc), 0.0)
    val = np.where(m1, bary(P, (1, 0), (1, 1), (.5, .5), f10, f11, fc), val)
    val = np.where(m2, bary(P, (1, 1), (0, 1), (.5, .5), f11, f01, fc), val)
    val = np.where(m3, bary(P, (0, 1), (0, 0), (.5, .5), f01, f00, fc), val)
    return float(np.mean(val > 0))


def test_face_open_closed_forms():
    """Linear psi is reproduced exactly by the four triangles, so the open fraction is the area
    of a half-plane within the unit square."""
    assert O.face_open(1, 2, 3, 4) == 1.0
    assert O.face_open(-1, 0, -2, 0) == 0.0
    for c in (0.1, 0.25, 0.5, 0.9):           # psi = c - t: open for t < c
        assert O.face_open(c, c, c - 1, c - 1) == pytest.approx(c, abs=1e-15)
    for c in (0.2, 0.5, 0.8, 1.0, 1.3, 1.7):  # psi = s + t - c: open where s + t > c
        expect = 1 - c * c / 2 if c <= 1 else (2 - c) ** 2 / 2
        got = O.face_open(-c, 1 - c, 1 - c, 2 - c)
        assert got == pytest.approx(expect, abs=1e-14), c
    # psi = s - c along the other axis
    for c in (0.3, 0.6):
        assert O.face_open(-c, 1 - c, -c, 1 - c) == pytest.approx(1 - c, abs=1e-15)


def test_face_open_matches_brute_force():
    rng = np.random.default_rng(5)
    for _ in range(40):
        f = rng.standard_normal(4)
        got = O.face_open(*f)
        assert 0.0 <= got <= 1.0
        assert got == pytest.approx(_brute_open(*f), abs=3e-3), f


def _nodes(n, h):
    x = np.arange(n + 1) * h
    return np.meshgrid(x, x, x, indexing="ij")  # returns X[i,j,k]


def test_plane_areas_exact():
    """psi = z - z0 (body below z0): vertical faces open above z0, horizontal faces open iff
    above z0, walls 0 -- checks the face/corner indexing of every axis."""
    n, h, z0 = 8, 1.0 / 8, 0.3
    x = np.arange(n + 1) * h
    Z = np.broadcast_to(x[:, None, None], (n + 1, n + 1, n + 1))  # psi[k, j, i] = z_k - z0
    ax, ay, az = O.face_areas(Z - z0)
    k = np.arange(n)
    vert = np.clip(((k + 1) * h - z0) / h, 0, 1)
    assert np.allclose(ax[:, :, 1:], vert[:, None, None], atol=1e-14)
    assert np.allclose(ay[:, 1:, :], vert[:, None, None], atol=1e-14)
    assert np.all(ax[:, :, 0] == 0) and np.all(ay[:, 0, :] == 0) and np.all(az[0] == 0)
    horiz = (k * h > z0).astype(float)
    assert np.array_equal(az[1:], np.broadcast_to(horiz[1:, None, None], az[1:].shape))
    # the same plane along x: psi = x - x0 opens the faces normal to y and z from x0 on
    X = np.broadcast_to(x[None, None, :], (n + 1, n + 1, n + 1))
    bx, by, bz = O.face_areas(X - z0)
    i = np.arange(n)
    vert_x = np.clip(((i + 1) * h - z0) / h, 0, 1)
    assert np.allclose(by[:, 1:, :], vert_x[None, None, :], atol=1e-14)
    assert np.allclose(bz[1:, :, :], vert_x[None, None, :], atol=1e-14)


def test_sphere_cross_sections():
    """Summed open area of the x-faces in a plane x = x_i cutting a sphere: the square minus the
    disc of radius sqrt(r^2 - (x_i - c)^2), to within a band of the disc's perimeter."""
    n = 48
    h = 1.0 / n
    r, c = 0.3, np.array([0.5, 0.47, 0.52])
    x = np.arange(n + 1) * h
    K, J, I = np.meshgrid(x, x, x, indexing="ij")
    psi = np.sqrt((I - c[0]) ** 2 + (J - c[1]) ** 2 + (K - c[2]) ** 2) - r
    ax, ay, az = O.face_areas(psi)
    for i in (10, 18, 24, 30):
        xi = i * h
        rho2 = r * r - (xi - c[0]) ** 2
        disc = np.pi * rho2 if rho2 > 0 else 0.0
        got = ax[:, :, i].sum() * h * h
        assert got == pytest.approx(1.0 - disc, abs=2 * np.pi * np.sqrt(max(rho2, 0)) * h * 0.2 + 1e-12), i
    # z-faces in plane z_k
    k = 20
    rho2 = r * r - (k * h - c[2]) ** 2
    assert az[k].sum() * h * h == pytest.approx(1.0 - np.pi * rho2, abs=2 * np.pi * np.sqrt(rho2) * h * 0.2)


def _sphere_case(n=16, seed=3):
    case = synth.small_case(n, n, n, seed=seed, solid="none", interface="wave")
    h = case.h
    x = np.arange(n + 1) * h
    K, J, I = np.meshgrid(x, x, x, indexing="ij")
    psi = np.sqrt((I - 0.52) ** 2 + (J - 0.47) ** 2 + (K - 0.45) ** 2) - 0.23
    return case, O.face_areas(psi)


def test_unit_areas_reproduce_binary_projection():
    case, _ = _sphere_case()
    nz, ny, nx = case.shape
    ones = tuple(np.ones(case.shape) for _ in range(3))
    ones[0][:, :, 0] = 0
    ones[1][:, 0, :] = 0
    ones[2][0] = 0
    u_a, p_a, _, rhs_a = O.project_area(case.phi, ones, case.u_star, case.h, lam=case.lam)
    u_b, p_b, _, rhs_b = O.project(case.phi, None, case.u_star, case.h, lam=case.lam)
    assert np.array_equal(rhs_a, rhs_b)
    assert np.array_equal(p_a, p_b)
    for a, b in zip(u_a, u_b):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("moving", [False, True])
def test_projection_with_areas_is_divergence_free(moving):
    """D_a (u - v) = 0 after the projection (static body: v = 0; moving: a rigid translation plus
    rotation sampled at the face centres)."""
    case, areas = _sphere_case()
    v = None
    if moving:
        n = case.shape[0]
        h = case.h
        xc = (np.arange(n) + 0.5) * h
        xf = np.arange(n) * h
        Kc, Jc, Ic = np.meshgrid(xc, xc, xc, indexing="ij")
        om, V = np.array([0.0, 0.0, 0.7]), np.array([0.3, -0.2, 0.1])
        # face centres: x-faces at (x_f, y_c, z_c) etc.; v = V + om x (x - x0)
        x0 = np.array([0.52, 0.47, 0.45])
        Kx, Jx, Ix = np.meshgrid(xc, xc, xf, indexing="ij")
        Ky, Jy, Iy = np.meshgrid(xc, xf, xc, indexing="ij")
        Kz, Jz, Iz = np.meshgrid(xf, xc, xc, indexing="ij")
        vx = V[0] + om[1] * (Kx - x0[2]) - om[2] * (Jx - x0[1])
        vy = V[1] + om[2] * (Iy - x0[0]) - om[0] * (Ky - x0[2])
        vz = V[2] + om[0] * (Jz - x0[1]) - om[1] * (Iz - x0[0])
        v = (vx, vy, vz)
    # the moving body's flux sits in cut cells of open area down to 1e-5, which puts the residual's
    # rounding floor near 2e-13: solve to 1e-12
    u, p, beta, rhs = O.project_area(case.phi, areas, case.u_star, case.h, lam=case.lam, tol=1e-12, v=v)
    d0 = O.divergence_area(areas, case.u_star, case.h, 1.0, v)
    d1 = O.divergence_area(areas, u, case.h, 1.0, v)
    assert np.linalg.norm(d1) <= 1e-9 * np.linalg.norm(d0)
    if moving:   # the body term reaches only the cells the body cuts
        cut = (areas[0] > 0) & (areas[0] < 1)
        assert np.abs(d0).max() > 0 and cut.any()


def test_adjoint_with_areas_linearity_and_phi():
    """grad_u* by exact linearity (L = <w, u> is linear in u*), grad_phi by Richardson-extrapolated
    central differences of the forward projection."""
    case, areas = _sphere_case(12, seed=4)
    rng = np.random.default_rng(9)
    w = tuple(rng.standard_normal(case.shape) for _ in range(3))
    u, p, beta, _ = O.project_area(case.phi, areas, case.u_star, case.h, lam=case.lam, tol=1e-14)
    gu, gb, gphi = O.project_adjoint_area(beta, areas, p, w, case.h, lam=case.lam, tol=1e-14)
    L = lambda us, phi: sum(float((x * y).sum()) for x, y in zip(
        O.project_area(phi, areas, us, case.h, lam=case.lam, tol=1e-14)[0], w))
    du = tuple(rng.standard_normal(case.shape) for _ in range(3))
    lin = L(tuple(a + b for a, b in zip(case.u_star, du)), case.phi) - L(case.u_star, case.phi)
    assert lin == pytest.approx(sum(float((g * d).sum()) for g, d in zip(gu, du)), rel=1e-9)
    # phi: a few interface cells, and a few cells whose low x-face the body cuts (0 < a < 1),
    # where the area enters the coefficient gradient
    idx = list(np.argwhere((case.phi > 0.05) & (case.phi < 0.95))[:4])
    cut = np.argwhere((areas[0] > 0) & (areas[0] < 1))
    assert len(cut) >= 4
    idx += list(cut[np.random.default_rng(11).choice(len(cut), size=4, replace=False)])
    for (k, j, i) in idx:
        def Lphi(e):
            ph = case.phi.copy()
            ph[k, j, i] += e
            return L(case.u_star, ph)
        e = 1e-3
        d1 = (Lphi(e) - Lphi(-e)) / (2 * e)
        d2 = (Lphi(e / 2) - Lphi(-e / 2)) / e
        fd = (4 * d2 - d1) / 3
        assert gphi[k, j, i] == pytest.approx(fd, rel=1e-5, abs=1e-8 * max(1.0, abs(fd)))


def test_area_divergence_composes_with_plain_divergence():
    """D_a (u - v) is the (pinned) open-face divergence of a (u - v): the area weights each flux,
    the body velocity enters every open face, and nothing else changes."""
    case, areas = _sphere_case(12, seed=6)
    rng = np.random.default_rng(2)
    v = tuple(rng.standard_normal(case.shape) for _ in range(3))
    mask = tuple(np.where(a > 0, 1.0, 0.0) for a in areas)
    for vv in (None, v):
        got = O.divergence_area(areas, case.u_star, case.h, 0.5, vv)
        flux = tuple(a * (u - (0.0 if vv is None else x)) for a, u, x in
                     zip(areas, case.u_star, (0, 0, 0) if vv is None else vv))
        ref = O.divergence(mask, flux, case.h, 0.5)
        assert np.array_equal(got, ref)
