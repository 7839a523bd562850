"""Fractional face areas on the GPU against the oracle (Body Boundary Conditions section,
Eq. integral2), through the C ABI: face areas, the area-weighted coefficient hierarchy and
divergence bit for bit; projections (static and moving body) and the adjoint to the oracle's
solution."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1410_2240_gb300 import synth

from _gpu_util import dev, faces_dev, faces_host, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_2240_gb300 import mgproj
    return mgproj


def _case(nx, ny, nz, seed, centre=(0.52, 0.47, 0.45), r=0.23):
    case = synth.small_case(nx, ny, nz, seed=seed, solid="none", interface="wave")
    h = case.h
    K, J, I = np.meshgrid(np.arange(nz + 1) * h, np.arange(ny + 1) * h, np.arange(nx + 1) * h, indexing="ij")
    ext = np.array([nx, ny, nz]) * h
    c = np.array(centre) * ext
    psi = np.sqrt((I - c[0]) ** 2 + (J - c[1]) ** 2 + ((K - c[2]) * 1.3) ** 2) - r * ext.min()
    return case, np.ascontiguousarray(psi)


def _rigid_velocity(case, V=(0.3, -0.2, 0.1), om=(0.0, 0.2, 0.7), x0=(0.5, 0.5, 0.5)):
    nz, ny, nx = case.shape
    h = case.h
    xc = lambda n: (np.arange(n) + 0.5) * h
    xf = lambda n: np.arange(n) * h
    grids = [np.meshgrid(xc(nz), xc(ny), xf(nx), indexing="ij"), np.meshgrid(xc(nz), xf(ny), xc(nx), indexing="ij"),
             np.meshgrid(xf(nz), xc(ny), xc(nx), indexing="ij")]
    out = []
    for a, (K, J, I) in enumerate(grids):
        X = (I - x0[0], J - x0[1], K - x0[2])
        cross = (om[1] * X[2] - om[2] * X[1], om[2] * X[0] - om[0] * X[2], om[0] * X[1] - om[1] * X[0])
        out.append(V[a] + cross[a])
    return tuple(np.ascontiguousarray(x) for x in out)


CASES = {"cube_16": (16, 16, 16, 3), "ragged_40x24x16": (40, 24, 16, 4), "c2_32": (32, 32, 32, 5)}


@pytest.mark.parametrize("name", list(CASES))
def test_face_areas_bit_exact(mgp, name):
    case, psi = _case(*CASES[name])
    rng = np.random.default_rng(1)
    psi = psi + 1e-3 * rng.standard_normal(psi.shape)
    got = mgp.face_areas(dev(psi), case.h)
    for a, b in zip(faces_host(got), O.face_areas(psi)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name", list(CASES))
def test_area_hierarchy_and_divergence_bit_exact(mgp, name):
    case, psi = _case(*CASES[name])
    areas = O.face_areas(psi)
    beta = O.face_coeffs(case.phi, None, case.lam)
    ctx = mgp.Context(faces_dev(beta), case.h, coarse_max_cells=2048)
    ctx.set_face_areas(faces_dev(areas))
    mg = O.MG(O.area_coeffs(areas, beta), case.h, max_coarse=4096)
    assert ctx.num_levels == mg.nlev
    for l in range(mg.nlev):
        for which in range(4):
            assert np.array_equal(host(ctx.level_array(l, which)), mg.level_array(l, which)), (l, which)
    v = _rigid_velocity(case)
    assert np.array_equal(host(ctx.divergence(faces_dev(case.u_star), dt=0.5)),
                          O.divergence_area(areas, case.u_star, case.h, 0.5))
    ctx.set_body_velocity(faces_dev(v))
    assert np.array_equal(host(ctx.divergence(faces_dev(case.u_star), dt=0.5)),
                          O.divergence_area(areas, case.u_star, case.h, 0.5, v))


@pytest.mark.parametrize("moving", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_projection_with_areas_matches_oracle(mgp, moving, prec):
    case, psi = _case(32, 32, 32, 5)
    areas = O.face_areas(psi)
    v = _rigid_velocity(case) if moving else None
    u_o, p_o, beta, rhs_o = O.project_area(case.phi, areas, case.u_star, case.h, lam=case.lam, tol=1e-11, v=v)
    ctx = mgp.Context(faces_dev(beta), case.h, prec=prec, krylov=1, inner_cycles=2, coarse_max_cells=2048)
    ctx.set_face_areas(faces_dev(areas))
    if moving:
        ctx.set_body_velocity(faces_dev(v))
    u_g, p_g, st = ctx.project(faces_dev(case.u_star), tol=1e-10)
    scale = max(np.abs(x).max() for x in u_o)
    for a, b in zip(faces_host(u_g), u_o):
        assert np.abs(a - b).max() <= 1e-7 * scale
    d = O.divergence_area(areas, faces_host(u_g), case.h, 1.0, v)
    assert np.linalg.norm(d) <= 1e-8 * np.linalg.norm(rhs_o)


def test_adjoint_with_areas_matches_oracle(mgp):
    case, psi = _case(32, 32, 32, 6)
    areas = O.face_areas(psi)
    u_o, p_o, beta, _ = O.project_area(case.phi, areas, case.u_star, case.h, lam=case.lam, tol=1e-11)
    gu_o, gb_o, gphi_o = O.project_adjoint_area(beta, areas, p_o, case.w, case.h, lam=case.lam, tol=1e-11)
    ctx = mgp.Context(faces_dev(beta), case.h, krylov=1, coarse_max_cells=2048)
    ctx.set_face_areas(faces_dev(areas))
    gu_g, gb_g, _ = ctx.project_adjoint(faces_dev(case.w), dev(p_o), tol=1e-12)
    for a, b in zip(faces_host(gu_g), gu_o):
        assert np.abs(a - b).max() <= 1e-7 * max(np.abs(b).max(), 1.0)
    for a, b in zip(faces_host(gb_g), gb_o):
        assert np.abs(a - b).max() <= 1e-7 * max(np.abs(b).max(), 1.0)
    gphi = mgp.phi_grad(faces_dev(beta), gb_g, case.h, rho_air=case.lam)
    assert rel(host(gphi), gphi_o) <= 1e-7


def test_unit_areas_identical_to_whole_faces(mgp):
    case, _ = _case(32, 32, 32, 7)
    beta = O.face_coeffs(case.phi, None, case.lam)
    ones = [np.ones(case.shape) for _ in range(3)]
    ones[0][:, :, 0] = 0
    ones[1][:, 0, :] = 0
    ones[2][0] = 0
    res = []
    for use in (False, True):
        ctx = mgp.Context(faces_dev(beta), case.h, prec="mixed", krylov=1, inner_cycles=2, coarse_max_cells=2048)
        if use:
            ctx.set_face_areas(faces_dev(ones))
        u, p, st = ctx.project(faces_dev(case.u_star), tol=1e-10)
        res.append((faces_host(u), host(p), st.cycles))
    assert res[0][2] == res[1][2] and np.array_equal(res[0][1], res[1][1])
    for a, b in zip(res[0][0], res[1][0]):
        assert np.array_equal(a, b)
