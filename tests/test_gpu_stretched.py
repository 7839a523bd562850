"""Stretched grids on the GPU against the oracle: the metrics bit for bit, projections on a
context built from them (h = 1, the metrics' areas as face areas) to the oracle's solution, and
uniform widths against the library's own uniform projection."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1410_2240_gb300 import synth

from _gpu_util import dev, faces_dev, faces_host, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_2240_gb300 import mgproj
    return mgproj


def _widths(n, ratio, phase=0.0):
    t = (np.arange(n) + 0.5) / n
    w = 1.0 + (ratio - 1.0) * (0.5 - 0.5 * np.cos(2 * np.pi * (t + phase)))
    return w / w.sum()


def _grid(nx, ny, nz):
    return _widths(nx, 1.5), _widths(ny, 2.0, 0.1), _widths(nz, 3.5, 0.2)


@pytest.mark.parametrize("with_frac", [False, True])
def test_metrics_bit_exact(mgp, with_frac):
    case = synth.small_case(24, 16, 32, seed=1, solid="none", interface="wave")
    hx, hy, hz = _grid(24, 16, 32)
    beta = O.face_coeffs(case.phi, None, case.lam)
    frac = None
    if with_frac:
        rng = np.random.default_rng(3)
        frac = tuple(rng.uniform(0.0, 1.0, case.shape) for _ in range(3))
    bo, ao = mgp.stretched_metrics(dev(hx), dev(hy), dev(hz), faces_dev(beta), None if frac is None else faces_dev(frac))
    bo_o, ao_o = O.stretched_metrics(hx, hy, hz, beta, frac)
    for a, b in zip(faces_host(bo) + faces_host(ao), bo_o + ao_o):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_stretched_projection_matches_oracle(mgp, prec):
    case = synth.small_case(32, 32, 32, seed=5, solid="none", interface="wave")
    hx, hy, hz = _grid(32, 32, 32)
    u_o, p_o, bi, area, rhs_o = O.project_stretched(case.phi, hx, hy, hz, case.u_star, lam=case.lam, tol=1e-11)
    beta = O.face_coeffs(case.phi, None, case.lam)
    bo, ao = mgp.stretched_metrics(dev(hx), dev(hy), dev(hz), faces_dev(beta))
    ctx = mgp.Context(bo, 1.0, prec=prec, krylov=1, inner_cycles=2, coarse_max_cells=2048)
    ctx.set_face_areas(ao)
    assert np.array_equal(host(ctx.divergence(faces_dev(case.u_star))), rhs_o)
    u_g, p_g, st = ctx.project(faces_dev(case.u_star), tol=1e-10)
    scale = max(np.abs(x).max() for x in u_o)
    for a, b in zip(faces_host(u_g), u_o):
        assert np.abs(a - b).max() <= 1e-7 * scale
    d = O.divergence_area(area, faces_host(u_g), 1.0, 1.0)
    assert np.linalg.norm(d) <= 1e-8 * np.linalg.norm(rhs_o)


def test_uniform_widths_match_uniform_context(mgp):
    case = synth.small_case(32, 32, 32, seed=6, solid="none", interface="wave")
    n, h = 32, case.h
    w = np.full(n, h)
    beta = mgp.face_coeffs(dev(case.phi), h, None, rho_air=case.lam)
    bo, ao = mgp.stretched_metrics(dev(w), dev(w), dev(w), beta)
    s_ctx = mgp.Context(bo, 1.0, krylov=1, coarse_max_cells=2048)
    s_ctx.set_face_areas(ao)
    u_s, p_s, _ = s_ctx.project(faces_dev(case.u_star), tol=1e-11)
    u_ctx = mgp.Context(beta, h, krylov=1, coarse_max_cells=2048)
    u_u, p_u, _ = u_ctx.project(faces_dev(case.u_star), tol=1e-11)
    pu = host(p_u)
    assert np.linalg.norm(host(p_s) - pu) <= 1e-9 * np.linalg.norm(pu)
    for a, b in zip(faces_host(u_s), faces_host(u_u)):
        assert np.abs(a - b).max() <= 1e-9 * max(np.abs(b).max(), 1.0)


def _row_kinds(bx, by, bz):
    """Numbers of uniform and of banded-but-not-uniform interior rows (every x-face but the wall,
    the low and high y-faces, the low and the high z-faces each holding one positive value)."""
    nz, ny, nx = bx.shape
    uni = band = 0
    for k in range(nz - 1):
        for j in range(ny - 1):
            vx, vy, vzl, vzh = bx[k, j, 1], by[k, j, 0], bz[k, j, 0], bz[k + 1, j, 0]
            ok = (vx > 0 and vy > 0 and vzl > 0 and vzh > 0 and np.all(bx[k, j, 1:] == vx)
                  and np.all(by[k, j] == vy) and np.all(by[k, j + 1] == vy) and np.all(bz[k, j] == vzl)
                  and np.all(bz[k + 1, j] == vzh))
            if ok and vx == vy == vzl == vzh:
                uni += 1
            elif ok:
                band += 1
    return uni, band


def test_z_stretched_banded_rows_bit_identical_to_fused_sweeps(mgp):
    """On a grid stretched in z alone the rows away from the interface hold four face values (x,
    y, low z, high z); the colour passes take them from per-row records instead of loading the
    faces.  The mixed projection (stationary refinement: CG's FP32 dot products would sum the
    colour-split and the natural layout in different orders) must equal, bit for bit, the one whose
    fused sweeps load every face."""
    # a level interface (the face values of a row then depend on its plane alone) and a body, so
    # that both banded rows and rows whose faces are loaded occur
    case = synth.small_case(32, 32, 32, seed=7, solid="ellipsoid", interface="flat")
    h = case.h
    hx = np.full(32, h)
    hy = np.full(32, h)
    hz = _widths(32, 3.5, 0.2)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    bo, ao = mgp.stretched_metrics(dev(hx), dev(hy), dev(hz), faces_dev(beta))
    coef = [(a * b).astype(np.float32) for a, b in zip(faces_host(ao), faces_host(bo))]
    uni, band = _row_kinds(*coef)
    assert band > uni and band < 31 * 31, (uni, band)
    out = []
    for sm in (1, 2):
        ctx = mgp.Context(bo, 1.0, prec="mixed", smoother=sm, coarse_max_cells=2048)
        ctx.set_face_areas(ao)
        u_g, p_g, st = ctx.project(faces_dev(case.u_star), tol=1e-10)
        out.append((p_g, u_g, st.cycles))
    assert out[0][2] == out[1][2]
    assert torch.equal(out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):
        assert torch.equal(a, b)
