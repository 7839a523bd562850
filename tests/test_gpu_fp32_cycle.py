"""One FP32 V-cycle of the mixed solves against the oracle's FP64 V-cycle, cell by cell.

mg_vcycle on a mixed context runs the cycle the mixed solves use -- FP32 storage and arithmetic,
the colour-split finest level with its uniform-row or banded-row records, the FP64 coarsest solve
-- on the caller's FP64 right-hand side and iterate rounded to FP32, and widens the result.  The
oracle's cycle is the same map in FP64 (the multigrid of the Poisson-solver section with the
readings of the design notes: red-black Gauss-Seidel, face-coefficient restriction, 8-child mean,
trilinear prolongation, exact coarsest solve).  The two differ by FP32 rounding alone.

Bound: with the FP32 unit roundoff u = 2^-24 = 6.0e-8, each smoothing update rounds ~7 times
(six fused products and the scaling) and a level runs 8 sweeps, but Gauss-Seidel damps the
rounding it has already made, so the smoothed values carry a few u relative to the local
magnitudes; the residual that feeds the coarse-grid correction loses a further factor to
cancellation once the iterate is smooth.  Measured on GB300: 1.9e-7 to 6.1e-7 (3 to 10 u) over
the cases below.  The tests bound max|p_gpu - p_oracle| by 3e-6 max|p_oracle| (50 u) on the first
cycle from p = 0 and on the second from the oracle's first iterate.  A smoother or transfer with
one wrong coefficient, sign or neighbour misses this by orders of magnitude; the cycles the solver
runs are the kernels tested here (k_smooth_split4 with uniform rows at 256^3, with banded-row
records on a z-stretched grid, k_smooth_split where nx % 8 != 0).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1410_2240_gb300 import synth

from _gpu_util import case_rhs, dev, faces_dev, faces_host, host

pytestmark = pytest.mark.gpu

BOUND = 3e-6


@pytest.fixture(scope="module")
def mgp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_2240_gb300 import mgproj
    return mgproj


def _row_kinds(bx, by, bz):
    """Interior x-rows whose faces (all x-faces but the low wall, the two y-faces and the two
    z-faces of every cell) hold one positive value (uniform), or one value per kind of face
    (banded but not uniform).  Vectorised over the rows."""
    vx = bx[1:-1, 1:-1, 1:2]
    okx = np.all(bx[1:-1, 1:-1, 1:] == vx, axis=2)
    vyl, vyh = by[1:-1, 1:-1, :1], by[1:-1, 2:, :1]
    oky = np.all(by[1:-1, 1:-1, :] == vyl, axis=2) & np.all(by[1:-1, 2:, :] == vyh, axis=2) & (vyl == vyh)[..., 0]
    vzl, vzh = bz[1:-1, 1:-1, :1], bz[2:, 1:-1, :1]
    okz = np.all(bz[1:-1, 1:-1, :] == vzl, axis=2) & np.all(bz[2:, 1:-1, :] == vzh, axis=2)
    pos = (vx > 0)[..., 0] & (vyl > 0)[..., 0] & (vzl > 0)[..., 0] & (vzh > 0)[..., 0]
    band = okx & oky & okz & pos
    uni = band & (vx == vyl)[..., 0] & (vx == vzl)[..., 0] & (vx == vzh)[..., 0]
    return int(uni.sum()), int((band & ~uni).sum())


def _compare_cycles(mgp, mg, ctx, b, label):
    """Two cycles: from p = 0, then from the oracle's first iterate; returns the errors."""
    errs = []
    p = np.zeros(b.shape)
    bd = dev(b)
    for it in range(2):
        pd = dev(p)
        p_o = mg.vcycle(b, p)
        ctx.vcycle(bd, pd)
        pg = host(pd)
        err = float(np.abs(pg - p_o).max() / np.abs(p_o).max())
        errs.append(err)
        print(f"{label} cycle {it + 1}: max|p32 - p64| / max|p64| = {err:.3e}")
        assert err <= BOUND, (label, it, err)
        p = p_o
    return errs


def test_fp32_cycle_256_uniform_rows(mgp):
    """The benchmark's 256^3 workload: most rows uniform (k_smooth_split4 without records)."""
    case = synth.case_c3(256)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    uni, band = _row_kinds(*(x.astype(np.float32) for x in beta_o))
    assert uni > 0.5 * 254 * 254, uni
    b = O.remove_mean(case_rhs(case, beta_o), *O.components(beta_o))
    mg = O.MG(beta_o, case.h)
    beta = mgp.face_coeffs(dev(case.phi), case.h, dev(case.solid, torch.uint8), rho_air=case.lam)
    ctx = mgp.Context(beta, case.h, prec="mixed")
    _compare_cycles(mgp, mg, ctx, b, "c3_256")


def test_fp32_cycle_z_stretched_banded_rows(mgp):
    """A grid stretched in z: rows away from the interface hold four face values (banded-row
    records, k_smooth_split4<BAND>)."""
    n = 64
    case = synth.small_case(n, n, n, seed=7, solid="ellipsoid", interface="flat")
    hx = np.full(n, case.h)
    hy = np.full(n, case.h)
    hz = synth.stretched_widths(n, 3.5, 0.5)
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    bi, area = O.stretched_metrics(hx, hy, hz, beta)
    coef = O.area_coeffs(area, bi)
    uni, band = _row_kinds(*(x.astype(np.float32) for x in coef))
    assert band > uni and band > 0.3 * (n - 2) ** 2, (uni, band)
    rhs = O.divergence_area(area, case.u_star, 1.0, 1.0)
    b = O.remove_mean(rhs, *O.components(coef))
    mg = O.MG(coef, 1.0, max_coarse=4096)
    bo, ao = mgp.stretched_metrics(dev(hx), dev(hy), dev(hz), faces_dev(beta))
    ctx = mgp.Context(bo, 1.0, prec="mixed", coarse_max_cells=2048)
    ctx.set_face_areas(ao)
    _compare_cycles(mgp, mg, ctx, b, "z_stretched_64")


@pytest.mark.parametrize("shape", [(36, 32, 32), (20, 24, 16)])
def test_fp32_cycle_ragged_rows(mgp, shape):
    """nx % 8 != 0 with every axis even: the one-cell-per-thread colour pass (k_smooth_split)."""
    nx, ny, nz = shape
    case = synth.small_case(nx, ny, nz, seed=11, solid="ellipsoid")
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    b = O.remove_mean(case_rhs(case, beta_o), *O.components(beta_o))
    mg = O.MG(beta_o, case.h, max_coarse=4096)
    beta = mgp.face_coeffs(dev(case.phi), case.h, dev(case.solid, torch.uint8), rho_air=case.lam)
    ctx = mgp.Context(beta, case.h, prec="mixed", coarse_max_cells=2048)
    assert ctx.num_levels == mg.nlev >= 2
    _compare_cycles(mgp, mg, ctx, b, f"ragged_{nx}x{ny}x{nz}")


def test_fp32_cycle_c2_128(mgp):
    """128^3, the free surface and the ellipsoid: the coarse levels' natural-layout FP32 passes
    and the one-CTA coarse tail below them."""
    case = synth.case_c2(128)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    b = O.remove_mean(case_rhs(case, beta_o), *O.components(beta_o))
    mg = O.MG(beta_o, case.h)
    beta = mgp.face_coeffs(dev(case.phi), case.h, dev(case.solid, torch.uint8), rho_air=case.lam)
    ctx = mgp.Context(beta, case.h, prec="mixed")
    _compare_cycles(mgp, mg, ctx, b, "c2_128")
