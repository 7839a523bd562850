"""Edge cases and failure reporting of the C ABI on the GPU (no fault is provoked:
every bad input here is rejected on the host or handled by the kernels' guards)."""
import math
import warnings

import numpy as np
import pytest
import torch

import oracle as O
from paper_1410_2240_gb300 import synth

from _gpu_util import case_rhs, dev, faces_dev, faces_host, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_2240_gb300 import mgproj
    return mgproj


def _beta(mgp, case):
    solid = None if case.solid is None else dev(case.solid, torch.uint8)
    return mgp.face_coeffs(dev(case.phi), case.h, solid, rho_air=case.lam)


def test_zero_rhs_gives_zero_pressure(mgp):
    case = synth.small_case(16, seed=1)
    ctx = mgp.Context(_beta(mgp, case), case.h)
    p = torch.full(case.shape, 3.0, dtype=torch.float64, device="cuda")
    p, st = ctx.solve(torch.zeros_like(p), p)
    assert st.cycles == 0 and torch.count_nonzero(p) == 0


def test_constant_rhs_is_incompatible_part_only(mgp):
    """A constant rhs is removed entirely by the compatibility projection (mean removal): p = 0."""
    case = synth.small_case(16, seed=2)
    ctx = mgp.Context(_beta(mgp, case), case.h)
    p, st = ctx.solve(torch.full(case.shape, 5.0, dtype=torch.float64, device="cuda"))
    assert st.rhs_mean_removed == pytest.approx(5.0)
    assert torch.count_nonzero(p) == 0


def test_nan_rhs_is_reported(mgp):
    case = synth.small_case(16, seed=3)
    ctx = mgp.Context(_beta(mgp, case), case.h)
    rhs = dev(case.rhs)
    rhs[3, 4, 5] = float("nan")
    with pytest.raises(mgp.MGError) as e:
        ctx.solve(rhs)
    assert e.value.code == mgp.MG_ERR_NAN


def test_not_converged_keeps_last_iterate(mgp):
    case = synth.case_c2(32)
    beta = _beta(mgp, case)
    ctx = mgp.Context(beta, case.h, max_cycles=2)
    rhs = ctx.divergence(faces_dev(case.u_star))
    with pytest.raises(mgp.NotConverged):
        ctx.solve(rhs)
    p, st = ctx.solve(rhs, allow_not_converged=True)
    assert st.cycles == 2 and 1e-10 < st.rel_resid < 1.0
    assert torch.isfinite(p).all()


def test_all_solid_domain(mgp):
    case = synth.small_case(8, seed=4)
    solid = torch.ones(case.shape, dtype=torch.uint8, device="cuda")
    beta = mgp.face_coeffs(dev(case.phi), case.h, solid)
    assert all(torch.count_nonzero(b) == 0 for b in beta)
    ctx = mgp.Context(beta, case.h)
    p, st = ctx.solve(dev(case.rhs))
    assert torch.count_nonzero(p) == 0


@pytest.mark.parametrize("n", [2, 4, 6, 8])
def test_tiny_grids_single_and_two_levels(mgp, n):
    """n <= 6: the whole grid is the coarsest grid (exact dense solve); n = 8: two levels."""
    case = synth.small_case(n, solid="none", seed=5)
    ctx = mgp.Context(_beta(mgp, case), case.h)
    assert ctx.num_levels == (2 if n == 8 else 1)
    beta_o = O.face_coeffs(case.phi, None, case.lam)
    lab, nc = O.components(beta_o)
    p_dense, _ = O.dense_solve(beta_o, case.rhs, case.h, lab, nc)
    p, st = ctx.solve(dev(case.rhs), tol=1e-12)
    assert rel(host(p), p_dense) <= 1e-10


def test_rejects_bad_arguments(mgp):
    case = synth.small_case(8, seed=6)
    beta = _beta(mgp, case)
    with pytest.raises(mgp.MGError) as e:
        mgp.Context(beta, case.h, nu1=0, nu2=0)
    assert e.value.code == mgp.MG_ERR_ARG
    with pytest.raises(mgp.MGError):
        mgp.Context(beta, -1.0)
    odd = synth.small_case(33, 5, 5, seed=7)
    with pytest.raises(mgp.MGError) as e:
        mgp.Context(_beta(mgp, odd), odd.h)  # 33x5x5 cannot coarsen: 825 cells > 512
    assert "coarse" in str(e.value)
    ctx = mgp.Context(beta, case.h)
    with pytest.raises(mgp.MGError):
        ctx.solve(dev(case.rhs), tol=0.0)
    with pytest.raises((TypeError, ValueError)):
        ctx.solve(dev(case.rhs).float())


def test_update_equals_fresh_setup(mgp):
    a = synth.case_c2(32)
    b = synth.small_case(32, solid="ellipsoid", interface="random", seed=8)
    ctx = mgp.Context(_beta(mgp, a), a.h)
    ctx.update(_beta(mgp, b))
    fresh = mgp.Context(_beta(mgp, b), b.h)
    for l in range(ctx.num_levels):
        for w in range(4):
            assert torch.equal(ctx.level_array(l, w), fresh.level_array(l, w))
    rhs = dev(b.rhs)
    p1, _ = ctx.solve(rhs)
    p2, _ = fresh.solve(rhs)
    assert torch.equal(p1, p2)


def test_non_default_stream(mgp):
    case = synth.case_c2(32)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        beta = _beta(mgp, case)
        ctx = mgp.Context(beta, case.h)
        u, p, st = ctx.project(faces_dev(case.u_star), tol=1e-10)
    s.synchronize()
    uo, po, _, _ = O.project(case.phi, case.solid, case.u_star, case.h, lam=case.lam, tol=1e-12)
    assert rel(host(p), po) <= 1e-9


def _pockets_case(n=32, seed=21):
    """A box split by a solid wall into two chambers, with two sealed pockets (hollow solid cubes
    whose inside is fluid) in one of them: four connected fluid regions."""
    case = synth.small_case(n, solid="wall", seed=seed)
    solid = case.solid.copy()
    for lo, hi in ((3, 9), (20, 27)):
        solid[lo:hi, lo:hi, lo // 2 + 1:lo // 2 + 1 + (hi - lo)] = 1
        solid[lo + 1:hi - 1, lo + 1:hi - 1, lo // 2 + 2:lo // 2 + (hi - lo)] = 0
    case.solid = solid
    return case


@pytest.mark.parametrize("kw", [dict(), dict(krylov=1), dict(prec="mixed", krylov=1, inner_cycles=2),
                                dict(prec="mixed")])
def test_fluid_regions_match_oracle(mgp, kw):
    """Several connected fluid regions (a wall and two sealed pockets): the library labels them and
    pins p to zero mean on each, as the oracle does (the minimum-norm solution of Eq. neumann with
    Eq. pois), so p and u match the oracle's; a velocity field gives a compatible rhs (no warning)."""
    case = _pockets_case()
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    lab, nc = O.components(beta_o)
    live = O.diag_inv(beta_o) > 0
    assert len(np.unique(lab[live])) == 4
    ctx = mgp.Context(_beta(mgp, case), case.h, coarse_max_cells=2048, **kw)
    with warnings.catch_warnings():
        warnings.simplefilter("error", mgp.IncompatibleRhsWarning)
        u, p, st = ctx.project(faces_dev(case.u_star), tol=1e-10)
    uo, po, _, _ = O.project(case.phi, case.solid, case.u_star, case.h, lam=case.lam, tol=1e-12)
    assert rel(host(p), po) <= 1e-9
    scale = max(np.abs(x).max() for x in uo)
    for a, b in zip(faces_host(u), uo):
        assert np.abs(a - b).max() <= 1e-8 * scale
    pg = host(p)
    for m in np.unique(lab[live]):
        assert abs(pg[lab == m].mean()) <= 1e-12 * np.abs(pg).max()


def test_incompatible_rhs_on_regions_is_solved_and_reported(mgp):
    """A raw random rhs has a different mean on each region: each is removed, the solve converges
    to the oracle's solution, and the status MG_ERR_INCOMPATIBLE is reported (a warning in Python)."""
    case = _pockets_case(seed=22)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    p_o, cyc, _ = O.MG(beta_o, case.h, max_coarse=4096).solve(case.rhs, tol=1e-12, max_cycles=300)
    assert cyc > 0
    ctx = mgp.Context(_beta(mgp, case), case.h, coarse_max_cells=2048)
    with pytest.warns(mgp.IncompatibleRhsWarning, match="incompatible"):
        p, st = ctx.solve(dev(case.rhs), tol=1e-10)
    assert st.rel_resid <= 1e-10
    assert rel(host(p), p_o) <= 1e-9
    assert st.rhs_mean_removed == pytest.approx(case.rhs[O.diag_inv(beta_o) > 0].mean(), rel=1e-12)


def test_incompatible_rhs_connected_domain(mgp):
    """One region: a rhs with a mean above 1e-8 of its RMS is reported; its solution is that of the
    mean-free rhs, which alone passes without a warning."""
    case = synth.case_c2(32)
    beta = _beta(mgp, case)
    ctx = mgp.Context(beta, case.h)
    rhs = ctx.divergence(faces_dev(case.u_star))
    rms = float(torch.sqrt((rhs * rhs).mean()))
    with warnings.catch_warnings():
        warnings.simplefilter("error", mgp.IncompatibleRhsWarning)
        p0, st0 = ctx.solve(rhs, tol=1e-11)
        # a shift of 1e-9 x RMS stays below the threshold
        ctx.solve(rhs + 1e-9 * rms, tol=1e-11)
    with pytest.warns(mgp.IncompatibleRhsWarning):
        p1, st1 = ctx.solve(rhs + 1e-6 * rms, tol=1e-11)
    assert st1.rhs_mean_removed == pytest.approx(st0.rhs_mean_removed + 1e-6 * rms, rel=1e-6)
    assert rel(host(p1), host(p0)) <= 1e-10
    # the raw C status
    st = mgp.Stats()
    shifted = rhs + 1e-6 * rms
    p2 = torch.zeros_like(rhs)
    code = mgp._lib.mg_solve(ctx._c, mgp._vp(shifted.data_ptr()), mgp._vp(p2.data_ptr()), 1e-10, mgp.ctypes.byref(st))
    torch.cuda.synchronize()
    assert code == mgp.MG_ERR_INCOMPATIBLE
    assert "incompatible" in mgp._lib.mg_last_error().decode()


def test_launch_counter_advances(mgp):
    case = synth.small_case(16, seed=10)
    n0 = mgp.kernel_launches()
    ctx = mgp.Context(_beta(mgp, case), case.h)
    ctx.solve(dev(case.rhs))
    assert mgp.kernel_launches() > n0
