"""Edge cases and failure reporting of the C ABI on the GPU (no fault is provoked:
every bad input here is rejected on the host or handled by the kernels' guards)."""
import math

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


def test_two_chambers_velocity_matches_and_pressure_differs_by_constants(mgp):
    """A solid wall splits the fluid.  The velocity is unique and matches the oracle; the
    library's p is mean-zero over all fluid cells, the oracle's per chamber, so they differ by
    one constant per chamber (a documented convention, not an error)."""
    case = synth.small_case(16, solid="wall", seed=9)
    ctx = mgp.Context(_beta(mgp, case), case.h)
    u, p, st = ctx.project(faces_dev(case.u_star), tol=1e-10)
    uo, po, beta_o, _ = O.project(case.phi, case.solid, case.u_star, case.h, lam=case.lam, tol=1e-12)
    scale = max(np.abs(x).max() for x in uo)
    for a, b in zip(faces_host(u), uo):
        assert np.abs(a - b).max() <= 1e-8 * scale
    lab, nc = O.components(beta_o)
    d = host(p) - po
    for m in range(nc):
        sel = lab == m
        assert np.ptp(d[sel]) <= 1e-8 * np.abs(po).max()


def test_launch_counter_advances(mgp):
    case = synth.small_case(16, seed=10)
    n0 = mgp.kernel_launches()
    ctx = mgp.Context(_beta(mgp, case), case.h)
    ctx.solve(dev(case.rhs))
    assert mgp.kernel_launches() > n0
