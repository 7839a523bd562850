"""The allocation-free residual check (mg_residual_norm_noalloc) against mg_solve's report.

This entry point serves callers that cannot call cudaMalloc (device memory owned by a
pool they must not bypass, loops where a possibly synchronising allocation is not
allowed, hosts without an allocator for plug-ins).  It is called here through the C ABI
on two calls in a row and must agree with what mg_solve reports in mg_stats for the same
rhs and initial pressure (relative residual, rhs norm, removed mean), within the 1e-12
relative tolerance the V-cycle parity tests use.  The file name makes pytest collect it
last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1410_2240_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_2240_gb300 import mgproj
    return mgproj


def _call_noalloc(mgp, grid, beta, rhs, p, out):
    code = mgp._lib.mg_residual_norm_noalloc(ctypes.byref(grid), mgp._P3(*[ctypes.c_void_p(b.data_ptr()) for b in beta]),
                                             ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code


def test_noalloc_residual_matches_solver_report(mgp):
    case = synth.case_c2(64)
    dev = lambda a, dt=torch.float64: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
    beta = mgp.face_coeffs(dev(case.phi), case.h, dev(case.solid, torch.uint8), rho_air=case.lam)
    ctx = mgp.Context(beta, case.h, max_cycles=0)  # reports the initial iterate's residual
    rhs = ctx.divergence(tuple(dev(x) for x in case.u_star)) + 0.25  # a mean to remove
    nlive = int((ctx.level_array(0, 3) > 0).sum().item())
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(11)
    for call in range(2):
        p0 = dev(rng.standard_normal(case.shape) * (0.01 if call else 1.0))
        p_solver = p0.clone()
        _, st = ctx.solve(rhs, p_solver, allow_not_converged=True)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        assert _call_noalloc(mgp, ctx.grid, beta, rhs, p0, out) == mgp.MG_OK, mgp._lib.mg_last_error()
        torch.cuda.synchronize()
        if call == 1:  # after the first call's one-time set-up, a call allocates nothing
            assert torch.cuda.mem_get_info()[0] == free_before
        r = out.cpu().numpy()
        assert r[0] == pytest.approx(st.rel_resid, rel=1e-12)
        assert r[1] == pytest.approx(st.rhs_norm, rel=1e-12)
        assert r[2] == pytest.approx(st.rhs_mean_removed, rel=1e-12)
        assert r[3] == nlive


def test_noalloc_rejects_too_many_planes(mgp):
    grid = mgp.Grid(2, 2, 4097, 1.0)
    x = torch.zeros(4097 * 4, dtype=torch.float64, device="cuda")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    code = mgp._lib.mg_residual_norm_noalloc(ctypes.byref(grid), mgp._P3(*[ctypes.c_void_p(x.data_ptr())] * 3),
                                             ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()), None)
    assert code == mgp.MG_ERR_ARG
    assert b"4096" in mgp._lib.mg_last_error()
