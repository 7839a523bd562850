"""GPU <-> oracle parity through the C ABI (libmgproj.so via its ctypes binding).

Tolerances: integer/structural results and the operations the library performs as
separately rounded IEEE operations in the oracle's order (face coefficients, the
coefficient hierarchy, inverse diagonals, divergence, correction, adjoint faces,
phi chain rule) are compared bit for bit.  The V-cycle uses fused multiply-adds and
an independently computed coarsest inverse, so one V-cycle must match the oracle's to
1e-12 relative (FP64).  Solves must reach relative residual 1e-10 (checked with the
oracle's operator) and match the oracle's solution to 1e-9 relative.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1410_2240_gb300 import synth

from _gpu_util import case_rhs, cases_small, dev, faces_dev, faces_host, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mgp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_2240_gb300 import mgproj
    return mgproj


SMALL = cases_small()


def _ctx(mgp, case, **kw):
    beta = mgp.face_coeffs(dev(case.phi), case.h, None if case.solid is None else dev(case.solid, dtype=torch.uint8),
                           rho_air=case.lam, rho_water=1.0)
    kw.setdefault("coarse_max_cells", 2048)
    return beta, mgp.Context(beta, case.h, **kw)


@pytest.mark.parametrize("name", list(SMALL))
def test_face_coeffs_and_hierarchy_bit_exact(mgp, name):
    case = SMALL[name]
    beta_g, ctx = _ctx(mgp, case)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    for a, b in zip(faces_host(beta_g), beta_o):
        assert np.array_equal(a, b)
    mg = O.MG(beta_o, case.h, max_coarse=4096)
    assert ctx.num_levels == mg.nlev
    for l in range(mg.nlev):
        assert ctx.level_dims(l) == mg.level_dims(l)
        for which in range(4):
            assert np.array_equal(host(ctx.level_array(l, which)), mg.level_array(l, which)), (l, which)


@pytest.mark.parametrize("name", list(SMALL))
def test_vcycle_matches_oracle(mgp, name):
    """The solver's own iterates: from p = 0, three V-cycles, each restarted from the oracle's
    iterate.  One GPU V-cycle matches the oracle's to 1e-12 relative."""
    case = SMALL[name]
    beta_g, ctx = _ctx(mgp, case)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    lab, nc = O.components(beta_o)
    b = O.remove_mean(case_rhs(case, beta_o), lab, nc)
    mg = O.MG(beta_o, case.h, max_coarse=4096)
    p = np.zeros(case.shape)
    bd = dev(b)
    for it in range(3):
        pd = dev(p)
        p = mg.vcycle(b, p)
        ctx.vcycle(bd, pd)
        assert rel(host(pd), p) <= 1e-12, (it, rel(host(pd), p))


@pytest.mark.parametrize("name", list(SMALL))
def test_vcycle_from_rough_start(mgp, name):
    """From white noise the first cycle's coarse correction excites the coarsest grid's
    near-null mode, so the map amplifies the (independent, both correct) coarsest inverses'
    rounding by its condition number (~1e4): the bound is 1e-10 here."""
    case = SMALL[name]
    beta_g, ctx = _ctx(mgp, case)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    lab, nc = O.components(beta_o)
    b = O.remove_mean(case_rhs(case, beta_o), lab, nc)
    mg = O.MG(beta_o, case.h, max_coarse=4096)
    rng = np.random.default_rng(7)
    p = np.where(O.diag_inv(beta_o) > 0, rng.standard_normal(case.shape), 0.0)
    pd = dev(p)
    ctx.vcycle(dev(b), pd)
    assert rel(host(pd), mg.vcycle(b, p)) <= 1e-10


@pytest.mark.parametrize("name", ["c1", "c2_64", "ell16", "odd_coarse_24", "aniso_64x32x16"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_matches_oracle(mgp, name, prec):
    case = SMALL[name]
    beta_g, ctx = _ctx(mgp, case, prec=prec)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    rhs = case_rhs(case, beta_o)
    p_o, cyc_o, _ = O.MG(beta_o, case.h, max_coarse=4096).solve(rhs, tol=1e-12, max_cycles=300)
    assert cyc_o > 0
    p_g, st = ctx.solve(dev(rhs), tol=1e-10)
    pg = host(p_g)
    assert st.rel_resid <= 1e-10
    lab, nc = O.components(beta_o)
    b = O.remove_mean(rhs, lab, nc)
    r = O.residual(beta_o, b, pg, case.h)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.0001e-10
    assert rel(pg, p_o) <= 1e-9
    live = O.diag_inv(beta_o) > 0
    assert abs(pg[live].mean()) <= 1e-12 * np.abs(pg).max()
    assert np.all(pg[~live] == 0)
    if prec == "fp64":
        _, cyc10, _ = O.MG(beta_o, case.h, max_coarse=4096).solve(rhs, tol=1e-10, max_cycles=300)
        assert abs(st.cycles - cyc10) <= 1


def test_solve_c2_128_fp64_and_mixed(mgp):
    case = synth.case_c2(128)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    rhs = O.divergence(beta_o, case.u_star, case.h)
    p_o, cyc_o, _ = O.MG(beta_o, case.h).solve(rhs, tol=1e-12)
    lab, nc = O.components(beta_o)
    b = O.remove_mean(rhs, lab, nc)
    for prec in ("fp64", "mixed"):
        _, ctx = _ctx(mgp, case, prec=prec)
        p_g, st = ctx.solve(dev(rhs), tol=1e-10)
        pg = host(p_g)
        r = O.residual(beta_o, b, pg, case.h)
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.0001e-10, prec
        assert rel(pg, p_o) <= 1e-9, prec


@pytest.mark.parametrize("name", ["c2_64", "ell16", "aniso_64x32x16"])
def test_divergence_and_correction_bit_exact(mgp, name):
    case = SMALL[name]
    beta_g, ctx = _ctx(mgp, case)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    u = case.u_star
    for dt in (1.0, 2.5e-4):
        rg = host(ctx.divergence(faces_dev(u), dt=dt))
        assert np.array_equal(rg, O.divergence(beta_o, u, case.h, dt))
    p = np.random.default_rng(3).standard_normal(case.shape)
    ug = faces_host(ctx.correct(faces_dev(u), dev(p), dt=2.5e-4))
    uo = O.correct(beta_o, p, u, case.h, 2.5e-4)
    for a, b in zip(ug, uo):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name", ["c2_64", "ell16"])
def test_projection_matches_oracle(mgp, name):
    case = SMALL[name]
    beta_g, ctx = _ctx(mgp, case)
    uo, po, beta_o, rhs = O.project(case.phi, case.solid, case.u_star, case.h, lam=case.lam, tol=1e-12)
    ug, pg, st = ctx.project(faces_dev(case.u_star), tol=1e-10)
    ug = faces_host(ug)
    scale = max(np.abs(x).max() for x in uo)
    for a, b in zip(ug, uo):
        assert np.abs(a - b).max() <= 1e-8 * scale
    du = O.divergence(beta_o, ug, case.h)
    assert np.linalg.norm(du) <= 1.0001e-10 * np.linalg.norm(O.remove_mean(rhs, *O.components(beta_o)))


@pytest.mark.parametrize("name", ["c2_64", "ell16"])
def test_adjoint_faces_and_phi_grad_bit_exact_given_p_q(mgp, name):
    """Given the same p and w, the adjoint (its own solve for q) matches the oracle's to the solve
    tolerance, and the phi chain rule on the oracle's grad_beta is bit-exact."""
    case = SMALL[name]
    beta_g, ctx = _ctx(mgp, case)
    uo, po, beta_o, _ = O.project(case.phi, case.solid, case.u_star, case.h, lam=case.lam, tol=1e-12)
    gu_o, gb_o, gphi_o = O.project_adjoint(beta_o, po, case.w, case.h, lam=case.lam, tol=1e-12)
    gu_g, gb_g, st = ctx.project_adjoint(faces_dev(case.w), dev(po), tol=1e-12)
    for a, b in zip(faces_host(gu_g), gu_o):
        assert np.abs(a - b).max() <= 1e-8 * max(np.abs(b).max(), 1.0)
    for a, b in zip(faces_host(gb_g), gb_o):
        assert np.abs(a - b).max() <= 1e-8 * max(np.abs(b).max(), 1e-300)
    # phi chain rule bit-exact on the oracle's grad_beta
    gphi_g = host(mgp.phi_grad(beta_g, faces_dev(gb_o), case.h, rho_air=case.lam))
    assert np.array_equal(gphi_g, O.phi_grad(beta_o, gb_o, case.lam))


# rows longer than one block of the row-sharing kernels (k_phi_grad, k_divergence_mul): the x+
# products at the blocks' right edges are formed again there; h = 1/520 (division by h)
WIDE = "wide_520x32x32"


def _adjoint_case(name):
    if name == WIDE:
        return synth.small_case(520, 32, 32, seed=11, solid="ellipsoid")
    return SMALL[name]


@pytest.mark.parametrize("name", ["c2_64", "ell16", WIDE])
def test_adjoint_faces_bit_exact_given_q(mgp, name):
    """The adjoint's face gradients from the library's own q (read back through q_out) equal the
    oracle's formulas on the same p, q and w bit for bit: grad_u* = w - G q and grad_beta =
    dt (G p)(G q - w) on open faces, w and 0 on closed ones.  The right-hand side D(beta w) of
    that solve has the oracle's norm once its region means are removed (a dropped beta, sign or
    face would change it at O(1))."""
    case = _adjoint_case(name)
    beta_g, ctx = _ctx(mgp, case)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    p = np.random.default_rng(5).standard_normal(case.shape)
    dt = 2.5e-4
    q = torch.zeros(case.shape, dtype=torch.float64, device="cuda")
    gu_g, gb_g, st = ctx.project_adjoint(faces_dev(case.w), dev(p), dt=dt, tol=1e-10, q=q)
    qg = host(q)
    assert np.abs(qg).max() > 0
    gq = O.gradient(beta_o, qg, case.h)
    gp = O.gradient(beta_o, p, case.h)
    for b, x, g, a, ug, bg in zip(beta_o, case.w, gq, gp, faces_host(gu_g), faces_host(gb_g)):
        assert np.array_equal(ug, np.where(b > 0, x - g, x))
        assert np.array_equal(bg, np.where(b > 0, dt * a * (g - x), 0.0))
    c = O.divergence(beta_o, tuple(b * x for b, x in zip(beta_o, case.w)), case.h, 1.0)
    lab, nc = O.components(beta_o)
    assert st.rhs_norm == pytest.approx(np.linalg.norm(O.remove_mean(c, lab, nc)), rel=1e-12)


FUSED_CASES = {
    "c2_64": lambda: synth.case_c2(64),
    "ragged_160x32x32": lambda: synth.small_case(160, 32, 32, solid="ellipsoid", seed=41),
    "ragged_48x24x40": lambda: synth.small_case(48, 24, 40, solid="ellipsoid", seed=42),
    "aniso_64x32x16": lambda: synth.small_case(64, 32, 16, solid="ellipsoid", seed=43),
    "odd_x_34x16x16": lambda: synth.small_case(34, 16, 16, solid="none", seed=44),
    "c3_256": lambda: synth.case_c3(256),
}


@pytest.mark.parametrize("name", list(FUSED_CASES))
def test_fused_sweep_bit_identical_to_colour_passes(mgp, name):
    """The fused red-black sweeps (one pass, overlapped tiles, z-wavefront; register-staged for
    smoother=2, TMA-staged for FP32 in auto mode) give bit-identical V-cycles (FP64) and mixed
    solves (FP32 cycles) to one pass per colour."""
    case = FUSED_CASES[name]()
    beta = mgp.face_coeffs(dev(case.phi), case.h, None if case.solid is None else dev(case.solid, dtype=torch.uint8),
                           rho_air=case.lam)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    b = O.remove_mean(case_rhs(case, beta_o), *O.components(beta_o))
    bd = dev(b)
    colour = mgp.Context(beta, case.h, smoother=1, coarse_max_cells=2048)
    fused = mgp.Context(beta, case.h, smoother=2, coarse_max_cells=2048)
    p1 = torch.zeros_like(bd)
    p2 = torch.zeros_like(bd)
    for _ in range(3):
        colour.vcycle(bd, p1)
        fused.vcycle(bd, p2)
        assert torch.equal(p1, p2)
    m1 = mgp.Context(beta, case.h, prec="mixed", smoother=1, coarse_max_cells=2048)
    q1, s1 = m1.solve(bd, tol=1e-10)
    for sm in (0, 2, 3):
        m = mgp.Context(beta, case.h, prec="mixed", smoother=sm, coarse_max_cells=2048)
        q, st = m.solve(bd, tol=1e-10)
        assert st.cycles == s1.cycles and torch.equal(q, q1), sm


@pytest.mark.parametrize("name", ["c2_64", "ragged_160x32x32", "ragged_48x24x40", "c3_256"])
def test_pass_order_identical(mgp, name):
    """The finest colour passes in alternating plane order (descending, ascending, ...) and the
    restriction descending give bit-identical mixed solves (stationary and CG) to ascending order:
    the cells a colour pass updates do not depend on one another."""
    case = FUSED_CASES[name]()
    beta = mgp.face_coeffs(dev(case.phi), case.h, None if case.solid is None else dev(case.solid, dtype=torch.uint8),
                           rho_air=case.lam)
    rhs = mgp.Context(beta, case.h, coarse_max_cells=2048).divergence(faces_dev(case.u_star))
    for kw in ({"krylov": 0}, {"krylov": 1, "inner_cycles": 2}):
        res = []
        for order in (0, 1):
            ctx = mgp.Context(beta, case.h, prec="mixed", pass_order=order, coarse_max_cells=2048, **kw)
            q, st = ctx.solve(rhs, tol=1e-10)
            res.append((q, st.cycles))
        assert res[0][1] == res[1][1] and torch.equal(res[0][0], res[1][0]), kw


@pytest.mark.parametrize("name", ["c1", "c2_64", "ell16", "odd_coarse_24", "aniso_64x32x16"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("vcycles", [1, 2])
def test_pcg_solve_matches_oracle(mgp, name, prec, vcycles):
    """Multigrid-preconditioned CG on the GPU: residual 1e-10 by the oracle's operator, the oracle's
    solution to 1e-9, and the oracle's PCG iteration count (FP64 cycles) within one at the library's
    CG target of 0.4 tol (mixed: FP32 cycles that preconditioned worse would need more iterations)."""
    case = SMALL[name]
    beta_g, ctx = _ctx(mgp, case, prec=prec, krylov=1, inner_cycles=vcycles)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    rhs = case_rhs(case, beta_o)
    mg = O.MG(beta_o, case.h, max_coarse=4096)
    p_o, _, _ = mg.solve(rhs, tol=1e-12, max_cycles=300)
    p_g, st = ctx.solve(dev(rhs), tol=1e-10)
    pg = host(p_g)
    lab, nc = O.components(beta_o)
    b = O.remove_mean(rhs, lab, nc)
    assert np.linalg.norm(O.residual(beta_o, b, pg, case.h)) / np.linalg.norm(b) <= 1.0001e-10
    assert rel(pg, p_o) <= 1e-9
    assert st.rel_resid <= 0.4e-10
    _, it_o, _ = mg.pcg(rhs, tol=0.4e-10, vcycles=vcycles)
    assert abs(st.cycles - it_o) <= 1, (st.cycles, it_o)


def test_pcg_projection_and_adjoint(mgp):
    case = SMALL["c2_64"]
    beta_g, ctx = _ctx(mgp, case, prec="mixed", krylov=1, inner_cycles=2)
    uo, po, beta_o, rhs = O.project(case.phi, case.solid, case.u_star, case.h, lam=case.lam, tol=1e-12)
    ug, pg, st = ctx.project(faces_dev(case.u_star), tol=1e-10)
    scale = max(np.abs(x).max() for x in uo)
    for a, b in zip(faces_host(ug), uo):
        assert np.abs(a - b).max() <= 1e-8 * scale
    gu_o, gb_o, _ = O.project_adjoint(beta_o, po, case.w, case.h, lam=case.lam, tol=1e-12)
    gu_g, gb_g, st = ctx.project_adjoint(faces_dev(case.w), dev(po), tol=1e-12)
    for a, b in zip(faces_host(gu_g), gu_o):
        assert np.abs(a - b).max() <= 1e-8 * max(np.abs(b).max(), 1.0)


TAIL_CASES = {
    "c2_64": lambda: synth.case_c2(64),
    "ragged_160x32x32": lambda: synth.small_case(160, 32, 32, solid="ellipsoid", seed=41),
    "aniso_64x32x16": lambda: synth.small_case(64, 32, 16, solid="ellipsoid", seed=43),
    "c3_256": lambda: synth.case_c3(256),
}


@pytest.mark.parametrize("name", list(TAIL_CASES))
def test_coarse_tail_identical_to_launches(mgp, name):
    """Running the smallest levels in one CTA (two launches around the coarsest solve) gives the
    same V-cycles (FP64) and the same mixed solves (FP32 cycles, stationary and CG) bit for bit as
    a launch per pass, with and without the coarse-grid graph."""
    case = TAIL_CASES[name]()
    beta = mgp.face_coeffs(dev(case.phi), case.h, None if case.solid is None else dev(case.solid, dtype=torch.uint8),
                           rho_air=case.lam)
    rhs = mgp.Context(beta, case.h).divergence(faces_dev(case.u_star))
    p = {}
    for tail in (0, 1):
        ctx = mgp.Context(beta, case.h, coarse_tail=tail)
        q = torch.zeros_like(rhs)
        for _ in range(2):
            ctx.vcycle(rhs - rhs.mean(), q)
        p[tail] = q
    assert torch.equal(p[0], p[1])
    for kw in ({"krylov": 0}, {"krylov": 1, "inner_cycles": 2}, {"krylov": 1, "coarse_graph": 0}):
        res = []
        for tail in (0, 1):
            ctx = mgp.Context(beta, case.h, prec="mixed", coarse_tail=tail, **kw)
            q, st = ctx.solve(rhs, tol=1e-10)
            res.append((q, st.cycles))
        assert res[0][1] == res[1][1] and torch.equal(res[0][0], res[1][0]), kw


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_coarse_graph_identical_to_launches(mgp, prec):
    """Replaying the coarse-grid correction as a CUDA graph changes nothing."""
    case = SMALL["c2_64"]
    beta = mgp.face_coeffs(dev(case.phi), case.h, dev(case.solid, dtype=torch.uint8), rho_air=case.lam)
    rhs = mgp.Context(beta, case.h).divergence(faces_dev(case.u_star))
    out = []
    for g in (0, 1):
        ctx = mgp.Context(beta, case.h, prec=prec, coarse_graph=g, krylov=1, inner_cycles=2)
        p, st = ctx.solve(rhs, tol=1e-10)
        p2, st2 = ctx.solve(rhs, torch.zeros_like(rhs), tol=1e-10)  # the graph is replayed
        assert torch.equal(p, p2)
        out.append((p, st.cycles))
    assert out[0][1] == out[1][1] and torch.equal(out[0][0], out[1][0])


@pytest.mark.parametrize("name", ["c1", "c2_64"])
def test_jacobi_pcg_matches_oracle(mgp, name):
    """Diagonally preconditioned CG (the comparison solver of the Poisson-solver section): the
    oracle's iteration count within 3 at the same target (the library's CG stops at 0.4 tol), and
    its solution to 1e-9."""
    case = SMALL[name]
    beta_g, ctx = _ctx(mgp, case, krylov=1, precond=1, max_cycles=100000)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    rhs = case_rhs(case, beta_o)
    p_o, it_o = O.cg_solve(beta_o, rhs, case.h, tol=0.4e-10, max_it=100000)
    p_ref, _, _ = O.MG(beta_o, case.h, max_coarse=4096).solve(rhs, tol=1e-12, max_cycles=300)
    p_g, st = ctx.solve(dev(rhs), tol=1e-10)
    assert it_o > 0 and abs(st.cycles - it_o) <= 3, (st.cycles, it_o)
    assert rel(host(p_g), p_ref) <= 1e-9


def test_jacobi_pcg_grows_with_n_multigrid_does_not(mgp):
    """The scaling the Poisson-solver section reports: on one geometry at 32^3 and 64^3, the
    diagonally preconditioned CG needs about twice the iterations at twice the resolution, the
    multigrid-preconditioned CG about the same number."""
    its = {}
    for n in (32, 64):
        case = synth.case_c2(n)
        beta = mgp.face_coeffs(dev(case.phi), case.h, dev(case.solid, dtype=torch.uint8), rho_air=case.lam)
        rhs = mgp.Context(beta, case.h).divergence(faces_dev(case.u_star))
        for method, kw in (("jacobi", dict(precond=1, max_cycles=100000)), ("mg", dict(inner_cycles=1))):
            ctx = mgp.Context(beta, case.h, krylov=1, **kw)
            _, st = ctx.solve(rhs, tol=1e-10)
            its[method, n] = st.cycles
    assert its["jacobi", 64] >= 1.5 * its["jacobi", 32], its
    assert abs(its["mg", 64] - its["mg", 32]) <= 2, its
    assert its["jacobi", 32] > 3 * its["mg", 32], its


def test_phi_grad_wide_rows_bit_exact(mgp):
    """The phi chain rule on rows longer than one block (520 cells) and on random grad_beta:
    bit-exact, the block-edge products included."""
    case = _adjoint_case(WIDE)
    beta_g, _ = _ctx(mgp, case)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    gb = tuple(np.random.default_rng(6).standard_normal(case.shape) for _ in range(3))
    gphi_g = host(mgp.phi_grad(beta_g, faces_dev(gb), case.h, rho_air=case.lam))
    assert np.array_equal(gphi_g, O.phi_grad(beta_o, gb, case.lam))
