"""Full-size workloads on the GPU, in the launch configuration bench.py times.

At these sizes the oracle checks properties that hold at any size (its own FP64
residual of the GPU solution, divergence of the projected velocity, the dot-product
test between forward and adjoint), compares the full 256^3 solution with its own
solve, and checks finite differences on a 32^3 crop.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1410_2240_gb300 import synth

from _gpu_util import dev, faces_dev, faces_host, host, rel

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def mgp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_2240_gb300 import mgproj
    return mgproj


def _beta(mgp, case):
    solid = None if case.solid is None else dev(case.solid, torch.uint8)
    return mgp.face_coeffs(dev(case.phi), case.h, solid, rho_air=case.lam)


def _rel_resid_oracle(beta_o, rhs, p, h):
    lab, nc = O.components(beta_o)
    b = O.remove_mean(rhs, lab, nc)
    return np.linalg.norm(O.residual(beta_o, b, p, h)) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def c3():
    case = synth.case_c3(256)
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    rhs = O.divergence(beta_o, case.u_star, case.h)
    mg = O.MG(beta_o, case.h)
    p_o, cyc, hist = mg.solve(rhs, tol=1e-12, max_cycles=200)
    # stationary V(2,2) cycles the oracle needs to reach 1e-10 (its history from p = 0)
    cyc10 = int(np.argmax(hist <= 1e-10)) + 1
    return case, beta_o, rhs, p_o, mg, cyc10


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_c3_256_solve(mgp, c3, prec):
    """Stationary cycles (FP64 V-cycles, or one FP32 V-cycle per FP64 refinement step): residual and
    solution against the oracle, and the oracle's cycle count to 1e-10 within one -- an FP32 cycle
    that smoothed worse than the FP64 one would need more refinement steps."""
    case, beta_o, rhs, p_o, mg, cyc10 = c3
    ctx = mgp.Context(_beta(mgp, case), case.h, prec=prec)
    p, st = ctx.solve(dev(rhs), tol=1e-10)
    pg = host(p)
    assert _rel_resid_oracle(beta_o, rhs, pg, case.h) <= 1.0001e-10
    assert rel(pg, p_o) <= 1e-9
    assert abs(st.cycles - cyc10) <= 1, (st.cycles, cyc10)


# The solver options bench.py times and autograd.project uses: CG preconditioned by two FP32
# V-cycles (mixed) or one FP64 V-cycle (FP64); the CG stops at 0.4 tol.
BENCH_CONFIGS = {"mixed": dict(prec="mixed", krylov=1, inner_cycles=2),
                 "fp64": dict(prec="fp64", krylov=1, inner_cycles=1)}


@pytest.mark.parametrize("name", list(BENCH_CONFIGS))
def test_c3_256_bench_configuration(mgp, c3, name):
    """The benchmark's 256^3 projection and adjoint with the benchmark's solver options: the
    forward solve's residual <= 1e-10 by the oracle's operator and its p within 1e-9 of the
    oracle's solve continued to 1e-12; the CG iteration count within one of the oracle's own CG
    with as many FP64 V-cycles per preconditioner application, stopped at the same 0.4 tol; the
    projected velocity and the adjoint's gradient to u* against the oracle's."""
    case, beta_o, rhs, p_o, mg, _ = c3
    kw = BENCH_CONFIGS[name]
    ctx = mgp.Context(_beta(mgp, case), case.h, **kw)
    u_star = faces_dev(case.u_star)
    for _ in range(2):  # the second call replays the captured coarse-grid graph
        p = torch.zeros(case.shape, dtype=torch.float64, device="cuda")
        u, p, st = ctx.project(u_star, p=p, tol=1e-10)
    pg = host(p)
    assert st.rel_resid <= 0.4e-10
    assert _rel_resid_oracle(beta_o, rhs, pg, case.h) <= 0.4001e-10
    assert rel(pg, p_o) <= 1e-9, rel(pg, p_o)
    _, it_o, _ = mg.pcg(rhs, tol=0.4e-10, vcycles=kw["inner_cycles"])
    assert it_o > 0 and abs(st.cycles - it_o) <= 1, (st.cycles, it_o)
    uo = O.correct(beta_o, p_o, case.u_star, case.h)
    scale = max(np.abs(x).max() for x in uo)
    for a, b in zip(faces_host(u), uo):
        assert np.abs(a - b).max() <= 1e-8 * scale
    gu, _, st2 = ctx.project_adjoint(faces_dev(case.w), p, tol=1e-10, q=torch.zeros_like(p))
    assert st2.rel_resid <= 0.4e-10
    gu_o, _, _ = O.project_adjoint(beta_o, p_o, case.w, case.h, lam=case.lam, tol=1e-12)
    for a, b in zip(faces_host(gu), gu_o):
        # the adjoint's q within ~1e-9 of the oracle's; its face gradient differences the error
        assert np.abs(a - b).max() <= 1e-7 * max(np.abs(b).max(), 1.0)


def test_c3_256_projection_divergence_free(mgp, c3):
    case, beta_o, rhs, p_o, _, _ = c3
    ctx = mgp.Context(_beta(mgp, case), case.h, prec="mixed")
    u, p, st = ctx.project(faces_dev(case.u_star), tol=1e-10)
    du = O.divergence(beta_o, faces_host(u), case.h)
    assert np.linalg.norm(du) <= 1.0001e-10 * np.linalg.norm(rhs)


def test_c4_forward_backward_dot_product(mgp):
    """512x256x128 with 200 bubbles: <P a, b> = <a, P^T b> through the GPU forward and adjoint."""
    case = synth.case_c4()
    beta = _beta(mgp, case)
    ctx = mgp.Context(beta, case.h)
    a = faces_dev(case.u_star)
    bw = faces_dev(case.w)
    Pa, p, st = ctx.project(a, tol=1e-12)
    gu, gb, st2 = ctx.project_adjoint(bw, p, tol=1e-12)
    lhs = sum(float((x * y).sum()) for x, y in zip(Pa, bw))
    rhs = sum(float((x * y).sum()) for x, y in zip(a, gu))
    assert abs(lhs - rhs) <= 1e-9 * (abs(lhs) + abs(rhs))
    beta_o = O.face_coeffs(case.phi, None, case.lam)
    du = O.divergence(beta_o, faces_host(Pa), case.h)
    b0 = O.divergence(beta_o, case.u_star, case.h)
    assert np.linalg.norm(du) <= 1.0001e-12 * np.linalg.norm(b0)


def test_c4_crop_phi_gradient_finite_differences(mgp):
    """FP64 central differences (Richardson) of L = sum(w u) on a 32^3 crop around the bubble
    nearest the surface, and the FP64 CPU reference gradient on the same crop."""
    from paper_1410_2240_gb300.autograd import project
    full = synth.case_c4()
    c, r = min(full.bubbles, key=lambda br: 0.5 - br[0][2])
    ijk = [int(c[d] / full.h) for d in range(3)]
    case = synth.crop(full, ijk, 32)
    phi = dev(case.phi).requires_grad_(True)
    u = tuple(x.requires_grad_(True) for x in faces_dev(case.u_star))
    w = faces_dev(case.w)
    (ux, uy, uz), p = project(u, phi, case.h, rho_air=case.lam, tol=1e-12)
    torch.autograd.backward((ux, uy, uz), w)
    g = host(phi.grad)

    def loss(ph):
        with torch.no_grad():
            (a, b, cc), _ = project(faces_dev(case.u_star), dev(ph), case.h, rho_air=case.lam, tol=1e-12)
            return float((a * w[0]).sum() + (b * w[1]).sum() + (cc * w[2]).sum())

    band = np.argwhere((case.phi > 0.05) & (case.phi < 0.95))
    rng = np.random.default_rng(4)
    picks = band[rng.choice(len(band), size=min(20, len(band)), replace=False)]
    for k, j, i in picks:
        def cd(eps):
            pp = case.phi.copy(); pp[k, j, i] += eps
            pm = case.phi.copy(); pm[k, j, i] -= eps
            return (loss(pp) - loss(pm)) / (2 * eps)
        fd = (4 * cd(5e-4) - cd(1e-3)) / 3
        assert abs(fd - g[k, j, i]) <= 1e-6 * max(abs(fd), 1e-6 * np.abs(g).max()), (k, j, i, fd, g[k, j, i])
    # FP64 CPU reference gradient
    uo, po, beta_o, _ = O.project(case.phi, None, case.u_star, case.h, lam=case.lam, tol=1e-13)
    _, _, gphi_o = O.project_adjoint(beta_o, po, case.w, case.h, lam=case.lam, tol=1e-13)
    assert rel(g, gphi_o) <= 1e-8
    for x, gx in zip(u, O.project_adjoint(beta_o, po, case.w, case.h, lam=case.lam, tol=1e-13)[0]):
        assert rel(host(x.grad), gx) <= 1e-8


def test_c5_plunging_mixed_forward_backward(mgp):
    """1024x512x256 (134M cells), overturned interface + hull: mixed forward to 1e-10 and backward."""
    case = synth.case_c5()
    assert synth.overturned_columns(case.phi) >= 1
    beta = _beta(mgp, case)
    ctx = mgp.Context(beta, case.h, prec="mixed")
    u_star = tuple(torch.from_numpy(x).to("cuda", torch.float64) for x in case.u_star)
    u, p, st = ctx.project(u_star, tol=1e-10)
    assert st.rel_resid <= 1e-10
    w = tuple(torch.from_numpy(x).to("cuda", torch.float64) for x in case.w)
    gu, gb, st2 = ctx.project_adjoint(w, p, tol=1e-10)
    assert st2.rel_resid <= 1e-10
    gphi = mgp.phi_grad(beta, gb, case.h, rho_air=case.lam)
    assert torch.isfinite(gphi).all()
    # the oracle's FP64 residual of the GPU solution and divergence of u
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    rhs = O.divergence(beta_o, case.u_star, case.h)
    assert _rel_resid_oracle(beta_o, rhs, host(p), case.h) <= 1.0001e-10
    du = O.divergence(beta_o, faces_host(u), case.h)
    assert np.linalg.norm(du) <= 1.0001e-10 * np.linalg.norm(rhs)
