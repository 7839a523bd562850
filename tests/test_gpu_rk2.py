"""The Runge-Kutta time step on the GPU (mg_rk2_step) against the oracle's step: velocity,
volume fraction and pressure after one step with a body, gravity and (optionally) the viscous and
convective terms, FP64 and mixed; a hydrostatic column that stays at rest; the momentum
right-hand side (mg_momentum_rhs) bit for bit against the oracle's."""
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


MU_AIR = 1.8e-2


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["ell_32", "ragged_48x32x16"])
@pytest.mark.parametrize("full", [False, True])
def test_rk2_step_matches_oracle(mgp, prec, name, full):
    """One step; full: the viscous (1/Re = 0.01, mu ratio 0.018) and convective terms as well."""
    dims = {"ell_32": (32, 32, 32, 7), "ragged_48x32x16": (48, 32, 16, 8)}[name]
    case = synth.small_case(*dims[:3], seed=dims[3], solid="ellipsoid", interface="wave")
    dt, g = 0.2 * case.h, 1.0
    inv_re = 1e-2 if full else 0.0
    u_o, phi_o, P_o = O.rk2_step(case.phi, case.solid, case.u_star, case.h, dt, g, lam=case.lam, tol=1e-12,
                                 inv_re=inv_re, mu_air=MU_AIR, convect=full)
    beta = mgp.face_coeffs(dev(case.phi), case.h, dev(case.solid, torch.uint8), rho_air=case.lam)
    ctx = mgp.Context(beta, case.h, prec=prec, krylov=1, inner_cycles=2, coarse_max_cells=2048)
    u = list(faces_dev(case.u_star))
    f = mgp.forces(g=g, inv_re=inv_re, mu_air=MU_AIR, convection=full)
    phi1, P, st = ctx.rk2_step(dev(case.phi), u, dt, solid=dev(case.solid, torch.uint8), rho_air=case.lam,
                               tol=1e-11, forces=f)
    scale = max(np.abs(x).max() for x in u_o)
    for a, b in zip(faces_host(u), u_o):
        assert np.abs(a - b).max() <= 1e-7 * scale
    assert np.abs(host(phi1) - phi_o).max() <= 1e-9
    assert rel(host(P) - host(P).mean(), P_o - P_o.mean()) <= 1e-7


def test_rk2_hydrostatic_column_at_rest(mgp):
    case = synth.small_case(32, 32, 32, seed=1, solid="none", interface="flat")
    beta = mgp.face_coeffs(dev(case.phi), case.h, None, rho_air=case.lam)
    ctx = mgp.Context(beta, case.h, prec="mixed", krylov=1, inner_cycles=2, coarse_max_cells=2048)
    u = [torch.zeros(case.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    dt, g = 0.01, 1.0
    phi1, P, st = ctx.rk2_step(dev(case.phi), u, dt, g, rho_air=case.lam, tol=1e-11)
    assert max(float(x.abs().max()) for x in u) <= 1e-8 * dt * g
    assert float((phi1 - dev(case.phi)).abs().max()) <= 1e-8


MOM_CASES = {
    "ell_32_random_phi": lambda: synth.small_case(32, seed=11, solid="ellipsoid", interface="random"),
    "ragged_40x24x16_wave": lambda: synth.small_case(40, 24, 16, seed=12, solid="ellipsoid", interface="wave"),
    "wall_16": lambda: synth.small_case(16, seed=13, solid="wall", interface="wave"),
    "thin_1x6x5": lambda: synth.small_case(1, 6, 5, seed=14, solid="none", interface="random"),
}


@pytest.mark.parametrize("name", list(MOM_CASES))
@pytest.mark.parametrize("terms", ["all", "viscous", "convective"])
def test_momentum_rhs_bit_exact(mgp, name, terms):
    """R of Eq. navi on the GPU equals the oracle's bit for bit: the same separately rounded
    operations in the same order (walls, bodies, ragged and one-cell-wide grids)."""
    case = MOM_CASES[name]()
    beta_o = O.face_coeffs(case.phi, case.solid, case.lam)
    inv_re = 0.0 if terms == "convective" else 0.37
    conv = terms != "viscous"
    R_o = O.momentum_rhs(case.phi, beta_o, case.u_star, case.h, g=1.3, inv_re=inv_re, mu_air=MU_AIR, convect=conv)
    f = mgp.forces(g=1.3, inv_re=inv_re, mu_air=MU_AIR, convection=conv)
    R_g = mgp.momentum_rhs(dev(case.phi), faces_dev(beta_o), faces_dev(case.u_star), case.h, f)
    for a, b in zip(faces_host(R_g), R_o):
        assert np.array_equal(a, b)
