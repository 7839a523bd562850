"""Pins are strong enough: each planted mistake in a copy of the oracle's C source is caught.

The mistake is planted in a temporary copy of oracle/mg_oracle.c compiled on the CPU;
the pins of test_oracle_operator / test_oracle_solver then run against that copy and
at least one of them must fail.  The real oracle is restored afterwards.
"""
import inspect
import os
import subprocess
import tempfile

import pytest

import oracle as O
import test_oracle_areas as T3
import test_oracle_momentum as T6
import test_oracle_rk2 as T5
import test_oracle_stretched as T4
import test_oracle_operator as T1
import test_oracle_solver as T2

SRC = os.path.join(os.path.dirname(O.__file__), "mg_oracle.c")

# (name, original text, mutated text, pins that must catch it)
MUTANTS = [
    ("face harmonic mean -> arithmetic", "return 2.0 / (rhoL + rhoR);", "return 0.5 * (1.0 / rhoL + 1.0 / rhoR);",
     [T1.test_face_coeffs_golden_pairs, T1.test_face_coeffs_is_harmonic_mean_of_inverse_density]),
    ("density model lam <-> 1-lam", "double rhoL = lam + (1.0 - lam) * phiL;", "double rhoL = (1.0 - lam) + lam * phiL;",
     [T1.test_face_coeffs_golden_pairs]),
    ("operator drops the z+ term", "if (k < nz - 1) s += bz[IX(i, j, k + 1)] * (p[IX(i, j, k + 1)] - p[c]);", "",
     [T1.test_stencil_golden_3x3x3, T1.test_constant_coefficient_operator_is_neumann_laplacian]),
    ("operator uses the low y face twice", "if (j < ny - 1) s += by[IX(i, j + 1, k)] * (p[IX(i, j + 1, k)] - p[c]);",
     "if (j < ny - 1) s += by[c] * (p[IX(i, j + 1, k)] - p[c]);",
     [lambda: T1.test_operator_invariants("ellipsoid"), T1.test_dense_operator_matches_independent_assembly]),
    ("smoother sign of the source", "p[c] = dinv[c] * fma(-h2, b[c], s);", "p[c] = dinv[c] * fma(h2, b[c], s);",
     [lambda: T1.test_colour_sweep_zeroes_that_colours_residual(0)]),
    ("smoother reads the wrong x neighbour", "if (i < nx - 1) s = fma(bx[IX(i + 1, j, k)], p[IX(i + 1, j, k)], s);",
     "if (i < nx - 1) s = fma(bx[IX(i + 1, j, k)], p[IX(i, j, k)], s);",
     [lambda: T1.test_colour_sweep_zeroes_that_colours_residual(1)]),
    ("residual drops the y- flux", "if (j > 0) s = fma(by[c], p[IX(i, j - 1, k)] - p[c], s);", "",
     [lambda: T1.test_colour_sweep_zeroes_that_colours_residual(0)]),
    ("coefficient restriction scale", "cbx[C] = 0.25 * (", "cbx[C] = 0.5 * (",
     [T1.test_coefficient_restriction_invariants]),
    ("coefficient restriction takes the odd fine plane", "cbz[C] = 0.25 * (bz[IX(2 * I, 2 * J, 2 * K)] + bz[IX(2 * I + 1, 2 * J, 2 * K)] +",
     "cbz[C] = 0.25 * (bz[IX(2 * I, 2 * J, 2 * K + 1)] + bz[IX(2 * I + 1, 2 * J, 2 * K)] +",
     [T1.test_coefficient_restriction_invariants]),
    ("restriction weight", "rc[((size_t)K * NY + J) * NX + I] = 0.125 * s;", "rc[((size_t)K * NY + J) * NX + I] = 0.25 * s;",
     [T1.test_restriction_is_child_average]),
    ("prolongation weights swapped", "double w[2] = {0.75, 0.25};", "double w[2] = {0.25, 0.75};",
     [T1.test_prolongation_reproduces_linear_fields_and_constants]),
    ("prolongation neighbour on the wrong side", "int I1 = (i & 1) ? I0 + 1 : I0 - 1;", "int I1 = (i & 1) ? I0 - 1 : I0 + 1;",
     [T1.test_prolongation_reproduces_linear_fields_and_constants]),
    ("divergence sign of the z flux", "if (bz[c] > 0.0) d -= uz[c];", "if (bz[c] > 0.0) d += uz[c];",
     [T2.test_projection_is_divergence_free_and_idempotent]),
    ("correction uses the wrong neighbour", "if (by[c] > 0.0) uy[c] = uy0[c] - dt * by[c] * (p[c] - p[IX(i, j - 1, k)]) / h;",
     "if (by[c] > 0.0) uy[c] = uy0[c] - dt * by[c] * (p[c] - p[IX(i - 1, j, k)]) / h;",
     [T2.test_projection_is_divergence_free_and_idempotent]),
    ("phi gradient sign", "gphi[c] = -0.5 * (1.0 - lam) * s;", "gphi[c] = 0.5 * (1.0 - lam) * s;",
     [T2.test_adjoint_phi_gradient_central_differences]),
    ("phi gradient drops the high x face", "if (i < nx - 1) s += bx[IX(i + 1, j, k)] * bx[IX(i + 1, j, k)] * gbx[IX(i + 1, j, k)];", "",
     [T2.test_adjoint_phi_gradient_central_differences]),
    ("pseudo-inverse keeps the null space", "if (fabs(lam) <= 1e-9 * lmax) continue;", "if (fabs(lam) == 0.0) continue;",
     [T1.test_pinv_matches_numpy_and_penrose_conditions]),
    ("PCG drops the flexible correction of beta", "double beta = (rzn - dot(n, r, zo)) / rz;", "double beta = (rzn + dot(n, r, zo)) / rz;",
     [lambda: T2.test_pcg_and_stationary_cycles_agree("c1")]),
    ("PCG residual update sign", "p[c] += alpha * d[c]; r[c] -= alpha * q[c];", "p[c] += alpha * d[c]; r[c] += alpha * q[c];",
     [lambda: T2.test_pcg_matches_dense_pseudoinverse(1)]),
    ("component search ignores upper z faces", "if (k < nz - 1) { nb[m] = IX(i, j, k + 1); fb[m++] = bz[IX(i, j, k + 1)]; }", "",
     [T1.test_components_counts]),
    ("triangle open fraction not squared", "return (f * f) / ((f - g1) * (f - g2));", "return f / ((f - g1) * (f - g2));",
     [T3.test_face_open_closed_forms, T3.test_face_open_matches_brute_force]),
    ("x-face area takes a corner of the next x plane",
     "ax[c] = i == 0 ? 0.0 : orc_face_open(PSI(i, j, k), PSI(i, j + 1, k), PSI(i, j, k + 1), PSI(i, j + 1, k + 1));",
     "ax[c] = i == 0 ? 0.0 : orc_face_open(PSI(i, j, k), PSI(i, j + 1, k), PSI(i + 1, j, k + 1), PSI(i, j + 1, k + 1));",
     [T3.test_plane_areas_exact, T3.test_sphere_cross_sections]),
    ("area divergence drops the area of the low x face", "if (ax[c] > 0.0) d -= FLUX(ax, ux, vx, c);",
     "if (ax[c] > 0.0) d -= ux[c];", [T3.test_area_divergence_composes_with_plain_divergence]),
    ("area divergence ignores the body velocity",
     "#define FLUX(arr_a, arr_u, arr_v, idx) ((arr_a)[idx] * ((arr_u)[idx] - ((arr_v) ? (arr_v)[idx] : 0.0)))",
     "#define FLUX(arr_a, arr_u, arr_v, idx) ((arr_a)[idx] * (arr_u)[idx])",
     [T3.test_area_divergence_composes_with_plain_divergence]),
    ("stretched z distance is one width", "double d = 0.5 * (hz[k - 1] + hz[k]);", "double d = hz[k];",
     [T4.test_linear_pressure_face_gradients_exact, T4.test_layered_problem_matches_1d_finite_volumes]),
    ("stretched z-face area from the wrong widths", "az[c] = (hx[i] * hy[j]) * (fz ? fz[c] : 1.0);",
     "az[c] = (hx[i] * hz[k]) * (fz ? fz[c] : 1.0);", [T4.test_linear_pressure_face_gradients_exact]),
    ("VOF takes the downwind cell", "#define UPW(u, lo, hi) ((u) > 0.0 ? (u) * phi[lo] : (u) * phi[hi])",
     "#define UPW(u, lo, hi) ((u) > 0.0 ? (u) * phi[hi] : (u) * phi[lo])", [T5.test_vof_upwind_hand_example]),
    ("normal viscous stress without its factor 2", "const double tp = 2.0 * mup * ((up - u0) * ih);",
     "const double tp = mup * ((up - u0) * ih);", [lambda: T6.test_viscous_term_exact_for_quadratic_velocity(False)]),
    ("edge viscosity from two cells", "a < b ? 0.25 * (((m00 + m10) + m01) + m11)", "a < b ? 0.5 * (m01 + m11)",
     [lambda: T6.test_viscous_term_exact_for_quadratic_velocity(True)]),
    ("normal momentum flux sign", "conv = (cp * cp - cm * cm) * ih;", "conv = (cp * cp + cm * cm) * ih;",
     [T6.test_convective_term_exact_for_linear_velocity]),
    ("shear takes the wrong tangential face", "const double ub0 = fvel(U[b], b, si - ea[0], sj - ea[1], sk - ea[2], nx, ny, nz);",
     "const double ub0 = fvel(U[b], b, si - eb[0], sj - eb[1], sk - eb[2], nx, ny, nz);",
     [T6.test_convective_term_exact_for_linear_velocity, lambda: T6.test_viscous_term_exact_for_quadratic_velocity(False)]),
    ("viscous term without 1/rho", "r = r + (inv_re * B[a][c]) * (visc * ih);", "r = r + inv_re * (visc * ih);",
     [lambda: T6.test_viscous_term_exact_for_quadratic_velocity(False)]),
    ("walls hold zero ghosts instead of mirrored tangential velocity",
     "    i = clampi(i, 0, nx - 1);\n    j = clampi(j, 0, ny - 1);\n    k = clampi(k, 0, nz - 1);\n    return u[IX(i, j, k)];",
     "    if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return 0.0;\n    return u[IX(i, j, k)];",
     [T6.test_free_slip_walls_shear_closed_form]),
    ("momentum gravity points up", "if (a == 2) r = r - g;", "if (a == 2) r = r + g;",
     [T5.test_rk2_hydrostatic_column_stays_at_rest]),
    ("momentum flux at the high edge from the low rows",
     "const double ua1 = fvel(U[a], a, si, sj, sk, nx, ny, nz);",
     "const double ua1 = fvel(U[a], a, si - eb[0], sj - eb[1], sk - eb[2], nx, ny, nz);",
     [T6.test_free_slip_walls_flux_closed_form, T6.test_convective_term_exact_for_linear_velocity]),
]


def _compile(src_text, out):
    c = out + ".c"
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", out, c, "-lm"],
                   check=True)


@pytest.mark.parametrize("name,orig,mut,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, orig, mut, pins, tmp_path):
    src = open(SRC).read()
    assert src.count(orig) >= 1, f"mutation anchor not found: {orig}"
    lib = str(tmp_path / "mutant.so")
    _compile(src.replace(orig, mut, 1), lib)
    O.use_library(lib)
    try:
        caught = []
        for pin in pins:
            try:
                pin()
                caught.append(False)
            except (AssertionError, RuntimeError, ValueError, ZeroDivisionError, FloatingPointError):
                caught.append(True)
        assert any(caught), f"no pin caught the mutant '{name}'"
    finally:
        O.use_library(None)


# Mistakes planted in the oracle's Python steps (the time step of the Numerical Time Integration
# section, the fractional-area and stretched projections): (name, function, original text, mutated
# text, pins that must catch it)
PY_MUTANTS = [
    ("second stage drops the 1/2 of Eq. runge2", "rk2_step",
     "u1 = tuple(0.5 * x for x in correct(beta2, P, ut2, h, dt))", "u1 = tuple(correct(beta2, P, ut2, h, dt))",
     [T5.test_rk2_keeps_divergence_free_velocity_without_forces]),
    ("second stage leaves u^k out of Eq. poisson2", "rk2_step",
     "ut2 = tuple((a + b) + dt * r for a, b, r in zip(us, u, R2))", "ut2 = tuple(a + dt * r for a, r in zip(us, R2))",
     [T5.test_rk2_keeps_divergence_free_velocity_without_forces]),
    ("second stage's R from u^k instead of u*", "rk2_step",
     "R2 = momentum_rhs(phis, beta2, us, h, g, inv_re, mu_air, 1.0, convect)",
     "R2 = momentum_rhs(phis, beta2, u, h, g, inv_re, mu_air, 1.0, convect)", [T6.test_rk2_second_order_in_time]),
    ("second projection solved with the first stage's density", "rk2_step",
     "P = solve(beta2, divergence(beta2, ut2, h, dt), h, tol=tol)", "P = solve(beta, divergence(beta, ut2, h, dt), h, tol=tol)",
     [T5.test_rk2_returns_divergence_free_velocity]),
    ("projection rhs not divided by dt", "project", "rhs = divergence(beta, u_star, h, dt)",
     "rhs = divergence(beta, u_star, h, 1.0)", [T2.test_projection_is_divergence_free_and_idempotent]),
    ("adjoint rhs without beta", "project_adjoint", "bw = tuple(b * x for b, x in zip(beta, w))",
     "bw = tuple(x for b, x in zip(beta, w))", [T2.test_projection_dot_product_test]),
    ("adjoint grad_u* sign of G q", "project_adjoint", "np.where(b > 0, x - g, x)", "np.where(b > 0, x + g, x)",
     [T2.test_adjoint_u_gradient_is_exact_for_linear_loss]),
    ("adjoint grad_beta drops dt", "project_adjoint", "dt * a * (g - x)", "a * (g - x)",
     [T2.test_adjoint_phi_gradient_central_differences]),
    ("cut-cell operator without the area", "area_coeffs", "np.where(a > 0, a * b, 0.0)", "np.where(a > 0, b, 0.0)",
     [lambda: T3.test_projection_with_areas_is_divergence_free(False)]),
    ("cut-cell correction weighted by the area", "open_mask", "np.where(a > 0, b, 0.0)", "np.where(a > 0, a * b, 0.0)",
     [lambda: T3.test_projection_with_areas_is_divergence_free(False)]),
    ("adjoint grad_u* without the area", "project_adjoint_area", "np.where(a > 0, x - a * g, x)",
     "np.where(a > 0, x - g, x)", [T3.test_adjoint_with_areas_linearity_and_phi]),
    ("adjoint grad_beta without the area", "project_adjoint_area", "dt * gpp * (a * g - x)", "dt * gpp * (g - x)",
     [T3.test_adjoint_with_areas_linearity_and_phi]),
    ("stretched correction with the physical spacing", "project_stretched",
     "u = correct(open_mask(area, bi), p, u_star, 1.0, dt)", "u = correct(open_mask(area, bi), p, u_star, hz[0], dt)",
     [T4.test_uniform_widths_reproduce_uniform_projection, T4.test_stretched_projection_divergence_free]),
]


@pytest.mark.parametrize("name,fname,orig,mut,pins", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_planted_python_mistake_is_caught(name, fname, orig, mut, pins, monkeypatch):
    src = inspect.getsource(getattr(O, fname))
    assert src.count(orig) == 1, f"mutation anchor not found: {orig}"
    ns = dict(vars(O))
    exec(compile(src.replace(orig, mut, 1), f"<mutant {name}>", "exec"), ns)
    monkeypatch.setattr(O, fname, ns[fname])
    caught = []
    for pin in pins:
        try:
            pin()
            caught.append(False)
        except (AssertionError, RuntimeError, ValueError, ZeroDivisionError, FloatingPointError):
            caught.append(True)
    assert any(caught), f"no pin caught the mutant '{name}'"
