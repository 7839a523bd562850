"""The bounds-check build (-DMGP_CHECK) on the GPU: every kernel of the solver paths runs with its
index checks on, no index falls outside the array it indexes, and the results are those of the
normal build.

The check build is loaded in a child process (MGPROJ_LIB), which runs the workloads below and
prints the norms of its results and the check record as JSON; the parent runs the same workloads
with the normal build.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# one function per workload, run in both processes; each returns a dict of result norms
WORKLOADS = r'''
import numpy as np
import torch
from paper_1410_2240_gb300 import mgproj, synth

def dev(a, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)

def faces(fs):
    return tuple(dev(f) for f in fs)

def norm(t):
    return float(torch.linalg.vector_norm(t.double()))

def run_all():
    out = {}
    cases = {"c2_64": synth.case_c2(64), "ragged_36x32x32": synth.small_case(36, 32, 32, seed=3, solid="ellipsoid"),
             "wall_pockets_32": synth.small_case(32, seed=4, solid="wall")}
    for name, case in cases.items():
        solid = None if case.solid is None else dev(case.solid, torch.uint8)
        beta = mgproj.face_coeffs(dev(case.phi), case.h, solid, rho_air=case.lam)
        for tag, kw in (("fp64", dict()), ("mixed_cg", dict(prec="mixed", krylov=1, inner_cycles=2)),
                        ("mixed", dict(prec="mixed")), ("fp64_cg", dict(krylov=1)), ("tail0", dict(coarse_tail=0))):
            ctx = mgproj.Context(beta, case.h, coarse_max_cells=2048, **kw)
            u, p, st = ctx.project(faces(case.u_star), tol=1e-10)
            gu, gb, st2 = ctx.project_adjoint(faces(case.w), p, tol=1e-10)
            gphi = mgproj.phi_grad(beta, gb, case.h, rho_air=case.lam)
            out[f"{name}/{tag}"] = [norm(p), sum(norm(x) for x in u), sum(norm(x) for x in gu), norm(gphi),
                                    st.cycles, st2.cycles]
            q = torch.zeros_like(p)
            ctx.vcycle(ctx.divergence(faces(case.u_star)), q)
            out[f"{name}/{tag}/vcycle"] = [norm(q)]
        f = mgproj.forces(g=1.0, inv_re=0.01, convection=True)
        ctx = mgproj.Context(beta, case.h, prec="mixed", krylov=1, inner_cycles=2, coarse_max_cells=2048)
        u = list(faces(case.u_star))
        phi1, P, st = ctx.rk2_step(dev(case.phi), u, 0.2 * case.h, solid=solid, rho_air=case.lam, tol=1e-10, forces=f)
        out[f"{name}/rk2"] = [norm(phi1), norm(P), sum(norm(x) for x in u)]
    # a z-stretched grid (banded-row records) with face areas
    n = 32
    case = synth.small_case(n, seed=7, solid="ellipsoid", interface="flat")
    hz = synth.stretched_widths(n, 3.5, 0.5)
    beta = mgproj.face_coeffs(dev(case.phi), case.h, dev(case.solid, torch.uint8), rho_air=case.lam)
    bo, ao = mgproj.stretched_metrics(dev(np.full(n, case.h)), dev(np.full(n, case.h)), dev(hz), beta)
    ctx = mgproj.Context(bo, 1.0, prec="mixed", coarse_max_cells=2048)
    ctx.set_face_areas(ao)
    u, p, st = ctx.project(faces(case.u_star), tol=1e-10)
    out["stretched"] = [norm(p), st.cycles]
    # the benchmark's workload at 128^3
    case = synth.case_c2(128)
    beta = mgproj.face_coeffs(dev(case.phi), case.h, dev(case.solid, torch.uint8), rho_air=case.lam)
    ctx = mgproj.Context(beta, case.h, prec="mixed", krylov=1, inner_cycles=2)
    u, p, st = ctx.project(faces(case.u_star), tol=1e-10)
    out["c2_128"] = [norm(p), st.cycles]
    torch.cuda.synchronize()
    return out
'''

CHILD = WORKLOADS + r'''
import json, sys
res = run_all()
enabled, first, count = mgproj.check_read()
print(json.dumps({"enabled": enabled, "first": first, "count": count, "results": res}))
'''


def test_check_build_runs_clean_and_matches_normal_build(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_2240_gb300.build import build
    lib = build(check=True)
    script = tmp_path / "child.py"
    script.write_text(CHILD)
    env = dict(os.environ, MGPROJ_LIB=lib, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, str(script)], env=env, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    child = json.loads(r.stdout.strip().splitlines()[-1])
    assert child["enabled"] is True
    assert child["count"] == 0 and child["first"] == 0, child
    ns = {}
    exec(compile(WORKLOADS, "<workloads>", "exec"), ns)
    normal = ns["run_all"]()
    from paper_1410_2240_gb300 import mgproj
    assert mgproj.check_read() == (False, 0, 0)
    assert set(normal) == set(child["results"])
    for key, vals in normal.items():
        other = child["results"][key]
        for a, b in zip(vals, other):
            assert abs(a - b) <= 1e-12 * max(abs(a), 1e-300), (key, vals, other)
