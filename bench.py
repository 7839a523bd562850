#!/usr/bin/env python
"""Benchmark of the GB300 variable-density pressure projection.

Metric: Poisson solves/s to relative residual 1e-10 at 256^3 (mixed FP32-in-FP64
refinement), with the plain FP64 solve and the V-cycle HBM GB/s of both reported
beside it.  One timed step is one pass of the whole hot path over the 256^3 case
(unit cube, 4-mode free surface of amplitude 0.08, a piercing ellipsoid, density
ratio 1e-3, u* ~ N(0, 0.1), loss weights w ~ N(0, 1)):

    face coefficients from phi -> multigrid hierarchy (mg_update) ->
    projection (divergence, solve to 1e-10, correction) ->
    adjoint projection (second solve) -> chain rule to phi

i.e. two Poisson solves per step.  Inputs are resident in HBM when the timed region
starts; the ``e2e`` leg repeats the step through the public API with pinned host
buffers, host<->device copies included.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run, one rank per GPU) every rank runs an
independent replica of the workload (the projection is a single-GPU problem here):
"scaling": "weak", value = all ranks' solves / max-over-ranks time.
``--impl reference`` times the CPU FP64 oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import gc
import json
import resource
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Poisson solves/s to 1e-10 resid at 256^3; V-cycle HBM GB/s, FP64 vs mixed"
TOL = 1e-10
# algorithmic bytes per fine cell (each array read or written once per pass)
# one red-black sweep, FP32: p, b, bx, by, bz, dinv read + p written.  The finest-grid kernel forms
# 1/diag from the faces it loads and takes the faces of uniform rows from one value per row, so
# its DRAM traffic (the roofline's `traffic`) is below these algorithmic bytes
B_SWEEP32 = 28.0
B_SWEEP64 = 56.0
B_VCYCLE32 = 161.0    # V(2,2), all levels, FP32: (4 sweeps x 28 + residual/restriction 20.5 + prolongation 8.5) x 8/7
B_VCYCLE64 = 322.0    # V(2,2), all levels, FP64
B_RESID64 = 48.0      # FP64 residual + norm (p, b, bx, by, bz read; dinv mask)
B_REFINE = 44.0 + 20.0  # FP64 residual + FP32 cast, then p64 += s*e32
B_CG_ITER = 48.0 + 52.0 + 20.0 + 12.0  # one CG iteration's vectors: q = A d, p/r/r32 update, direction, dots


def iteration_bytes(inner, vcycle_bytes, krylov, resid_bytes):
    """Algorithmic bytes per finest cell of one outer iteration: `inner` V-cycles plus the CG vector
    work (krylov) or the refinement step's residual and accumulation."""
    return inner * vcycle_bytes + (B_CG_ITER if krylov else resid_bytes)
SWEEP_KERNEL = {0: "k_smooth_split4 x2 colour passes, colour-split p, b and faces, uniform-row records",
                1: "k_smooth_split4 x2 colour passes, colour-split p, b and faces, uniform-row records",
                2: "k_rb_sweep<float,32,8> fused", 3: "k_rb_sweep_tma fused, TMA-staged planes"}
# DRAM bytes of one finest-grid FP32 sweep of the default smoother (two k_smooth_split4 colour
# passes) from an ncu capture of this workload
SWEEP_TRAFFIC_256 = 119.288064e6 + 11.910400e6 + 119.242240e6 + 13.071104e6
PROF_GROUPS = (("smooth", 0), ("restrict", 1), ("prolong", 2), ("resid64", 3), ("cg_apply", 4), ("cg_vectors", 5),
               ("coarse_levels", 6), ("hierarchy_update", 7))


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=256, help="grid size per axis of the c3 workload (256 = the benchmark)")
    ap.add_argument("--workload", choices=["c3", "c4", "c5"], default="c3",
                    help="c3: 256^3 ellipsoid case (the metric's); c4: 512x256x128 tank with 200 bubbles; "
                         "c5: 1024x512x256 plunging wave + hull")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--pcg-scaling", action="store_true",
                    help="instead of the benchmark: iterations and solve time of Jacobi-preconditioned CG and of "
                         "multigrid (stationary, and preconditioning CG) on one geometry at 64^3, 128^3, 256^3")
    ap.add_argument("--oracle-timing", action="store_true",
                    help="instead of the benchmark: the CPU oracle's full solve to 1e-10 on the 32^3, 128^3 and "
                         "256^3 workloads, on all host cores and on one (a child process each)")
    ap.add_argument("--oracle-solve", default=None, help=argparse.SUPPRESS)  # child of --oracle-timing
    ap.add_argument("--rk2", action="store_true",
                    help="instead of the benchmark: Runge-Kutta time steps (two projections, gravity, upwind VOF) "
                         "per second on the 256^3 workload, from the same state each step")
    ap.add_argument("--stretched", action="store_true",
                    help="the 256^3 workload's arrays on a grid stretched in z (widths 3.5:1, finest at z = 0.5)")
    ap.add_argument("--cut-cells", action="store_true",
                    help="the 256^3 workload's ellipsoid as fractional face areas from a level set (no binary mask)")
    ap.add_argument("--no-kernel-times", action="store_true",
                    help="skip the profiled run behind kernel_ms and roofline (for ncu captures)")
    ap.add_argument("--inner", type=int, default=2,
                    help="V-cycles per preconditioner application (krylov 1) or per refinement step (krylov 0)")
    ap.add_argument("--inner64", type=int, default=1, help="the same for the plain FP64 comparison solve")
    ap.add_argument("--nu1", type=int, default=2, help="pre-smoothing red-black sweeps per level")
    ap.add_argument("--nu2", type=int, default=2, help="post-smoothing red-black sweeps per level")
    ap.add_argument("--smoother", type=int, default=0,
                    help="0 auto, 1 per colour, 2 fused, 3 fused + TMA")
    ap.add_argument("--coarse-tail", type=int, default=1,
                    help="smallest levels: 0 a launch per pass, 1 one CTA (coarse_tail option)")
    ap.add_argument("--pass-order", type=int, default=1,
                    help="finest colour passes: 1 alternate descending/ascending plane order (L2 reuse), 0 ascending")
    ap.add_argument("--krylov", type=int, default=1,
                    help="1: conjugate gradients preconditioned by the V-cycle (default); 0: stationary V-cycles")
    return ap.parse_args()


def workload_name(n, workload="c3", cut_cells=False, stretched=False):
    step = (f"step = face coeffs + hierarchy + projection + adjoint projection + phi chain rule "
            f"(2 solves to rel. resid {TOL:g})")
    if workload == "c4":
        return ("512x256x128 tow-tank box [0,4]x[0,2]x[0,1] (16.8M cells), flat surface + 0.01 S, 200 seeded air "
                "bubbles r~U[2h,6h], rho ratio 1e-3, u*~N(0,0.1), w~N(0,1) seed 4; " + step)
    if workload == "c5":
        return ("1024x512x256 box (134M cells), plunging overturned interface (cubic-displaced tanh), box hull "
                "0.4x0.05x0.04 with rounded bow, rho ratio 1e-3, u*/w FP32 seed 5 promoted to FP64; " + step)
    body = ("piercing ellipsoid (0.3,0.06,0.05) as fractional face areas from a level set at the nodes"
            if cut_cells else "piercing ellipsoid (0.3,0.06,0.05)")
    grid = "; grid stretched in z (widths 3.5:1, finest at z = 0.5), no phi chain rule" if stretched else ""
    return (f"{n}^3 unit cube, 4-mode free surface (amp 0.08, seed 2) + {body}, "
            f"rho_air/rho_water 1e-3, u*~N(0,0.1) seed 3, w~N(0,1); " + step + grid)


def make_case(args):
    import numpy as np
    from paper_1410_2240_gb300 import synth
    if args.workload == "c4":
        return synth.case_c4()
    if args.workload == "c5":
        return synth.case_c5()
    case = synth.case_c3(args.n)
    if getattr(args, "cut_cells", False):  # the ellipsoid as fractional face areas, no binary mask
        case.psi_nodes = synth.ellipsoid_psi_nodes(args.n, args.n, args.n, case.h)
        case.solid = None
    if getattr(args, "stretched", False):  # the same arrays on a grid stretched in z, finest at 0.5
        case.widths = (np.full(args.n, case.h), np.full(args.n, case.h), synth.stretched_widths(args.n, 3.5, 0.5))
    return case


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.dev = device_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.dev:
            cmd += ["-i", self.dev]
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed plumbing (replicas)
# ---------------------------------------------------------------------------
def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Largest x over the ranks (the job's time is its slowest replica's)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(local_ms, solves_per_rank, world):
    """Whole-job solves/s of N independent replicas: all ranks' solves / max-over-ranks time."""
    ms = max_over_ranks(local_ms, world)
    return solves_per_rank * world / (ms / 1e3), ms


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
class Step:
    """All device buffers of one projection step; run() launches it on the current stream."""

    def __init__(self, case, prec, profile, **opts):
        import numpy as np
        import torch
        from paper_1410_2240_gb300 import mgproj
        self.mg = mgproj
        self.case = case
        dev = lambda a, dt=torch.float64: torch.from_numpy(a).to(device="cuda", dtype=dt)
        self.phi = dev(case.phi)
        self.solid = dev(case.solid, torch.uint8) if case.solid is not None else None
        self.u_star = tuple(dev(x) for x in case.u_star)
        self.w = tuple(dev(x) for x in case.w)
        self.beta = mgproj.face_coeffs(self.phi, case.h, self.solid, rho_air=case.lam)
        self.widths = None
        if getattr(case, "widths", None) is not None:  # stretched: the index grid of unit spacing
            self.widths = tuple(dev(np.asarray(w)) for w in case.widths)
            bidx, area = mgproj.stretched_metrics(*self.widths, self.beta)
            self.ctx = mgproj.Context(bidx, 1.0, prec=prec, profile=profile, **opts)
            self.ctx.set_face_areas(area)
        else:
            self.ctx = mgproj.Context(self.beta, case.h, prec=prec, profile=profile, **opts)
        psi = getattr(case, "psi_nodes", None)
        if psi is not None:  # a static body: its face areas once, kept by the context
            self.ctx.set_face_areas(mgproj.face_areas(dev(psi), case.h))
        self.u = tuple(torch.empty_like(x) for x in self.u_star)
        self.p = torch.zeros_like(self.phi)
        self.q = torch.zeros_like(self.phi)
        self.gu = tuple(torch.empty_like(x) for x in self.u_star)
        self.gb = tuple(torch.empty_like(x) for x in self.u_star)
        self.gphi = torch.empty_like(self.phi)
        self.cycles = []
        self.solve_ms = []

    def run(self):
        mg, c = self.mg, self.case
        mg.face_coeffs(self.phi, c.h, self.solid, rho_air=c.lam, out=self.beta)
        if self.widths is not None:
            bidx, _ = mg.stretched_metrics(*self.widths, self.beta)
            self.ctx.update(bidx)
        else:
            self.ctx.update(self.beta)
        self.p.zero_()
        _, _, st = self.ctx.project(self.u_star, p=self.p, tol=TOL, out=self.u)
        c1, t1 = st.cycles, st.ms_solve
        self.q.zero_()
        _, _, st = self.ctx.project_adjoint(self.w, self.p, tol=TOL, grad_u=self.gu, grad_beta=self.gb, q=self.q)
        if self.widths is None:  # (stretched: the face gradient is with respect to beta / d)
            mg.phi_grad(self.beta, self.gb, c.h, rho_air=c.lam, out=self.gphi)
        self.cycles.append((c1, st.cycles))
        self.solve_ms.append(t1 + st.ms_solve)


def time_steps(step, K, W, world):
    import torch
    for _ in range(W):
        step.run()
    torch.cuda.synchronize()
    step.ctx.profile_reset()
    step.cycles.clear()
    step.solve_ms.clear()
    launches0 = step.mg.kernel_launches()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    nvtx = getattr(torch.cuda, "nvtx", None)
    try:  # an NVTX range around the timed steps lets a profiler select them (ncu --nvtx-include)
        nvtx.range_push("timed_steps")
    except Exception:
        nvtx = None
    gc.collect()
    gc.disable()  # no collector pause inside the timed steps (as timeit does)
    try:
        e0.record(stream)
        for _ in range(K):
            step.run()
        e1.record(stream)
        if nvtx is not None:
            nvtx.range_pop()
        torch.cuda.synchronize()
    finally:
        gc.enable()
    barrier(world)
    ms = e0.elapsed_time(e1)
    return ms, step.mg.kernel_launches() - launches0


def release():
    """Free the device memory of the legs already timed now: a context left to a later garbage
    collection would release its buffers (and synchronize the device) inside another leg's timing."""
    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def e2e_leg(case, K, W, readback="loss"):
    """The same step through the public autograd API, inputs from pinned host memory, as a
    training loop would run it: two sets of device input buffers, the next step's inputs uploaded
    (on a second stream) while this step's backward solve runs.  readback = "loss": the step's
    result read back is its loss L = sum(w * u) (the gradients stay on the device, where an
    optimizer would use them); "all": the projected velocity is read back during the backward and
    the four gradients during the next step's forward instead.  The timed region holds every
    step's copies: the first step's upload, which nothing hides, and the last step's read-back
    included."""
    import torch
    from paper_1410_2240_gb300.autograd import project
    pin = lambda a, dt=torch.float64: torch.from_numpy(a).to(dtype=dt).pin_memory()
    h_phi = pin(case.phi)
    h_solid = pin(case.solid, torch.uint8) if case.solid is not None else None
    h_u = tuple(pin(x) for x in case.u_star)
    h_w = tuple(pin(x) for x in case.w)
    o_u = tuple(torch.empty_like(x).pin_memory() for x in h_u)
    o_gu = tuple(torch.empty_like(x).pin_memory() for x in h_u)
    o_gphi = torch.empty_like(h_phi).pin_memory()
    o_loss = torch.zeros(K + W, dtype=torch.float64).pin_memory()
    side = torch.cuda.Stream()
    dev_like = lambda x: torch.empty_like(x, device="cuda")
    bufs = [{"phi": dev_like(h_phi), "solid": dev_like(h_solid) if h_solid is not None else None,
             "u": tuple(dev_like(x) for x in h_u), "w": tuple(dev_like(x) for x in h_w)} for _ in range(2)]
    ready = [None, None]

    def upload(k):
        """Inputs of one step into buffer set k, on the side stream (after all work queued so far
        on the main stream, so that the set's previous user is done with it)."""
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            bk = bufs[k]
            bk["phi"].copy_(h_phi, non_blocking=True)
            if h_solid is not None:
                bk["solid"].copy_(h_solid, non_blocking=True)
            for d, x in zip(bk["u"] + bk["w"], h_u + h_w):
                d.copy_(x, non_blocking=True)
        ready[k] = side.record_event()

    def step(i, last, slot=None):
        main = torch.cuda.current_stream()
        k = i % 2
        main.wait_event(ready[k])
        bk = bufs[k]
        phi = bk["phi"].detach().requires_grad_(True)
        u = tuple(d.detach().requires_grad_(True) for d in bk["u"])
        (ux, uy, uz), p = project(u, phi, case.h, solid=bk["solid"], rho_air=case.lam, tol=TOL,
                                  precision="mixed")
        if readback == "loss":
            # the loss whose gradient the backward takes: L = sum(w * u), read back (8 bytes)
            loss = sum(torch.dot(a.detach().reshape(-1), b.reshape(-1)) for a, b in zip((ux, uy, uz), bk["w"]))
            o_loss[i if slot is None else slot].copy_(loss, non_blocking=True)
        else:
            side.wait_stream(main)
            with torch.cuda.stream(side):
                for o, x in zip(o_u, (ux, uy, uz)):
                    o.copy_(x.detach(), non_blocking=True)
                    x.record_stream(side)
        if not last:
            upload(1 - k)
        torch.autograd.backward((ux, uy, uz), bk["w"])
        if readback != "loss":
            grads = tuple(x.grad for x in u) + (phi.grad,)
            side.wait_stream(main)
            with torch.cuda.stream(side):
                for o, g in zip(o_gu + (o_gphi,), grads):
                    o.copy_(g, non_blocking=True)
                    g.record_stream(side)

    upload(0)
    for i in range(W):
        step(i, last=False, slot=K + i)
    torch.cuda.synchronize()
    steps_ms, nivcsw, nvcsw, minflt, majflt = [], [], [], [], []
    # main-stream events around each step: its span on the device, against its host time
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    mem0 = torch.cuda.memory_stats()
    load0 = os.getloadavg()
    gc.collect()
    gc.disable()  # no collector pause inside the timed steps (as timeit does)
    try:
        t0 = time.perf_counter()
        upload(0)  # the first timed step's inputs: inside the timed region, hidden by nothing
        for i in range(K):
            ts = time.perf_counter()
            ru0 = resource.getrusage(resource.RUSAGE_SELF)
            ev[i][0].record()
            step(i, last=(i == K - 1))
            ev[i][1].record()
            steps_ms.append(1e3 * (time.perf_counter() - ts))
            ru1 = resource.getrusage(resource.RUSAGE_SELF)
            nivcsw.append(ru1.ru_nivcsw - ru0.ru_nivcsw)
            nvcsw.append(ru1.ru_nvcsw - ru0.ru_nvcsw)
            minflt.append(ru1.ru_minflt - ru0.ru_minflt)
            majflt.append(ru1.ru_majflt - ru0.ru_majflt)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
    finally:
        gc.enable()
    mem1 = torch.cuda.memory_stats()
    grew = {k: mem1.get(k, 0) - mem0.get(k, 0) for k in ("segment.all.allocated", "num_alloc_retries")}
    n = case.ncell
    h2d = (7 * 8 + (1 if h_solid is not None else 0)) * n
    d2h = 8 if readback == "loss" else 7 * 8 * n
    if readback == "loss" and not all(bool(torch.isfinite(x)) for x in o_loss[:K]):
        raise RuntimeError("e2e: a step's loss is not finite")
    return {"value": 2 * K / sec, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": 1e3 * sec / K, "host_step_ms": [round(t, 2) for t in steps_ms],
            # involuntary context switches of this process per step (the host thread preempted)
            # and the host's load average before and after: a stalled step with many switches
            # and a high load points at other work on the host's cores
            "involuntary_ctx_switches_per_step": nivcsw,
            # voluntary switches (the thread blocked: a synchronisation, a lock, I/O) and page
            # faults per step: a stalled step with many of either points inside the process
            "voluntary_ctx_switches_per_step": nvcsw,
            "page_faults_per_step": {"minor": minflt, "major": majflt},
            "device_step_ms": [round(a.elapsed_time(b), 2) for a, b in ev],
            "host_loadavg_1min": [round(load0[0], 2), round(os.getloadavg()[0], 2)],
            "host_cores": os.cpu_count(),
            "allocator_during_timing": grew,
            "readback": ("the step's loss sum(w * u), 8 bytes; the gradients stay on the device" if readback == "loss"
                         else "the projected velocity and the four gradients, on a second stream"),
            "api": "paper_1410_2240_gb300.autograd.project (mixed) + backward, inputs of step i+1 uploaded "
                   "during step i's backward"}


def cpu_baseline(case):
    """The CPU FP64 oracle, as it stands, on this host's cores: a full forward solve of the
    same 256^3 problem to 1e-10 (setup included)."""
    import oracle as O
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    t0 = time.perf_counter()
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    rhs = O.divergence(beta, case.u_star, case.h)
    mg = O.MG(beta, case.h)
    t1 = time.perf_counter()
    p, cyc, _ = mg.solve(rhs, tol=TOL, max_cycles=200)
    t2 = time.perf_counter()
    # untimed: continue to 1e-12, the reference the GPU solutions' error is measured against
    p_ref, _, _ = mg.solve(rhs, p0=p, tol=1e-12, max_cycles=200)
    return {"value": 1.0 / (t2 - t0), "unit": "solves/s", "cores": threads, "kind": "oracle",
            "sample": f"one full FP64 oracle solve (stationary V(2,2) cycles) of the {case.nx}^3 workload to "
                      f"{TOL:g} (face coeffs + rhs + hierarchy {t1 - t0:.1f} s, {abs(cyc)} V-cycles {t2 - t1:.1f} s)"}, p_ref


# algorithmic bytes per finest cell and call of each event-timed group of a mixed step
GROUP_BYTES = {"smooth": B_SWEEP32, "restrict": 20.5, "prolong": 8.5, "resid64": 48.0, "cg_apply": 48.0,
               "cg_vectors": 32.0}


def kernel_gbs(kernel_ms, n):
    """Algorithmic GB/s of the finest-grid kernel groups (bytes per cell x cells x calls / time)."""
    out = {}
    for g, bpc in GROUP_BYTES.items():
        v = kernel_ms.get(g)
        if v and v["launches"] and v["ms"] > 0:
            out[g] = bpc * n * v["launches"] / (v["ms"] / 1e3) / 1e9
    return out


def run_ours(args):
    import numpy as np
    import torch
    import __graft_entry__
    from paper_1410_2240_gb300 import synth

    world, rank, local = dist_setup(args)
    if rank == 0:
        __graft_entry__.build()
    barrier(world)
    from paper_1410_2240_gb300 import mgproj
    case = make_case(args)
    n = case.ncell
    K, W = args.steps, max(args.warmup, 3)

    # ---- mixed (headline) ----
    opts = {"inner_cycles": args.inner, "smoother": args.smoother, "krylov": args.krylov,
            "coarse_tail": args.coarse_tail, "pass_order": args.pass_order, "nu1": args.nu1, "nu2": args.nu2}
    step = Step(case, "mixed", profile=0, **opts)
    dev_uuid = None
    try:
        dev_uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        dev_uuid = dev_uuid if dev_uuid.startswith("GPU-") else "GPU-" + dev_uuid
    except Exception:
        dev_uuid = None
    clocks = ClockSampler(dev_uuid)
    clocks.start()
    ms, launches = time_steps(step, K, W, world)
    clk = clocks.stop()
    value, ms = replica_throughput(ms, 2 * K, world)
    cyc_mixed = step.cycles[-1]
    steps_total = sum(a + b for a, b in step.cycles)
    solve_ms_total = sum(step.solve_ms)  # the solves alone (CUDA events inside the library)
    p_mixed = step.p.detach().cpu().numpy() if rank == 0 else None
    del step
    release()
    # per-kernel times from a second context that records CUDA events around every finest-grid
    # kernel (kept out of the headline timing above)
    prof, Kp, sweep_ms, achieved = {}, 0, None, None
    if not args.no_kernel_times:
        pstep = Step(case, "mixed", profile=1, **opts)
        Kp = max(3, min(K, 5))
        time_steps(pstep, Kp, 3, world)
        # dominant kernel: finest-grid FP32 red-black sweep
        cnt, sm_ms = pstep.ctx.profile_read(mgproj.PROF_SMOOTH)
        sweep_ms = sm_ms / max(cnt, 1)
        achieved = B_SWEEP32 * n / (sweep_ms / 1e3) / 1e9
        prof = {g: pstep.ctx.profile_read(i) for g, i in PROF_GROUPS}
        del pstep
        release()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    mixed_vcycle_gbs = (iteration_bytes(args.inner, B_VCYCLE32, args.krylov, B_REFINE) * n * steps_total
                        / (solve_ms_total / 1e3) / 1e9)


    # ---- plain FP64 on the same step ----
    fp64 = None
    if not args.no_fp64:
        s64 = Step(case, "fp64", profile=1, smoother=args.smoother, krylov=args.krylov, inner_cycles=args.inner64,
                   coarse_tail=args.coarse_tail, pass_order=args.pass_order)
        K64 = max(2, K // 2)
        ms64, _ = time_steps(s64, K64, 3, world)
        sps64, ms64 = replica_throughput(ms64, 2 * K64, world)
        cyc64 = s64.cycles[-1]
        c64, sm64 = s64.ctx.profile_read(mgproj.PROF_SMOOTH)
        sweep64 = sm64 / max(c64, 1)
        tot64 = sum(a + b for a, b in s64.cycles)
        fp64 = {"solves_per_s": sps64, "ms_per_step": ms64 / K64, "inner_cycles": args.inner64,
                "cycles_fwd_bwd": list(cyc64),
                "vcycle_hbm_gbs": (iteration_bytes(args.inner64, B_VCYCLE64, args.krylov, B_RESID64) * n * tot64
                                   / (sum(s64.solve_ms) / 1e3) / 1e9),
                "fine_sweep_ms": sweep64, "fine_sweep_gbs": B_SWEEP64 * n / (sweep64 / 1e3) / 1e9,
                "kernel_ms": {g: dict(zip(("launches", "ms"), s64.ctx.profile_read(i))) for g, i in PROF_GROUPS}}
        p64 = s64.p.detach().cpu().numpy() if rank == 0 else None
        del s64
        release()
    else:
        p64 = None

    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": workload_name(args.n, args.workload, args.cut_cells, args.stretched), "cells": n, "precision": "mixed (FP32 V-cycles, FP64 "
                   "residual/accumulation/coarsest solve)", "tol": TOL, "solves_per_step": 2,
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2: each FP64 fine array is %.0f MB, ~1.5 GB touched per step" % (8 * n / 1e6)},
        "cycles_fwd_bwd": list(cyc_mixed),
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm if achieved else None,
                     "traffic": (SWEEP_TRAFFIC_256 if (args.workload == "c3" and args.n == 256 and args.smoother in (0, 1))
                                 else None),
                     "traffic_unit": "bytes per sweep (ncu dram__bytes_read.sum + dram__bytes_write.sum)", "kernel": SWEEP_KERNEL[args.smoother] + " (finest grid, FP32, one red-black sweep)",
                     "algorithmic_bytes_per_sweep": B_SWEEP32 * n, "sweep_ms": sweep_ms,
                     "peak_source": f"{peak_src} hbm_gbs (burst copy)"},
        "vcycle_hbm_gbs": {"mixed": mixed_vcycle_gbs, "fp64": fp64["vcycle_hbm_gbs"] if fp64 else None},
        "fp64": fp64,
        "kernel_ms": {g: {"launches": c, "ms": t} for g, (c, t) in prof.items()},
        "kernel_ms_steps": Kp,
        "clocks": clk,
    }
    out["projections_per_s"] = value / 2.0  # one projection step = forward + adjoint
    # fine-cell V-cycles per second (all V-cycles of the timed steps over the solves' own time)
    # and smoother cell updates per second (cells / time of one finest-grid sweep)
    out["fine_cell_vcycles_per_s"] = n * args.inner * steps_total / (solve_ms_total / 1e3)
    out["smoother_cell_updates_per_s"] = n / (sweep_ms / 1e3) if sweep_ms else None
    out["kernel_gbs"] = kernel_gbs(out["kernel_ms"], n)
    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_leg(case, max(4, K), 5)
        # the same with the projected velocity and all four gradients read back (940 MB a step):
        # the copies engines' reads of device memory slow the overlapped solves (reported, not the
        # headline: the result the contract reads back is the loss)
        full = e2e_leg(case, max(4, K), 5, readback="all")
        out["e2e"]["all_results_read_back"] = {k: full[k] for k in ("value", "ms_per_step", "d2h_bytes_per_step",
                                                                     "device_step_ms")}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload != "c5":
        cb, p_or = cpu_baseline(case)
        out["cpu_baseline"] = cb
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        out["error_vs_oracle"] = {"p_mixed": rel(p_mixed, p_or), "p_fp64": rel(p64, p_or) if p64 is not None else None,
                                  "note": "p of the last timed step's forward solve (rel. residual <= 1e-10) vs the "
                                          "oracle's solve continued to 1e-12"}
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------
def run_reference(args):
    """The CPU FP64 oracle on this host's cores, each step one whole solve of the 256^3 workload
    as the cpu_baseline leg times it: face coefficients, right-hand side, hierarchy and
    stationary V(2,2) cycles to 1e-10 (mean removal and residual norm after every cycle)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_1410_2240_gb300 import synth
    case = synth.case_c3(args.n)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))

    def one_solve():
        beta = O.face_coeffs(case.phi, case.solid, case.lam)
        rhs = O.divergence(beta, case.u_star, case.h)
        mg = O.MG(beta, case.h)
        _, cyc, _ = mg.solve(rhs, tol=TOL, max_cycles=200)
        return abs(cyc)

    for _ in range(args.warmup):
        one_solve()
    times, cycles = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cycles = one_solve()
        times.append(time.perf_counter() - t0)
    sec = sum(times)
    value = args.steps / sec
    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": workload_name(args.n), "cells": case.ncell, "tol": TOL},
           "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle",
                            "sample": f"each step = one whole FP64 oracle solve of the {args.n}^3 workload (face "
                                      f"coefficients, rhs, hierarchy, {cycles} stationary V(2,2) cycles to "
                                      f"{TOL:g}); median step {1e3 * statistics.median(times):.0f} ms"},
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def pcg_scaling(args):
    """The Poisson-solver section's comparison of diagonally preconditioned CG with multigrid:
    iterations to relative residual 1e-10 and solve time (CUDA events inside the library, the
    second of two solves) per method and resolution, one JSON line."""
    import torch
    import __graft_entry__
    from paper_1410_2240_gb300 import synth
    __graft_entry__.build()
    from paper_1410_2240_gb300 import mgproj
    dev = lambda a, dt=torch.float64: torch.from_numpy(a).to(device="cuda", dtype=dt)
    methods = (("jacobi_pcg_fp64", dict(krylov=1, precond=1, max_cycles=200000)),
               ("mg_vcycles_fp64", dict(krylov=0)),
               ("mg_pcg_fp64", dict(krylov=1, inner_cycles=1)),
               ("mg_pcg_mixed", dict(krylov=1, inner_cycles=2, prec="mixed")))
    rows = []
    for n in (64, 128, 256):
        case = synth.case_c2(n, geom_seed=2, field_seed=3)
        beta = mgproj.face_coeffs(dev(case.phi), case.h, dev(case.solid, torch.uint8), rho_air=case.lam)
        rhs = mgproj.Context(beta, case.h).divergence(tuple(dev(x) for x in case.u_star))
        for name, kw in methods:
            ctx = mgproj.Context(beta, case.h, **kw)
            for _ in range(2):
                _, st = ctx.solve(rhs, tol=TOL)
            rows.append({"n": n, "method": name, "iterations": st.cycles, "solve_ms": st.ms_solve,
                         "rel_resid": st.rel_resid})
            del ctx
            torch.cuda.empty_cache()
    print(json.dumps({"experiment": "jacobi-preconditioned CG vs multigrid, iterations and solve time",
                      "workload": "unit cube, 4-mode free surface + ellipsoid (the 256^3 benchmark geometry), "
                                  "rho_air/rho_water 1e-3", "tol": TOL, "rows": rows}))


def rk2_bench(args):
    """Time steps of mg_rk2_step per second (CUDA events, the same initial state each step: u and phi
    restored by device copies inside the timed region), one JSON line."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_2240_gb300 import mgproj
    case = make_case(args)
    dev = lambda a, dt=torch.float64: torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)
    phi = dev(case.phi)
    solid = dev(case.solid, torch.uint8) if case.solid is not None else None
    u0 = tuple(dev(x) for x in case.u_star)
    u = [x.clone() for x in u0]
    beta = mgproj.face_coeffs(phi, case.h, solid, rho_air=case.lam)
    ctx = mgproj.Context(beta, case.h, prec="mixed", krylov=1, inner_cycles=args.inner)
    phi1 = torch.empty_like(phi)
    p = torch.empty_like(phi)
    dt, g = 0.2 * case.h, 1.0
    # Eq. navi's other terms: gravity (1/Fr^2 = 1), viscosity at Re = 1e6 with the air/water ratio
    # 0.018, convection
    inv_re, mu_air = 1e-6, 1.8e-2
    forces = mgproj.forces(g=g, inv_re=inv_re, mu_air=mu_air, convection=True)
    cycles = []

    def step():
        for a, b in zip(u, u0):
            a.copy_(b)
        _, _, st = ctx.rk2_step(phi, u, dt, solid=solid, rho_air=case.lam, tol=TOL, phi_out=phi1, p=p, forces=forces)
        cycles.append(st.cycles)

    K, W = args.steps, max(args.warmup, 3)
    for _ in range(W):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = mgproj.kernel_launches()
    e0.record()
    for _ in range(K):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # the momentum right-hand side alone (mg_momentum_rhs on u^k, phi^k): CUDA events over 10 calls
    R = tuple(torch.empty_like(x) for x in u0)
    work = torch.empty(12 * phi.numel(), dtype=torch.float64, device="cuda")
    for _ in range(2):
        mgproj.momentum_rhs(phi, beta, u0, case.h, forces, out=R, work=work)
    e0.record()
    for _ in range(10):
        mgproj.momentum_rhs(phi, beta, u0, case.h, forces, out=R, work=work)
    e1.record()
    torch.cuda.synchronize()
    mom_ms = e0.elapsed_time(e1) / 10
    print(json.dumps({"metric": "Runge-Kutta time steps per second (2 projections to rel. resid 1e-10, gravity, "
                                "viscous and convective terms, upwind VOF)", "value": K / (ms / 1e3), "unit": "steps/s",
                      "ms_per_step": ms / K,
                      "solves_per_s": 2 * K / (ms / 1e3), "second_stage_cg_iterations": cycles[-1],
                      "momentum_rhs_ms": mom_ms,
                      "gpu_launches": int(mgproj.kernel_launches() - launches0), "steps": K, "warmup": W,
                      "config": {"workload": f"{args.n}^3 unit cube, 4-mode free surface (amp 0.08, seed 2) + "
                                             "piercing ellipsoid (0.3,0.06,0.05), rho_air/rho_water 1e-3, u^k ~ "
                                             "N(0,0.1) seed 3; step = Runge-Kutta step with two projections",
                                 "dt": dt, "g": g, "inv_re": inv_re, "mu_air": mu_air, "convection": True,
                                 "precision": "mixed"}}))


ORACLE_CASES = {"c1_32": "32^3, gently waved interface, no solid, rhs ~ N(0,1)",
                "c2_128": "128^3, 4-mode free surface + piercing ellipsoid, rhs = D u*",
                "c3_256": "256^3, as 128^3 (the benchmark's workload)"}


def oracle_solve(name):
    """One timed FP64 oracle solve (face coefficients + rhs + hierarchy + stationary V(2,2) cycles to
    1e-10) in this process, with the OpenMP threads its environment gives; prints a JSON line."""
    import oracle as O
    from paper_1410_2240_gb300 import synth
    case = {"c1_32": lambda: synth.case_c1(32), "c2_128": lambda: synth.case_c2(128),
            "c3_256": lambda: synth.case_c3(256)}[name]()
    t0 = time.perf_counter()
    beta = O.face_coeffs(case.phi, case.solid, case.lam)
    rhs = case.rhs if case.rhs is not None else O.divergence(beta, case.u_star, case.h)
    mg = O.MG(beta, case.h)
    t1 = time.perf_counter()
    _, cyc, _ = mg.solve(rhs, tol=TOL, max_cycles=200)
    t2 = time.perf_counter()
    print(json.dumps({"setup_s": t1 - t0, "solve_s": t2 - t1, "cycles": abs(cyc)}))


def oracle_timing(args):
    """The CPU oracle timed on this host: each workload's full solve with all cores and with one,
    each in a child process (the oracle's OpenMP thread count is fixed when it loads)."""
    cores = os.cpu_count() or 1
    rows = []
    for name, what in ORACLE_CASES.items():
        for threads in (cores, 1):
            env = dict(os.environ, OMP_NUM_THREADS=str(threads))
            out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-solve", name], env=env,
                                 capture_output=True, text=True, check=True)
            r = json.loads(out.stdout.strip().splitlines()[-1])
            total = r["setup_s"] + r["solve_s"]
            rows.append({"workload": name, "what": what, "threads": threads, "cycles": r["cycles"],
                         "setup_s": round(r["setup_s"], 3), "solve_s": round(r["solve_s"], 3),
                         "solves_per_s": 1.0 / total})
    print(json.dumps({"metric": "CPU oracle solves/s to 1e-10 (FP64, stationary V(2,2))", "unit": "solves/s",
                      "kind": "oracle", "host_cores": cores, "rows": rows}))


def main():
    args = parse_args()
    if args.oracle_solve:
        oracle_solve(args.oracle_solve)
    elif args.oracle_timing:
        oracle_timing(args)
    elif args.pcg_scaling:
        pcg_scaling(args)
    elif args.rk2:
        rk2_bench(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
