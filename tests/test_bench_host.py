"""Host logic of bench.py's replica mode on CPU: two gloo ranks (world size 2, no GPU)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [1000.0, 1500.0][rank]
    value, ms = bench.replica_throughput(local_ms, 40, world)
    bench.barrier(world)
    out[rank] = (value, ms)
    dist.destroy_process_group()


def test_replica_throughput_is_max_over_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        value, ms = res[r]
        assert ms == 1500.0                      # slowest replica
        assert value == pytest.approx(80 / 1.5)  # all ranks' solves / max time


def test_reference_arm_nonzero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_prints_contract_line_small_grid():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "32",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_oracle_timing_child_times_a_full_solve():
    """The child of --oracle-timing: one oracle solve of the 32^3 workload on one thread, its
    setup and solve seconds and its V-cycle count as JSON (the cycle count is the oracle's own)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-solve", "c1_32"], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["setup_s"] > 0 and line["solve_s"] > 0
    assert 5 <= line["cycles"] <= 40


def test_iteration_bytes_count_every_v_cycle():
    sys.path.insert(0, ROOT)
    import bench
    # two FP32 V-cycles and the CG vectors per iteration; one cycle and the refinement step otherwise
    assert bench.iteration_bytes(2, bench.B_VCYCLE32, 1, bench.B_REFINE) == 2 * bench.B_VCYCLE32 + bench.B_CG_ITER
    assert bench.iteration_bytes(1, bench.B_VCYCLE64, 0, bench.B_RESID64) == bench.B_VCYCLE64 + bench.B_RESID64
