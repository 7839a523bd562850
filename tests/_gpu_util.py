"""Helpers shared by the GPU parity tests (host <-> device marshalling only)."""
import numpy as np
import torch

import oracle as O
from paper_1410_2240_gb300 import synth


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def faces_dev(fs):
    return tuple(dev(f) for f in fs)


def faces_host(fs):
    return tuple(host(f) for f in fs)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def case_rhs(case, beta):
    """The case's raw rhs, or D u* / dt computed by the oracle."""
    if case.rhs is not None:
        return case.rhs
    return O.divergence(beta, case.u_star, case.h, case.dt)


def cases_small():
    return {
        "c1": synth.case_c1(),
        "c2_64": synth.case_c2(64),
        "ell16": synth.small_case(16, solid="ellipsoid", seed=31),
        "ragged_160x32x32": synth.small_case(160, 32, 32, solid="none", seed=32),
        "odd_coarse_24": synth.small_case(24, solid="ellipsoid", seed=33),
        "aniso_64x32x16": synth.small_case(64, 32, 16, solid="ellipsoid", seed=34),
    }
