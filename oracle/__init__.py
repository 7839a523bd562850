"""CPU FP64 oracle of the variable-density pressure projection (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library neither imports nor
links it, and it imports nothing from the product package.

The arithmetic lives in ``mg_oracle.c`` (plain loops, FP64).  The smoother,
the residual and the prolongation accumulate their stencil products with C99
``fma`` in the order x-, x+, y-, y+, z-, z+ (the rounding the paper leaves open,
read the same way on both sides); every other operation is a separately rounded
IEEE operation.  This module compiles it with gcc on first use and wraps it with
ctypes and NumPy.  Dense NumPy/SciPy helpers here (``dense_solve``,
``thomas_layered``) are independent second computations used by the pins.

Function -> paper passage:
  face_coeffs      Eq. density (H(phi) = phi) and the Poisson-solver section's
                   face product (1/rho) * area, harmonic face mean of 1/rho
  apply_A          Eq. pois in the finite-volume form of Eq. integral2
  divergence       right-hand side of Eq. poisson1 (static body: no flux)
  correct          Eq. runge1's pressure term
  mg_solve/vcycle  the multigrid of the Poisson-solver section (face-coefficient
                   restriction); smoother, transfers and cycle are the readings
                   listed in the design notes (the paper does not give them)
  cg_solve         the paper's earlier solver family (preconditioned CG)
  MG.pcg           CG preconditioned by the multigrid cycle (the two combined)
  project_adjoint  derived adjoint of the projection
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile mg_oracle.c into _build/liboracle.so (gcc, -O2, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def use_library(path: Optional[str]) -> None:
    """Load the oracle from another compiled copy of mg_oracle.c (None = the default build).

    Used only by the mutation tests, which plant a mistake in a copy of the source and
    check that the pins catch it."""
    global _lib
    with _lock:
        _lib = None
    _load(path)


def _load(path: Optional[str] = None):
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(path or build())
            sz = ctypes.c_size_t
            i = ctypes.c_int
            d = ctypes.c_double
            v = ctypes.c_void_p
            lib.orc_face_coeffs.argtypes = [i, i, i, _D, v, d, _D, _D, _D]
            lib.orc_apply_A.argtypes = [i, i, i, d, _D, _D, _D, _D, _D]
            lib.orc_diag_inv.argtypes = [i, i, i, _D, _D, _D, _D]
            lib.orc_components.argtypes = [i, i, i, _D, _D, _D, _I]
            lib.orc_components.restype = i
            lib.orc_remove_mean.argtypes = [sz, _I, i, _D]
            lib.orc_smooth_colour.argtypes = [i, i, i, d, _D, _D, _D, _D, _D, _D, i]
            lib.orc_restrict_coeffs.argtypes = [i, i, i, _D, _D, _D, _D, _D, _D]
            lib.orc_residual.argtypes = [i, i, i, d, _D, _D, _D, _D, _D, _D]
            lib.orc_restrict.argtypes = [i, i, i, _D, _D]
            lib.orc_prolong_add.argtypes = [i, i, i, _D, _D, _D]
            lib.orc_pinv_sym.argtypes = [i, _D, _D]
            lib.orc_dense_A.argtypes = [i, i, i, d, _D, _D, _D, _D]
            lib.orc_mg_create.argtypes = [i, i, i, d, _D, _D, _D, i, i, i]
            lib.orc_mg_create.restype = v
            lib.orc_mg_free.argtypes = [v]
            lib.orc_mg_nlev.argtypes = [v]
            lib.orc_mg_nlev.restype = i
            lib.orc_mg_ok.argtypes = [v]
            lib.orc_mg_ok.restype = i
            lib.orc_mg_level_dims.argtypes = [v, i, _I]
            lib.orc_mg_level_array.argtypes = [v, i, i]
            lib.orc_mg_level_array.restype = _D
            lib.orc_mg_pinv.argtypes = [v]
            lib.orc_mg_pinv.restype = _D
            lib.orc_mg_vcycle.argtypes = [v, _D, _D]
            lib.orc_mg_solve.argtypes = [v, _D, _D, d, i, _D]
            lib.orc_mg_solve.restype = i
            lib.orc_mg_pcg.argtypes = [v, _D, _D, d, i, i, _D]
            lib.orc_mg_pcg.restype = i
            lib.orc_cg_solve.argtypes = [i, i, i, d, _D, _D, _D, _D, _D, d, i]
            lib.orc_cg_solve.restype = i
            lib.orc_divergence.argtypes = [i, i, i, d, d, _D, _D, _D, _D, _D, _D, _D]
            lib.orc_correct.argtypes = [i, i, i, d, d, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]
            lib.orc_face_scale.argtypes = [sz, _D, _D, _D, _D, _D, _D, _D, _D, _D]
            lib.orc_gradient.argtypes = [i, i, i, d, _D, _D, _D, _D, _D, _D, _D]
            lib.orc_phi_grad.argtypes = [i, i, i, d, _D, _D, _D, _D, _D, _D, _D]
            lib.orc_face_open.argtypes = [d, d, d, d]
            lib.orc_face_open.restype = d
            lib.orc_face_areas.argtypes = [i, i, i, _D, _D, _D, _D]
            lib.orc_divergence_area.argtypes = [i, i, i, d, d] + [_D] * 10
            lib.orc_stretched_metrics.argtypes = [i, i, i] + [_D] * 15
            lib.orc_vof_upwind.argtypes = [i, i, i, d, d] + [_D] * 8
            lib.orc_momentum_rhs.argtypes = [i, i, i, d, _D, d, d, d, d, i] + [_D] * 9
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous, (a.dtype, a.flags)
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dims(a: np.ndarray):
    nz, ny, nx = a.shape
    return nx, ny, nz


# ---------------------------------------------------------------------------
# Elementary operators
# ---------------------------------------------------------------------------

def face_coeffs(phi, solid=None, lam=1e-3):
    """(bx, by, bz): beta = 2 / (rho_L + rho_R) on open faces, rho = lam + (1-lam) phi."""
    lib = _load()
    phi = _f64(phi)
    nx, ny, nz = _dims(phi)
    out = [np.empty_like(phi) for _ in range(3)]
    sp = None
    if solid is not None:
        solid = np.ascontiguousarray(solid, dtype=np.uint8)
        sp = solid.ctypes.data_as(ctypes.c_void_p)
    lib.orc_face_coeffs(nx, ny, nz, _p(phi), sp, lam, *[_p(o) for o in out])
    return tuple(out)


def apply_A(beta, p, h):
    lib = _load()
    p = _f64(p)
    nx, ny, nz = _dims(p)
    out = np.empty_like(p)
    lib.orc_apply_A(nx, ny, nz, h, *[_p(_f64(b)) for b in beta], _p(p), _p(out))
    return out


def diag_inv(beta):
    lib = _load()
    nx, ny, nz = _dims(beta[0])
    out = np.empty_like(_f64(beta[0]))
    lib.orc_diag_inv(nx, ny, nz, *[_p(_f64(b)) for b in beta], _p(out))
    return out


def components(beta):
    """(labels int32 array, count): connected fluid components over open faces."""
    lib = _load()
    nx, ny, nz = _dims(beta[0])
    lab = np.empty(beta[0].shape, dtype=np.int32)
    n = lib.orc_components(nx, ny, nz, *[_p(_f64(b)) for b in beta], lab.ctypes.data_as(_I))
    return lab, n


def remove_mean(v, labels, ncomp):
    lib = _load()
    v = _f64(v).copy()
    lib.orc_remove_mean(v.size, np.ascontiguousarray(labels, np.int32).ctypes.data_as(_I), ncomp, _p(v))
    return v


def smooth_colour(beta, dinv, b, p, h, colour):
    lib = _load()
    p = _f64(p).copy()
    nx, ny, nz = _dims(p)
    lib.orc_smooth_colour(nx, ny, nz, h, *[_p(_f64(x)) for x in beta], _p(_f64(dinv)), _p(_f64(b)), _p(p), colour)
    return p


def restrict_coeffs(beta):
    lib = _load()
    nx, ny, nz = _dims(beta[0])
    out = [np.empty((nz // 2, ny // 2, nx // 2)) for _ in range(3)]
    lib.orc_restrict_coeffs(nx, ny, nz, *[_p(_f64(b)) for b in beta], *[_p(o) for o in out])
    return tuple(out)


def residual(beta, b, p, h):
    lib = _load()
    p = _f64(p)
    nx, ny, nz = _dims(p)
    out = np.empty_like(p)
    lib.orc_residual(nx, ny, nz, h, *[_p(_f64(x)) for x in beta], _p(_f64(b)), _p(p), _p(out))
    return out


def restrict(r):
    lib = _load()
    r = _f64(r)
    nx, ny, nz = _dims(r)
    out = np.empty((nz // 2, ny // 2, nx // 2))
    lib.orc_restrict(nx, ny, nz, _p(r), _p(out))
    return out


def prolong_add(ec, dinv, p):
    lib = _load()
    p = _f64(p).copy()
    nx, ny, nz = _dims(p)
    lib.orc_prolong_add(nx, ny, nz, _p(_f64(ec)), _p(_f64(dinv)), _p(p))
    return p


def pinv_sym(A):
    lib = _load()
    A = _f64(A)
    n = A.shape[0]
    out = np.empty_like(A)
    lib.orc_pinv_sym(n, _p(A), _p(out))
    return out


def dense_A(beta, h):
    lib = _load()
    nx, ny, nz = _dims(beta[0])
    n = nx * ny * nz
    out = np.empty((n, n))
    lib.orc_dense_A(nx, ny, nz, h, *[_p(_f64(b)) for b in beta], _p(out))
    return out


# ---------------------------------------------------------------------------
# Multigrid
# ---------------------------------------------------------------------------

class MG:
    """Oracle multigrid hierarchy: V(nu1, nu2), red-black GS, exact coarsest solve."""

    def __init__(self, beta, h, nu1=2, nu2=2, max_coarse=4096):
        self._lib = _load()
        self.beta = tuple(_f64(b) for b in beta)
        nx, ny, nz = _dims(self.beta[0])
        self.shape = (nz, ny, nx)
        self.h = h
        self._m = self._lib.orc_mg_create(nx, ny, nz, h, *[_p(b) for b in self.beta], nu1, nu2, max_coarse)
        if not self._lib.orc_mg_ok(self._m):
            self._lib.orc_mg_free(self._m)
            self._m = None
            raise ValueError("coarsest grid too large for the dense solve")

    def __del__(self):
        if getattr(self, "_m", None):
            self._lib.orc_mg_free(self._m)
            self._m = None

    @property
    def nlev(self):
        return self._lib.orc_mg_nlev(self._m)

    def level_dims(self, l):
        d = (ctypes.c_int * 3)()
        self._lib.orc_mg_level_dims(self._m, l, d)
        return tuple(d)

    def level_array(self, l, which):
        """which: 0,1,2 = beta x,y,z; 3 = dinv.  Returns a copy of shape (nz, ny, nx)."""
        nx, ny, nz = self.level_dims(l)
        ptr = self._lib.orc_mg_level_array(self._m, l, which)
        return np.ctypeslib.as_array(ptr, shape=(nz * ny * nx,)).reshape(nz, ny, nx).copy()

    def coarse_pinv(self):
        nx, ny, nz = self.level_dims(self.nlev - 1)
        n = nx * ny * nz
        return np.ctypeslib.as_array(self._lib.orc_mg_pinv(self._m), shape=(n * n,)).reshape(n, n).copy()

    def vcycle(self, b, p):
        p = _f64(p).copy()
        self._lib.orc_mg_vcycle(self._m, _p(_f64(b)), _p(p))
        return p

    def pcg(self, b, p0=None, tol=1e-10, max_it=100, vcycles=1):
        """Multigrid-preconditioned CG: returns (p, iterations, history); iterations < 0 if not converged."""
        p = np.zeros(self.shape) if p0 is None else _f64(p0).copy()
        hist = np.zeros(max_it)
        it = self._lib.orc_mg_pcg(self._m, _p(_f64(b)), _p(p), tol, max_it, vcycles, _p(hist))
        return p, it, hist[: abs(it)]

    def solve(self, b, p0=None, tol=1e-10, max_cycles=100):
        """Returns (p, cycles, history).  cycles < 0 if not converged."""
        p = np.zeros(self.shape) if p0 is None else _f64(p0).copy()
        hist = np.zeros(max_cycles)
        cyc = self._lib.orc_mg_solve(self._m, _p(_f64(b)), _p(p), tol, max_cycles, _p(hist))
        return p, cyc, hist[: abs(cyc)]


def cg_solve(beta, b, h, tol=1e-13, max_it=20000, p0=None):
    lib = _load()
    b = _f64(b)
    nx, ny, nz = _dims(b)
    p = np.zeros_like(b) if p0 is None else _f64(p0).copy()
    it = lib.orc_cg_solve(nx, ny, nz, h, *[_p(_f64(x)) for x in beta], _p(b), _p(p), tol, max_it)
    return p, it


# ---------------------------------------------------------------------------
# Projection and its adjoint
# ---------------------------------------------------------------------------

def divergence(beta, u, h, dt=1.0):
    lib = _load()
    nx, ny, nz = _dims(beta[0])
    out = np.empty((nz, ny, nx))
    lib.orc_divergence(nx, ny, nz, h, dt, *[_p(_f64(b)) for b in beta], *[_p(_f64(x)) for x in u], _p(out))
    return out


def correct(beta, p, u_star, h, dt=1.0):
    lib = _load()
    nx, ny, nz = _dims(beta[0])
    out = [np.empty((nz, ny, nx)) for _ in range(3)]
    lib.orc_correct(nx, ny, nz, h, dt, *[_p(_f64(b)) for b in beta], _p(_f64(p)),
                    *[_p(_f64(x)) for x in u_star], *[_p(o) for o in out])
    return tuple(out)


def gradient(beta, q, h):
    lib = _load()
    nx, ny, nz = _dims(beta[0])
    out = [np.empty((nz, ny, nx)) for _ in range(3)]
    lib.orc_gradient(nx, ny, nz, h, *[_p(_f64(b)) for b in beta], _p(_f64(q)), *[_p(o) for o in out])
    return tuple(out)


def phi_grad(beta, grad_beta, lam):
    lib = _load()
    nx, ny, nz = _dims(beta[0])
    out = np.empty((nz, ny, nx))
    lib.orc_phi_grad(nx, ny, nz, lam, *[_p(_f64(b)) for b in beta], *[_p(_f64(g)) for g in grad_beta], _p(out))
    return out


def solve(beta, b, h, tol=1e-12, method="mg", max_cycles=200):
    if method == "mg":
        p, cyc, _ = MG(beta, h).solve(b, tol=tol, max_cycles=max_cycles)
        if cyc < 0:
            raise RuntimeError("oracle multigrid did not converge")
        return p
    p, it = cg_solve(beta, b, h, tol=tol)
    if it < 0:
        raise RuntimeError("oracle CG did not converge")
    return p


def project(phi, solid, u_star, h, dt=1.0, lam=1e-3, tol=1e-12, method="mg"):
    """Forward projection: returns (u, p, beta, rhs)."""
    beta = face_coeffs(phi, solid, lam)
    rhs = divergence(beta, u_star, h, dt)
    p = solve(beta, rhs, h, tol=tol, method=method)
    u = correct(beta, p, u_star, h, dt)
    return u, p, beta, rhs


def project_adjoint(beta, p, w, h, dt=1.0, lam=1e-3, tol=1e-12, method="mg"):
    """Backward of the projection for the loss sum(w * u): returns (grad_u_star, grad_beta, grad_phi)."""
    bw = tuple(b * x for b, x in zip(beta, w))
    c = divergence(beta, bw, h, 1.0)
    q = solve(beta, c, h, tol=tol, method=method)
    gq = gradient(beta, q, h)
    gp = gradient(beta, p, h)
    grad_u = tuple(np.where(b > 0, x - g, x) for b, x, g in zip(beta, w, gq))
    grad_beta = tuple(np.where(b > 0, dt * a * (g - x), 0.0) for b, a, g, x in zip(beta, gp, gq, w))
    grad_phi = phi_grad(beta, grad_beta, lam)
    return grad_u, grad_beta, grad_phi


# ---------------------------------------------------------------------------
# Fractional face areas (Body Boundary Conditions section, Eq. integral2)
# ---------------------------------------------------------------------------

def face_open(f00, f10, f01, f11):
    """Open fraction of one face from its corner values of psi (orc_face_open)."""
    lib = _load()
    return lib.orc_face_open(float(f00), float(f10), float(f01), float(f11))


def face_areas(psi_nodes):
    """Open fractions (ax, ay, az) of the low faces from psi at the nodes ((nz+1, ny+1, nx+1)),
    psi > 0 outside the body; wall faces 0."""
    lib = _load()
    psi = _f64(psi_nodes)
    nz, ny, nx = (s - 1 for s in psi.shape)
    out = [np.empty((nz, ny, nx)) for _ in range(3)]
    lib.orc_face_areas(nx, ny, nz, _p(psi), *[_p(o) for o in out])
    return tuple(out)


def area_coeffs(areas, beta):
    """Operator coefficients of Eq. integral2: area fraction times 1/rho on each face (one rounded
    product; 0 where the area is 0)."""
    return tuple(np.where(a > 0, a * b, 0.0) for a, b in zip(areas, beta))


def open_mask(areas, beta):
    """1/rho on the faces with an open area, 0 elsewhere (the correction's coefficient)."""
    return tuple(np.where(a > 0, b, 0.0) for a, b in zip(areas, beta))


def divergence_area(areas, u, h, dt=1.0, v=None):
    """b = D_a (u - v) / dt (orc_divergence_area); v = None: a static body."""
    lib = _load()
    nx, ny, nz = _dims(areas[0])
    out = np.empty((nz, ny, nx))
    vv = [None, None, None] if v is None else [_p(_f64(x)) for x in v]
    lib.orc_divergence_area(nx, ny, nz, h, dt, *[_p(_f64(a)) for a in areas], *[_p(_f64(x)) for x in u],
                            *vv, _p(out))
    return out


def project_area(phi, areas, u_star, h, dt=1.0, lam=1e-3, tol=1e-12, v=None):
    """Forward projection with fractional face areas: the operator on area * 1/rho, the
    right-hand side D_a (u* - v)/dt, the correction with 1/rho on faces of open area.
    Returns (u, p, beta (1/rho, no solid mask), rhs)."""
    beta = face_coeffs(phi, None, lam)
    ce = area_coeffs(areas, beta)
    rhs = divergence_area(areas, u_star, h, dt, v)
    p = solve(ce, rhs, h, tol=tol)
    u = correct(open_mask(areas, beta), p, u_star, h, dt)
    return u, p, beta, rhs


def project_adjoint_area(beta, areas, p, w, h, dt=1.0, lam=1e-3, tol=1e-12):
    """Backward of project_area for the loss sum(w * u): with B = diag(1/rho), D_a = D diag(a),
    A = D_a B G, G = -D^T on open faces,
        grad_u*  = w - a (G q),                 A q = D (B w)
        grad_beta = dt (G p) (a (G q) - w)      (faces of open area; 0 elsewhere)
        grad_phi  as for binary faces, from grad_beta.
    Returns (grad_u_star, grad_beta, grad_phi)."""
    bo = open_mask(areas, beta)
    ce = area_coeffs(areas, beta)
    bw = tuple(b * x for b, x in zip(bo, w))
    c = divergence(bo, bw, h, 1.0)
    q = solve(ce, c, h, tol=tol)
    gq = gradient(bo, q, h)
    gp = gradient(bo, p, h)
    grad_u = tuple(np.where(a > 0, x - a * g, x) for a, x, g in zip(areas, w, gq))
    grad_beta = tuple(np.where(a > 0, dt * gpp * (a * g - x), 0.0) for a, gpp, g, x in zip(areas, gp, gq, w))
    grad_phi = phi_grad(bo, grad_beta, lam)
    return grad_u, grad_beta, grad_phi


# ---------------------------------------------------------------------------
# Stretched grids: the index-grid form (unit spacing) of Eq. integral2 times the cell volume
# ---------------------------------------------------------------------------

def stretched_metrics(hx, hy, hz, beta, frac=None):
    """(beta_idx, area) of every low face for cell widths hx (nx), hy (ny), hz (nz):
    beta_idx = beta / (distance between the cell centres), area = the face's two widths times
    the open fraction (frac, or 1); walls 0.  With these and unit spacing, the operator is
    area * beta_idx, the divergence the cell volume times b, the correction the physical one."""
    lib = _load()
    nx, ny, nz = len(hx), len(hy), len(hz)
    ob = [np.empty((nz, ny, nx)) for _ in range(3)]
    ar = [np.empty((nz, ny, nx)) for _ in range(3)]
    ff = [None, None, None] if frac is None else [_p(_f64(f)) for f in frac]
    lib.orc_stretched_metrics(nx, ny, nz, _p(_f64(hx)), _p(_f64(hy)), _p(_f64(hz)), *[_p(_f64(b)) for b in beta],
                              *ff, *[_p(o) for o in ob], *[_p(a) for a in ar])
    return tuple(ob), tuple(ar)


def project_stretched(phi, hx, hy, hz, u_star, dt=1.0, lam=1e-3, tol=1e-12, frac=None, v=None):
    """Forward projection on a stretched grid: the fractional-area projection on the index grid
    (unit spacing) with the metrics above.  Returns (u, p, beta_idx, area, rhs) with rhs = the
    cell volume times b."""
    beta = face_coeffs(phi, None, lam)
    bi, area = stretched_metrics(hx, hy, hz, beta, frac)
    ce = area_coeffs(area, bi)
    rhs = divergence_area(area, u_star, 1.0, dt, v)
    p = solve(ce, rhs, 1.0, tol=tol)
    u = correct(open_mask(area, bi), p, u_star, 1.0, dt)
    return u, p, bi, area, rhs


# ---------------------------------------------------------------------------
# The time step (Numerical Time Integration section): two projections, Eq. poisson1 / runge1 and
# Eq. poisson2 / runge2, and the VOF operator
# ---------------------------------------------------------------------------

def vof_upwind(beta, u, phi, h, dt):
    """VOF(u, phi, dt) of orc_vof_upwind (first-order upwind fluxes through the open faces)."""
    lib = _load()
    nx, ny, nz = _dims(beta[0])
    out = np.empty((nz, ny, nx))
    lib.orc_vof_upwind(nx, ny, nz, h, dt, *[_p(_f64(b)) for b in beta], *[_p(_f64(x)) for x in u], _p(_f64(phi)),
                       _p(out))
    return out


def momentum_rhs(phi, beta, u, h, g=0.0, inv_re=0.0, mu_air=1.8e-2, mu_water=1.0, convect=True):
    """R_i of Eq. navi without the pressure and sub-grid terms (orc_momentum_rhs): the convective
    term -d/dx_j (u_j u_i) (if convect), the viscous term inv_re * beta * d/dx_j (2 mu S_ij) with
    mu = mu_air + (mu_water - mu_air) phi (Eq. density) and beta = 1/rho on the face, and -g on the
    z-faces; open faces only (beta > 0), free-slip walls."""
    lib = _load()
    nx, ny, nz = _dims(beta[0])
    out = [np.empty((nz, ny, nx)) for _ in range(3)]
    lib.orc_momentum_rhs(nx, ny, nz, h, _p(_f64(phi)), mu_air, mu_water, inv_re, g, 1 if convect else 0,
                         *[_p(_f64(b)) for b in beta], *[_p(_f64(x)) for x in u], *[_p(o) for o in out])
    return tuple(out)


def rk2_step(phi, solid, u, h, dt, g, lam=1e-3, tol=1e-12, inv_re=0.0, mu_air=1.8e-2, convect=False):
    """One step of the second-order Runge-Kutta scheme:
        u~  = u^k + dt R(u^k, phi^k);  P* from Eq. poisson1 with rho(phi^k);
        u*  = u~ - dt B G P*                                                             (Eq. runge1)
        phi* = phi^k - VOF(u^k, phi^k, dt)
        u~~ = u* + u^k + dt R(u*, phi*);  P from Eq. poisson2 with rho(phi*);
        u^{k+1} = (u~~ - dt B* G P) / 2                                                  (Eq. runge2)
        phi^{k+1} = phi^k - VOF((u* + u^k)/2, phi^k, dt)
    R = momentum_rhs: the body force, and with inv_re > 0 the viscous term (mu_water = 1), with
    convect the convective term, each stage's R from that stage's velocity and volume fraction.
    Returns (u^{k+1}, phi^{k+1}, P)."""
    beta = face_coeffs(phi, solid, lam)
    R = momentum_rhs(phi, beta, u, h, g, inv_re, mu_air, 1.0, convect)
    ut = tuple(a + dt * r for a, r in zip(u, R))
    us = correct(beta, solve(beta, divergence(beta, ut, h, dt), h, tol=tol), ut, h, dt)
    phis = phi - vof_upwind(beta, u, phi, h, dt)
    beta2 = face_coeffs(phis, solid, lam)
    R2 = momentum_rhs(phis, beta2, us, h, g, inv_re, mu_air, 1.0, convect)
    ut2 = tuple((a + b) + dt * r for a, b, r in zip(us, u, R2))
    P = solve(beta2, divergence(beta2, ut2, h, dt), h, tol=tol)
    u1 = tuple(0.5 * x for x in correct(beta2, P, ut2, h, dt))
    uh = tuple(0.5 * (a + b) for a, b in zip(us, u))
    phi1 = phi - vof_upwind(beta, uh, phi, h, dt)
    return u1, phi1, P


# ---------------------------------------------------------------------------
# Independent second computations (NumPy / SciPy) used by the pins
# ---------------------------------------------------------------------------

def dense_solve(beta, b, h, labels=None, ncomp=None):
    """Minimum-norm solution of A p = b - per-component mean, by numpy.linalg.lstsq on the
    dense matrix built face by face in Python (independent of the C operator)."""
    nz, ny, nx = beta[0].shape
    n = nx * ny * nz
    A = np.zeros((n, n))
    idx = np.arange(n).reshape(nz, ny, nx)
    ih2 = 1.0 / (h * h)
    for axis, bb in zip((2, 1, 0), beta):
        sl_hi = [slice(None)] * 3
        sl_lo = [slice(None)] * 3
        sl_hi[axis] = slice(1, None)
        sl_lo[axis] = slice(None, -1)
        f = bb[tuple(sl_hi)].ravel()
        a = idx[tuple(sl_lo)].ravel()
        c = idx[tuple(sl_hi)].ravel()
        for fa, ia, ic in zip(f, a, c):
            if fa == 0.0:
                continue
            A[ia, ia] -= fa * ih2
            A[ic, ic] -= fa * ih2
            A[ia, ic] += fa * ih2
            A[ic, ia] += fa * ih2
    bb = b.ravel().copy()
    if labels is not None:
        lab = labels.ravel()
        for m in range(ncomp):
            sel = lab == m
            bb[sel] -= bb[sel].mean()
    x = np.linalg.lstsq(A, bb, rcond=1e-12)[0]
    return x.reshape(nz, ny, nx), A


def thomas_layered(bz_col, b_col, h):
    """1-D Neumann problem h^-2 [bz_{k+1}(p_{k+1}-p_k) - bz_k (p_k - p_{k-1})] = b_k solved by
    the Thomas algorithm with p_0 pinned to 0, then shifted to zero mean.  bz_col[0] is the wall."""
    nz = len(b_col)
    b = np.asarray(b_col, float) - np.mean(b_col)
    # unknowns p_1..p_{nz-1} with p_0 = 0; row k = 1..nz-1
    m = nz - 1
    lower = np.zeros(m)
    diag = np.zeros(m)
    upper = np.zeros(m)
    rhs = np.zeros(m)
    for r in range(m):
        k = r + 1
        lo = bz_col[k]
        hi = bz_col[k + 1] if k + 1 < nz else 0.0
        diag[r] = -(lo + hi)
        if r > 0:
            lower[r] = lo
        if k + 1 < nz:
            upper[r] = hi
        rhs[r] = h * h * b[k]
    # forward elimination
    cp = np.zeros(m)
    dp = np.zeros(m)
    cp[0] = upper[0] / diag[0]
    dp[0] = rhs[0] / diag[0]
    for r in range(1, m):
        den = diag[r] - lower[r] * cp[r - 1]
        cp[r] = upper[r] / den if r < m - 1 else 0.0
        dp[r] = (rhs[r] - lower[r] * dp[r - 1]) / den
    x = np.zeros(m)
    x[-1] = dp[-1]
    for r in range(m - 2, -1, -1):
        x[r] = dp[r] - cp[r] * x[r + 1]
    p = np.concatenate([[0.0], x])
    return p - p.mean()
