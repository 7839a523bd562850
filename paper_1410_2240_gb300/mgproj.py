"""ctypes binding of libmgproj.so (argument marshalling only).

Every function here forwards to the C ABI declared in ``include/mgproj.h`` with
the same name; all arithmetic runs in the library's CUDA kernels.  Tensors are
torch CUDA tensors (device memory and streams come from PyTorch): float64,
contiguous, shape (nz, ny, nx); face fields are 3-tuples of such tensors in the
low-face layout.  Importing this module loads the library and raises if it has
not been built (there is no fallback).  The environment variable MGPROJ_LIB names
another build of the same library to load instead (the bounds-check build,
build(check=True)).
"""
from __future__ import annotations

import ctypes
import os
import warnings
from typing import Optional, Sequence

import torch

from .build import LIB

MG_OK, MG_ERR_ARG, MG_ERR_CUDA, MG_ERR_NOT_CONVERGED, MG_ERR_NAN, MG_ERR_INCOMPATIBLE, MG_ERR_OOM = 0, 1, 2, 3, 4, 5, 6
MG_FP64, MG_MIXED = 0, 1

LIB_PATH = os.environ.get("MGPROJ_LIB", LIB)
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
                      "or `python -m paper_1410_2240_gb300.build`")
_lib = ctypes.CDLL(LIB_PATH)

_vp = ctypes.c_void_p
_P3 = _vp * 3
_PP = ctypes.POINTER(_vp)  # double *const x[3]; an _P3 instance or None


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double)]


class Bc(ctypes.Structure):
    _fields_ = [("wall", ctypes.c_int * 6)]


class Opts(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("max_cycles", ctypes.c_int),
                ("check_every", ctypes.c_int), ("coarse_max_cells", ctypes.c_int), ("prec", ctypes.c_int),
                ("inner_cycles", ctypes.c_int), ("profile", ctypes.c_int), ("smoother", ctypes.c_int),
                ("krylov", ctypes.c_int), ("coarse_graph", ctypes.c_int), ("coarse_tail", ctypes.c_int),
                ("precond", ctypes.c_int), ("pass_order", ctypes.c_int)]


class Forces(ctypes.Structure):
    """mg_forces: the terms of Eq. navi besides the pressure (body force, viscous, convective)."""
    _fields_ = [("g", ctypes.c_double), ("inv_re", ctypes.c_double), ("mu_air", ctypes.c_double),
                ("mu_water", ctypes.c_double), ("convection", ctypes.c_int)]


def forces(g=0.0, inv_re=0.0, mu_air=1.8e-2, mu_water=1.0, convection=False) -> Forces:
    return Forces(g, inv_re, mu_air, mu_water, 1 if convection else 0)


class Stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("rel_resid", ctypes.c_double), ("rhs_norm", ctypes.c_double),
                ("rhs_mean_removed", ctypes.c_double), ("resid_hist", ctypes.c_double * 256),
                ("ms_setup", ctypes.c_float), ("ms_solve", ctypes.c_float)]

    def as_dict(self):
        return {"cycles": self.cycles, "rel_resid": self.rel_resid, "rhs_norm": self.rhs_norm,
                "rhs_mean_removed": self.rhs_mean_removed,
                "resid_hist": list(self.resid_hist[: max(0, min(self.cycles, 256))]),
                "ms_setup": self.ms_setup, "ms_solve": self.ms_solve}


_lib.mg_default_opts.argtypes = [ctypes.POINTER(Opts)]
_lib.mg_last_error.restype = ctypes.c_char_p
_lib.mg_face_coeffs.argtypes = [ctypes.POINTER(Grid), _vp, _vp, ctypes.c_double, ctypes.c_double, _PP, _vp]
_lib.mg_setup.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(Grid), _PP, ctypes.POINTER(Bc), _vp,
                          ctypes.POINTER(Opts), _vp]
_lib.mg_solve.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.POINTER(Stats)]
_lib.mg_vcycle.argtypes = [_vp, _vp, _vp]
_lib.mg_divergence.argtypes = [_vp, _PP, ctypes.c_double, _vp]
_lib.mg_correct.argtypes = [_vp, _PP, _vp, ctypes.c_double, _PP]
_lib.mg_project.argtypes = [_vp, _PP, _PP, _vp, ctypes.c_double, ctypes.c_double, ctypes.POINTER(Stats)]
_lib.mg_project_adjoint.argtypes = [_vp, _PP, _vp, ctypes.c_double, ctypes.c_double, _PP, _PP, _vp,
                                    ctypes.POINTER(Stats)]
_lib.mg_phi_grad.argtypes = [ctypes.POINTER(Grid), _PP, _PP, ctypes.c_double, ctypes.c_double, _vp, _vp]
_lib.mg_num_levels.argtypes = [_vp]
_lib.mg_level_dims.argtypes = [_vp, ctypes.c_int, ctypes.c_int * 3]
_lib.mg_level_array.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp]
_lib.mg_update.argtypes = [_vp, _PP]
_lib.mg_face_areas.argtypes = [ctypes.POINTER(Grid), _vp, _PP, _vp]
_lib.mg_set_face_areas.argtypes = [_vp, _PP]
_lib.mg_set_body_velocity.argtypes = [_vp, _PP]
_lib.mg_rk2_step.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.POINTER(Forces),
                              ctypes.c_double, _PP, _vp, _vp, ctypes.c_double, ctypes.POINTER(Stats)]
_lib.mg_momentum_rhs.argtypes = [ctypes.POINTER(Grid), _vp, _PP, _PP, ctypes.POINTER(Forces), _PP, _vp, _vp]
_lib.mg_stretched_metrics.argtypes = [ctypes.POINTER(Grid), _vp, _vp, _vp, _PP, _PP, _PP, _PP, _vp]
_lib.mg_kernel_launches.restype = ctypes.c_uint64
_lib.mg_profile_read.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
_lib.mg_profile_reset.argtypes = [_vp]
_lib.mg_residual_norm_noalloc.argtypes = [ctypes.POINTER(Grid), _PP, _vp, _vp, _vp, _vp]
_lib.mg_destroy.argtypes = [_vp]
_lib.mg_check_read.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_uint64),
                               ctypes.POINTER(ctypes.c_uint64)]

PROF_SMOOTH, PROF_RESTRICT, PROF_PROLONG, PROF_RESID64, PROF_APPLY, PROF_KRYLOV, PROF_COARSE, PROF_UPDATE = range(8)


def check_read():
    """mg_check_read: (enabled, first record, count) of the bounds-check build since the last read;
    (False, 0, 0) from the normal build."""
    en, first, count = ctypes.c_int(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.mg_check_read(ctypes.byref(en), ctypes.byref(first), ctypes.byref(count)))
    return bool(en.value), int(first.value), int(count.value)


def kernel_launches() -> int:
    """mg_kernel_launches: kernels launched by the library so far in this process."""
    return int(_lib.mg_kernel_launches())

#: every symbol declared in include/mgproj.h
EXPORTS = ["mg_default_opts", "mg_face_coeffs", "mg_setup", "mg_update", "mg_solve", "mg_vcycle", "mg_divergence",
           "mg_correct", "mg_project", "mg_project_adjoint", "mg_phi_grad", "mg_num_levels", "mg_level_dims",
           "mg_level_array", "mg_kernel_launches", "mg_profile_read", "mg_profile_reset",
           "mg_residual_norm_noalloc", "mg_destroy", "mg_last_error", "mg_face_areas", "mg_set_face_areas",
           "mg_set_body_velocity", "mg_stretched_metrics", "mg_rk2_step", "mg_momentum_rhs", "mg_check_read"]


class MGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[mgproj status {code}] {msg}")
        self.code = code


class NotConverged(MGError):
    pass


class IncompatibleRhsWarning(UserWarning):
    """MG_ERR_INCOMPATIBLE: the solve converged after removing a rhs mean above the library's
    threshold on some fluid region; the results are those of the compatible rhs."""


def _check(code, allow_not_converged=False):
    if code == MG_OK:
        return code
    msg = _lib.mg_last_error().decode(errors="replace")
    if code == MG_ERR_INCOMPATIBLE:
        warnings.warn(f"[mgproj status {code}] {msg}", IncompatibleRhsWarning, stacklevel=3)
        return code
    if code == MG_ERR_NOT_CONVERGED:
        if allow_not_converged:
            return code
        raise NotConverged(code, msg)
    raise MGError(code, msg)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def _dev(t: torch.Tensor, shape, dtype=torch.float64, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with shape {tuple(shape)}, got {tuple(t.shape)}")
    if t.data_ptr() % 16:
        raise ValueError(f"{name} must start on a 16-byte boundary (a view offset into its storage does not)")
    return _vp(t.data_ptr())


def _faces(fs, shape, name):
    if len(fs) != 3:
        raise ValueError(f"{name} must be 3 face arrays")
    return _P3(*[_dev(f, shape, name=f"{name}[{a}]") for a, f in enumerate(fs)])


def default_opts(**kw) -> Opts:
    o = Opts()
    _lib.mg_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "prec" and isinstance(v, str):
            v = {"fp64": MG_FP64, "mixed": MG_MIXED}[v]
        setattr(o, k, v)
    return o


def face_coeffs(phi: torch.Tensor, h: float, solid: Optional[torch.Tensor] = None, rho_air: float = 1e-3,
                rho_water: float = 1.0, out=None, stream=None):
    """mg_face_coeffs: (bx, by, bz) from phi (and an optional uint8 solid mask)."""
    nz, ny, nx = phi.shape
    g = Grid(nx, ny, nz, h)
    if out is None:
        out = tuple(torch.empty_like(phi) for _ in range(3))
    sp = _vp(0) if solid is None else _dev(solid, phi.shape, torch.uint8, "solid")
    _check(_lib.mg_face_coeffs(ctypes.byref(g), _dev(phi, phi.shape, name="phi"), sp, rho_air, rho_water,
                               _faces(out, phi.shape, "beta_out"), _stream(stream)))
    return out


def face_areas(psi_nodes: torch.Tensor, h: float, out=None, stream=None):
    """mg_face_areas: open-area fractions (ax, ay, az) of the faces from psi at the grid nodes
    (shape (nz+1, ny+1, nx+1), psi > 0 outside the body)."""
    nz1, ny1, nx1 = psi_nodes.shape
    shape = (nz1 - 1, ny1 - 1, nx1 - 1)
    g = Grid(nx1 - 1, ny1 - 1, nz1 - 1, h)
    if out is None:
        out = tuple(torch.empty(shape, dtype=torch.float64, device=psi_nodes.device) for _ in range(3))
    _check(_lib.mg_face_areas(ctypes.byref(g), _dev(psi_nodes, psi_nodes.shape, name="psi_nodes"),
                              _faces(out, shape, "area_out"), _stream(stream)))
    return out


def stretched_metrics(hx: torch.Tensor, hy: torch.Tensor, hz: torch.Tensor, beta, frac=None, stream=None):
    """mg_stretched_metrics: (beta / centre distance, face widths * frac) of every low face for cell
    widths hx, hy, hz; a context on the first with h = 1 and the second as face areas solves the
    stretched problem."""
    shape = (hz.numel(), hy.numel(), hx.numel())
    g = Grid(shape[2], shape[1], shape[0], 1.0)
    bo = tuple(torch.empty(shape, dtype=torch.float64, device=hx.device) for _ in range(3))
    ao = tuple(torch.empty(shape, dtype=torch.float64, device=hx.device) for _ in range(3))
    _check(_lib.mg_stretched_metrics(ctypes.byref(g), _dev(hx, hx.shape, name="hx"), _dev(hy, hy.shape, name="hy"),
                                     _dev(hz, hz.shape, name="hz"), _faces(beta, shape, "beta"),
                                     None if frac is None else _faces(frac, shape, "frac"), _faces(bo, shape, "beta_out"),
                                     _faces(ao, shape, "area_out"), _stream(stream)))
    return bo, ao


def momentum_rhs(phi: torch.Tensor, beta: Sequence[torch.Tensor], u: Sequence[torch.Tensor], h: float,
                 f: Forces, out=None, work=None, stream=None):
    """mg_momentum_rhs: R_i of Eq. navi without the pressure (body force, viscous, convective) on
    the faces; beta = 1/rho on open faces (face_coeffs), 0 on closed ones.  work: scratch of
    12 * phi.numel() doubles (allocated when None)."""
    shape = phi.shape
    nz, ny, nx = shape
    g = Grid(nx, ny, nz, h)
    if out is None:
        out = tuple(torch.empty_like(phi) for _ in range(3))
    if work is None:
        work = torch.empty(12 * phi.numel(), dtype=torch.float64, device=phi.device)
    _check(_lib.mg_momentum_rhs(ctypes.byref(g), _dev(phi, shape, name="phi"), _faces(beta, shape, "beta"),
                                _faces(u, shape, "u"), ctypes.byref(f), _faces(out, shape, "R"),
                                _dev(work, (12 * phi.numel(),), name="work"), _stream(stream)))
    return out


def phi_grad(beta: Sequence[torch.Tensor], grad_beta: Sequence[torch.Tensor], h: float, rho_air=1e-3,
             rho_water=1.0, out=None, stream=None):
    """mg_phi_grad: chain rule from face coefficients to phi."""
    shape = beta[0].shape
    nz, ny, nx = shape
    g = Grid(nx, ny, nz, h)
    if out is None:
        out = torch.empty_like(beta[0])
    _check(_lib.mg_phi_grad(ctypes.byref(g), _faces(beta, shape, "beta"), _faces(grad_beta, shape, "grad_beta"),
                            rho_air, rho_water, _dev(out, shape, name="grad_phi"), _stream(stream)))
    return out


class Context:
    """An mg_ctx: the multigrid hierarchy for one set of face coefficients."""

    def __init__(self, beta: Sequence[torch.Tensor], h: float, solid: Optional[torch.Tensor] = None,
                 opts: Optional[Opts] = None, stream=None, **kw):
        self.shape = tuple(beta[0].shape)
        nz, ny, nx = self.shape
        self.h = h
        self.grid = Grid(nx, ny, nz, h)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.opts = opts if opts is not None else default_opts(**kw)
        self._c = _vp()
        sp = _vp(0) if solid is None else _dev(solid, self.shape, torch.uint8, "solid")
        _check(_lib.mg_setup(ctypes.byref(self._c), ctypes.byref(self.grid), _faces(beta, self.shape, "beta"), None,
                             sp, ctypes.byref(self.opts), _stream(self.stream)))
        self.last_stats = Stats()

    def close(self):
        if self._c:
            _lib.mg_destroy(self._c)
            self._c = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, beta):
        """mg_update: rebuild the hierarchy for new face coefficients (same grid, no allocation)."""
        _check(_lib.mg_update(self._c, _faces(beta, self.shape, "beta")))

    def set_face_areas(self, areas):
        """mg_set_face_areas: fractional open areas of the faces (None: whole faces); the face
        coefficients of this context are then 1/rho and the operator uses area * 1/rho."""
        _check(_lib.mg_set_face_areas(self._c, None if areas is None else _faces(areas, self.shape, "area")))

    def rk2_step(self, phi, u, dt, g=0.0, solid=None, rho_air=1e-3, rho_water=1.0, tol=1e-10, phi_out=None, p=None,
                 forces: Optional[Forces] = None):
        """mg_rk2_step: one Runge-Kutta step (u updated in place); returns (phi_new, p, stats).
        forces: an mg_forces (viscous and convective terms); None: the body force g alone."""
        if phi_out is None:
            phi_out = torch.empty_like(phi)
        if p is None:
            p = torch.empty_like(phi)
        f = forces if forces is not None else Forces(g, 0.0, 0.0, 1.0, 0)
        st = Stats()
        sp = _vp(0) if solid is None else _dev(solid, self.shape, torch.uint8, "solid")
        _check(_lib.mg_rk2_step(self._c, _dev(phi, self.shape, name="phi"), sp, rho_air, rho_water, ctypes.byref(f),
                                dt, _faces(u, self.shape, "u"), _dev(phi_out, self.shape, name="phi_out"),
                                _dev(p, self.shape, name="p"), tol, ctypes.byref(st)))
        return phi_out, p, st

    def set_body_velocity(self, v):
        """mg_set_body_velocity: the body velocity on the faces (None: a static body)."""
        _check(_lib.mg_set_body_velocity(self._c, None if v is None else _faces(v, self.shape, "v")))

    def profile_read(self, group):
        n = ctypes.c_int()
        ms = ctypes.c_double()
        _check(_lib.mg_profile_read(self._c, group, ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def profile_reset(self):
        _lib.mg_profile_reset(self._c)

    @property
    def num_levels(self):
        return _lib.mg_num_levels(self._c)

    def level_dims(self, level):
        d = (ctypes.c_int * 3)()
        _check(_lib.mg_level_dims(self._c, level, d))
        return tuple(d)

    def level_array(self, level, which):
        nx, ny, nz = self.level_dims(level)
        out = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")
        _check(_lib.mg_level_array(self._c, level, which, _vp(out.data_ptr())))
        return out

    def solve(self, rhs, p=None, tol=1e-10, allow_not_converged=False):
        if p is None:
            p = torch.zeros_like(rhs)
        st = Stats()
        code = _check(_lib.mg_solve(self._c, _dev(rhs, self.shape, name="rhs"), _dev(p, self.shape, name="p"), tol,
                                    ctypes.byref(st)), allow_not_converged)
        self.last_stats = st
        return p, st

    def vcycle(self, rhs, p):
        _check(_lib.mg_vcycle(self._c, _dev(rhs, self.shape, name="rhs"), _dev(p, self.shape, name="p")))
        return p

    def divergence(self, u, dt=1.0, out=None):
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        _check(_lib.mg_divergence(self._c, _faces(u, self.shape, "u"), dt, _dev(out, self.shape, name="rhs")))
        return out

    def correct(self, u_star, p, dt=1.0, out=None):
        if out is None:
            out = tuple(torch.empty_like(x) for x in u_star)
        _check(_lib.mg_correct(self._c, _faces(u_star, self.shape, "u_star"), _dev(p, self.shape, name="p"), dt,
                               _faces(out, self.shape, "u")))
        return out

    def project(self, u_star, p=None, dt=1.0, tol=1e-10, out=None, allow_not_converged=False):
        if p is None:
            p = torch.zeros(self.shape, dtype=torch.float64, device="cuda")
        if out is None:
            out = tuple(torch.empty_like(x) for x in u_star)
        st = Stats()
        _check(_lib.mg_project(self._c, _faces(u_star, self.shape, "u_star"), _faces(out, self.shape, "u"),
                               _dev(p, self.shape, name="p"), dt, tol, ctypes.byref(st)), allow_not_converged)
        self.last_stats = st
        return out, p, st

    def project_adjoint(self, w, p, dt=1.0, tol=1e-10, grad_u=None, grad_beta=None, want_grad_beta=True, q=None,
                        allow_not_converged=False):
        if grad_u is None:
            grad_u = tuple(torch.empty_like(x) for x in w)
        if want_grad_beta and grad_beta is None:
            grad_beta = tuple(torch.empty_like(x) for x in w)
        gb = _faces(grad_beta, self.shape, "grad_beta") if grad_beta is not None else None
        qp = _dev(q, self.shape, name="q") if q is not None else _vp(0)
        st = Stats()
        _check(_lib.mg_project_adjoint(self._c, _faces(w, self.shape, "w"), _dev(p, self.shape, name="p"), dt, tol,
                                       _faces(grad_u, self.shape, "grad_u"), gb, qp, ctypes.byref(st)),
               allow_not_converged)
        self.last_stats = st
        return grad_u, grad_beta, st
