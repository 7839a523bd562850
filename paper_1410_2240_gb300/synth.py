"""Seeded synthetic inputs for the variable-density pressure projection.

This module only *generates inputs*: volume fractions phi, solid masks, predicted
face velocities u*, right-hand sides and loss weights.  It holds none of the
method's arithmetic (no face coefficients, no divergence, no solver), so both the
CUDA path and the CPU oracle may draw their inputs from it.

Layout (shared by every array here): C order ``[k][j][i]`` with x fastest, shape
``(nz, ny, nx)``, cell centres at ``((i+1/2)h, (j+1/2)h, (k+1/2)h)``.  A face
array ``u_x[k][j][i]`` holds the x-face between cells ``(i-1,j,k)`` and
``(i,j,k)``; index ``i = 0`` is the low wall and the high wall face is not stored
(always closed).  Likewise for y and z.

The workloads stand in for the paper's towed-ship runs (Results section: a
Cartesian tow-tank grid of order 10^7 cells, air/water density ratio of order
1e-3, a hull that pierces the free surface, breaking waves and entrained air).
The paper's hull geometry and measured data are not available, so analytic
interfaces, analytic solids and seeded random fields take their place.  All
random numbers come from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

DENSITY_RATIO = 1.0e-3  # lambda = rho_air / rho_water (Eq. density)


@dataclasses.dataclass
class Case:
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    phi: np.ndarray                  # f64 (nz, ny, nx), water volume fraction in [0, 1]
    solid: Optional[np.ndarray]      # u8 (nz, ny, nx), 1 = cell centre inside the body
    rhs: Optional[np.ndarray] = None  # f64 (nz, ny, nx), raw right-hand side (mean NOT removed)
    u_star: Optional[tuple] = None   # 3 face arrays (ux, uy, uz), same shape as phi
    w: Optional[tuple] = None        # 3 face arrays of loss weights
    dt: float = 1.0
    lam: float = DENSITY_RATIO
    note: str = ""

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def centres(n: int, h: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def tanh_profile(s: np.ndarray, h: float) -> np.ndarray:
    """Water fraction 1/2 (1 - tanh(s / 1.5h)); s > 0 in air (smoothed over 1.5 cells)."""
    return 0.5 * (1.0 - np.tanh(s / (1.5 * h)))


def closed_face_masks(solid: Optional[np.ndarray], shape) -> tuple:
    """Boolean masks of faces that carry no flux: walls and faces touching a solid.

    This is input *structure* (which faces exist), used to put u* = 0 there.
    """
    nz, ny, nx = shape
    cx = np.zeros(shape, bool)
    cy = np.zeros(shape, bool)
    cz = np.zeros(shape, bool)
    cx[:, :, 0] = True
    cy[:, 0, :] = True
    cz[0, :, :] = True
    if solid is not None:
        s = solid.astype(bool)
        cx[:, :, 1:] |= s[:, :, 1:] | s[:, :, :-1]
        cx[:, :, 0] = True
        cy[:, 1:, :] |= s[:, 1:, :] | s[:, :-1, :]
        cz[1:, :, :] |= s[1:, :, :] | s[:-1, :, :]
    return cx, cy, cz


def random_face_field(rng, shape, sigma, solid, dtype=np.float64) -> tuple:
    """Three face arrays ~ N(0, sigma) drawn in order x, y, z; zero on closed faces."""
    out = []
    for closed in closed_face_masks(solid, shape):
        a = rng.standard_normal(size=shape, dtype=np.float64 if dtype == np.float64 else np.float32)
        a *= sigma
        a[closed] = 0
        out.append(np.ascontiguousarray(a.astype(dtype, copy=False)))
    return tuple(out)


def random_modes(rng: np.random.Generator, nmodes: int = 4):
    """Wavenumber pairs (m, n_m), n_m uniform in {-m..m}, and phases U[0, 2pi)."""
    ns = [int(rng.integers(-m, m + 1)) for m in range(1, nmodes + 1)]
    theta = rng.uniform(0.0, 2.0 * math.pi, size=nmodes)
    return ns, theta


def mode_sum(x: np.ndarray, y: np.ndarray, ns, theta) -> np.ndarray:
    """S(x, y) = sum_m cos(2 pi (m x + n_m y) + theta_m), m = 1..4."""
    s = np.zeros(np.broadcast(x, y).shape)
    for m, (n, th) in enumerate(zip(ns, theta), start=1):
        s += np.cos(2.0 * math.pi * (m * x + n * y) + th)
    return s


def ellipsoid_mask(nx, ny, nz, h, centre=(0.5, 0.5, 0.5), semi=(0.3, 0.06, 0.05)) -> np.ndarray:
    x = centres(nx, h)[None, None, :]
    y = centres(ny, h)[None, :, None]
    z = centres(nz, h)[:, None, None]
    q = ((x - centre[0]) / semi[0]) ** 2 + ((y - centre[1]) / semi[1]) ** 2 + ((z - centre[2]) / semi[2]) ** 2
    return np.ascontiguousarray((q <= 1.0).astype(np.uint8))


def stretched_widths(n: int, ratio: float = 3.5, finest: float = 0.5) -> np.ndarray:
    """Cell widths of an axis of unit length stretched smoothly: the narrowest cells at `finest`,
    the widest a factor `ratio` wider (the spread of the paper's grid, 0.002 to 0.007)."""
    t = (np.arange(n) + 0.5) / n
    w = 1.0 + (ratio - 1.0) * (0.5 - 0.5 * np.cos(2 * np.pi * (t - finest + 0.5)))
    return np.ascontiguousarray(w / w.sum())


def ellipsoid_psi_nodes(nx, ny, nz, h, centre=(0.5, 0.5, 0.5), semi=(0.3, 0.06, 0.05)) -> np.ndarray:
    """Level-set of the same ellipsoid at the grid nodes ((nz+1, ny+1, nx+1), node (i,j,k) at
    (i h, j h, k h)): > 0 outside, < 0 inside, (sqrt(q) - 1) * min(semi) (the distance to the surface
    near it, up to the ellipsoid's aspect)."""
    x = (np.arange(nx + 1) * h)[None, None, :]
    y = (np.arange(ny + 1) * h)[None, :, None]
    z = (np.arange(nz + 1) * h)[:, None, None]
    q = ((x - centre[0]) / semi[0]) ** 2 + ((y - centre[1]) / semi[1]) ** 2 + ((z - centre[2]) / semi[2]) ** 2
    return np.ascontiguousarray((np.sqrt(q) - 1.0) * min(semi))


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def case_c1(n: int = 32, seed: int = 1) -> Case:
    """32^3 unit cube, gently waved interface, no solid, rhs ~ N(0,1) i.i.d."""
    h = 1.0 / n
    x = centres(n, h)[None, None, :]
    y = centres(n, h)[None, :, None]
    z = centres(n, h)[:, None, None]
    s = z - (0.5 + 0.05 * np.sin(2 * math.pi * x) * np.cos(2 * math.pi * y))
    phi = np.ascontiguousarray(tanh_profile(s, h))
    rng = _rng(seed)
    rhs = rng.standard_normal(size=(n, n, n))
    return Case("c1", n, n, n, h, phi, None, rhs=rhs,
                note=f"{n}^3 unit cube, z=0.5+0.05 sin(2pi x)cos(2pi y), no solid, rhs~N(0,1) seed {seed}")


def _waved_ellipsoid_phi(n: int, geom_seed: int):
    h = 1.0 / n
    rng = _rng(geom_seed)
    ns, theta = random_modes(rng)
    x = centres(n, h)
    y = centres(n, h)
    S = mode_sum(x[None, :], y[:, None], ns, theta)  # (ny, nx)
    eta = 0.5 + 0.08 * S / np.max(np.abs(S))
    z = centres(n, h)[:, None, None]
    phi = np.ascontiguousarray(tanh_profile(z - eta[None, :, :], h))
    solid = ellipsoid_mask(n, n, n, h)
    return h, phi, solid


def case_c2(n: int = 128, geom_seed: int = 2, field_seed: int = 2) -> Case:
    """128^3, 4 random-phase modes (amplitude 0.08), piercing ellipsoid, u* ~ N(0, 0.1)."""
    h, phi, solid = _waved_ellipsoid_phi(n, geom_seed)
    rng = _rng(field_seed)
    u = random_face_field(rng, phi.shape, 0.1, solid)
    w = random_face_field(rng, phi.shape, 1.0, solid)
    return Case(f"c2_{n}", n, n, n, h, phi, solid, u_star=u, w=w,
                note=f"{n}^3, 4-mode interface (seed {geom_seed}), ellipsoid (0.3,0.06,0.05), u*~N(0,0.1) seed {field_seed}")


def case_c3(n: int = 256) -> Case:
    """256^3, same geometry as the 128^3 case (geometry seed 2), u* seed 3."""
    c = case_c2(n, geom_seed=2, field_seed=3)
    c.name = f"c3_{n}"
    return c


def _bubbles(rng, nb, h, L, eta_fn):
    out = []
    while len(out) < nb:
        r = rng.uniform(2 * h, 6 * h)
        m = r + 2 * h
        c = np.array([rng.uniform(m, L[0] - m), rng.uniform(m, L[1] - m), rng.uniform(m, L[2] - m)])
        if c[2] <= eta_fn(c[0], c[1]) - m:
            out.append((c, r))
    return out


def case_c4(nx: int = 512, ny: int = 256, nz: int = 128, seed: int = 4, nbubbles: int = 200) -> Case:
    """Tow-tank box [0,4]x[0,2]x[0,1] at h=1/128 (16.8 M cells): flat surface + 200 air bubbles."""
    h = 1.0 / nz
    L = (nx * h, ny * h, nz * h)
    rng = _rng(seed)
    ns, theta = random_modes(rng)
    x = centres(nx, h)
    y = centres(ny, h)
    S = mode_sum(x[None, :], y[:, None], ns, theta)
    smax = np.max(np.abs(S))
    eta = 0.5 + 0.01 * S / smax

    def eta_fn(px, py):
        return 0.5 + 0.01 * mode_sum(np.array(px), np.array(py), ns, theta) / smax

    z = centres(nz, h)
    phi = tanh_profile(z[:, None, None] - eta[None, :, :], h)
    bubbles = _bubbles(rng, nbubbles, h, L, eta_fn)
    # each bubble's profile is applied inside a box of half-width r + 12h about its centre
    for c, r in bubbles:
        half = r + 12 * h
        lo = [max(0, int(math.floor((c[d] - half) / h))) for d in range(3)]
        hi = [min(n, int(math.ceil((c[d] + half) / h)) + 1) for d, n in enumerate((nx, ny, nz))]
        xs = centres(nx, h)[lo[0]:hi[0]]
        ys = centres(ny, h)[lo[1]:hi[1]]
        zs = centres(nz, h)[lo[2]:hi[2]]
        d = np.sqrt((xs[None, None, :] - c[0]) ** 2 + (ys[None, :, None] - c[1]) ** 2 + (zs[:, None, None] - c[2]) ** 2)
        pb = 0.5 * (1.0 + np.tanh((d - r) / (1.5 * h)))
        sub = phi[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        np.minimum(sub, pb, out=sub)
    phi = np.ascontiguousarray(phi)
    u = random_face_field(rng, phi.shape, 0.1, None)
    w = random_face_field(rng, phi.shape, 1.0, None)
    c = Case(f"c4_{nx}x{ny}x{nz}", nx, ny, nz, h, phi, None, u_star=u, w=w,
             note=f"{nx}x{ny}x{nz} box h=1/{nz}, surface 0.5+0.01 S, {nbubbles} bubbles r~U[2h,6h], seed {seed}")
    c.bubbles = bubbles
    c.eta = eta
    return c


def hull_mask(nx, ny, nz, h) -> np.ndarray:
    """Box hull x in [1.0,1.4], y in [0.975,1.025], z in [0.48,0.52]; bow (x > 1.375) rounded
    to a half-disc of radius 0.025 in plan."""
    x = centres(nx, h)[None, None, :]
    y = centres(ny, h)[None, :, None]
    z = centres(nz, h)[:, None, None]
    inbox = (x >= 1.0) & (x <= 1.4) & (y >= 0.975) & (y <= 1.025) & (z >= 0.48) & (z <= 0.52)
    bow = x > 1.375
    round_ok = (x - 1.375) ** 2 + (y - 1.0) ** 2 <= 0.025 ** 2
    m = inbox & (~bow | round_ok)
    return np.ascontiguousarray(m.astype(np.uint8))


def case_c5(nx: int = 1024, ny: int = 512, nz: int = 256, seed: int = 5) -> Case:
    """Plunging-wave-like overturned interface plus a box hull with a rounded bow.

    Fields are FP32 (u*, w) as in the large mixed-precision configuration."""
    h = 1.0 / nz
    rng = _rng(seed)
    theta = rng.uniform(0.0, 2.0 * math.pi)
    x = centres(nx, h)[None, None, :]
    y = centres(ny, h)[None, :, None]
    z = centres(nz, h)[:, None, None]
    zeta = z - 0.5
    xi = x - 2.5 - 40.0 * zeta ** 3
    s = zeta - 0.15 * (1.0 + 0.2 * np.cos(math.pi * y + theta)) * np.exp(-(xi / 0.12) ** 2)
    phi = np.ascontiguousarray(tanh_profile(s, h))
    del s, xi, zeta
    solid = hull_mask(nx, ny, nz, h)
    u = random_face_field(rng, phi.shape, 0.1, solid, dtype=np.float32)
    w = random_face_field(rng, phi.shape, 1.0, solid, dtype=np.float32)
    return Case(f"c5_{nx}x{ny}x{nz}", nx, ny, nz, h, phi, solid, u_star=u, w=w,
                note=f"{nx}x{ny}x{nz} plunging interface, hull box with rounded bow, seed {seed}")


def overturned_columns(phi: np.ndarray) -> int:
    """Number of (x, y) columns in which phi is not monotone non-increasing in z."""
    d = np.diff(phi, axis=0)
    return int(np.count_nonzero(np.any(d > 1e-6, axis=0)))


# ---------------------------------------------------------------------------
# Small cases for tests
# ---------------------------------------------------------------------------

def small_case(nx: int, ny: int = None, nz: int = None, seed: int = 0, solid: str = "none",
               interface: str = "wave", ratio: float = DENSITY_RATIO, fields: bool = True) -> Case:
    """A small test grid on [0, nx h] x [0, ny h] x [0, nz h] with h = 1/nx.

    interface: "wave" (tanh-smoothed waved plane at mid-depth), "flat" (phi = phi(z)),
    "none" (phi = 1), or "random" (phi ~ U[0,1] i.i.d.).
    solid: "none", "ellipsoid" (centred, semi-axes (0.3, 0.18, 0.15) x extent) or
    "wall" (a solid slab splitting the domain into two chambers in x).
    """
    ny = ny or nx
    nz = nz or nx
    h = 1.0 / nx
    rng = _rng(seed)
    x = centres(nx, h)[None, None, :]
    y = centres(ny, h)[None, :, None]
    z = centres(nz, h)[:, None, None]
    Lz = nz * h
    if interface == "wave":
        s = z - (0.5 * Lz + 0.1 * Lz * np.sin(2 * math.pi * x) * np.cos(2 * math.pi * y * nx / ny))
        phi = tanh_profile(s + 0 * x * y, h)
    elif interface == "flat":
        phi = tanh_profile(z - 0.5 * Lz + 0 * x * y, h)
    elif interface == "none":
        phi = np.ones((nz, ny, nx))
    elif interface == "random":
        phi = rng.uniform(0.0, 1.0, size=(nz, ny, nx))
    else:
        raise ValueError(interface)
    phi = np.ascontiguousarray(np.broadcast_to(phi, (nz, ny, nx)).astype(np.float64))
    if solid == "none":
        sm = None
    elif solid == "ellipsoid":
        Lx, Ly = nx * h, ny * h
        q = ((x - 0.5 * Lx) / (0.3 * Lx)) ** 2 + ((y - 0.5 * Ly) / (0.18 * Ly)) ** 2 + ((z - 0.5 * Lz) / (0.15 * Lz)) ** 2
        sm = np.ascontiguousarray((q <= 1.0).astype(np.uint8))
    elif solid == "wall":
        sm = np.zeros((nz, ny, nx), np.uint8)
        sm[:, :, nx // 2] = 1
    else:
        raise ValueError(solid)
    rhs = rng.standard_normal(size=(nz, ny, nx))
    u = w = None
    if fields:
        u = random_face_field(rng, (nz, ny, nx), 0.1, sm)
        w = random_face_field(rng, (nz, ny, nx), 1.0, sm)
    return Case(f"small_{nx}x{ny}x{nz}_{interface}_{solid}", nx, ny, nz, h, phi, sm,
                rhs=rhs, u_star=u, w=w, lam=ratio)


def fourier_mode(nx, ny, nz, kx, ky, kz) -> np.ndarray:
    """prod_d cos(pi k_d (i_d + 1/2) / n_d): a cell-centred cosine on the Neumann box."""
    cx = np.cos(math.pi * kx * (np.arange(nx) + 0.5) / nx)
    cy = np.cos(math.pi * ky * (np.arange(ny) + 0.5) / ny)
    cz = np.cos(math.pi * kz * (np.arange(nz) + 0.5) / nz)
    return np.ascontiguousarray(cz[:, None, None] * cy[None, :, None] * cx[None, None, :])


def crop(case: Case, centre_ijk, n: int = 32) -> Case:
    """An n^3 sub-box of a case, used as its own closed (Neumann) box."""
    i0 = [min(max(0, c - n // 2), N - n) for c, N in zip(centre_ijk, (case.nx, case.ny, case.nz))]
    sl = (slice(i0[2], i0[2] + n), slice(i0[1], i0[1] + n), slice(i0[0], i0[0] + n))
    phi = np.ascontiguousarray(case.phi[sl])
    solid = None if case.solid is None else np.ascontiguousarray(case.solid[sl])
    closed = closed_face_masks(solid, phi.shape)
    def cut(fs):
        if fs is None:
            return None
        out = []
        for a, cl in zip(fs, closed):
            b = np.array(a[sl], dtype=np.float64)
            b[cl] = 0
            out.append(np.ascontiguousarray(b))
        return tuple(out)
    return Case(case.name + f"_crop{n}", n, n, n, case.h, phi, solid, u_star=cut(case.u_star),
                w=cut(case.w), dt=case.dt, lam=case.lam, note=f"crop at {i0}")
