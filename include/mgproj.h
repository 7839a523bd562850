/*
 * mgproj.h -- C ABI of the GB300 (sm_103a) variable-density pressure projection.
 *
 * The library solves, on one GPU, the pressure Poisson problem of the paper's
 * time integrator (Eq. poisson1 / Eq. poisson2) in the finite-volume form of
 * Eq. integral2 on a uniform Cartesian MAC grid,
 *
 *     (A p)_c = h^-2 * sum_{open faces f of c} beta_f (p_nb - p_c) = b_c ,
 *
 * with face coefficients beta_f = area_f / rho_f (the product of one over the
 * density and the cut-surface area that the Poisson-solver section moves to
 * the coarse grids as one unit), and applies the velocity correction of
 * Eq. runge1, u = u* - dt beta grad p.  The solver is geometric multigrid
 * (red-black Gauss-Seidel, face-coefficient restriction, cell-centred
 * restriction and trilinear prolongation, exact coarsest-grid solve) in FP64,
 * or FP32 V-cycles inside FP64 iterative refinement.
 *
 * Layout of every field: C order [k][j][i], x fastest, nx*ny*nz entries.
 * Face arrays use the low-face convention: bx[k][j][i] / ux[k][j][i] belong to
 * the x-face between cells (i-1,j,k) and (i,j,k); entries with i = 0 are the
 * low wall; the high wall face is not stored.  Likewise for y (index j) and z
 * (index k).  Walls are closed (homogeneous Neumann, Eq. neumann with a wall
 * velocity of 0); a face that touches a solid cell is closed (binary cut
 * cells, area 0, static body).
 *
 * Pointers: every array argument is a DEVICE pointer (cudaMalloc'd or from a
 * caching allocator) unless marked "host", and starts on a 16-byte boundary
 * (every cudaMalloc and PyTorch allocation does; a view offset by an odd
 * number of doubles does not): the kernels move aligned pairs, and a call
 * given an unaligned array returns MG_ERR_ARG.  The caller owns every buffer it
 * passes; the library never frees or retains them beyond the call, except as
 * stated for mg_setup.  All work is ordered on the CUDA stream given to
 * mg_setup (or to the stand-alone calls); pass NULL for the legacy default
 * stream.  Calls that return a convergence result synchronise with that
 * stream once per residual check (a 16-byte device-to-host read).
 *
 * Errors: every function returns an mg_status; on failure mg_last_error()
 * gives a message (thread-local, valid until the next call on that thread).
 * No function aborts, traps or prints.
 */
#ifndef MGPROJ_H
#define MGPROJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MG_OK = 0,
    MG_ERR_ARG = 1,            /* bad argument (null pointer, size, option) */
    MG_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    MG_ERR_NOT_CONVERGED = 3,  /* max_cycles reached; p and stats hold the last iterate */
    MG_ERR_NAN = 4,            /* a residual norm was not finite */
    MG_ERR_INCOMPATIBLE = 5,   /* the solve converged, but its rhs was incompatible with the Neumann
                                  problem: on some connected fluid region |mean of the rhs| exceeded
                                  1e-8 x the RMS of the rhs over all fluid cells (both before the
                                  means were removed); each region's mean was removed and p, u and
                                  stats are those of that compatible rhs */
    MG_ERR_OOM = 6             /* device allocation failed */
} mg_status;

/* Grid: cells per axis and the isotropic spacing h. */
typedef struct {
    int nx, ny, nz;
    double h;
} mg_grid;

/* Wall conditions.  Only homogeneous Neumann (closed walls, the no-flux
 * condition of Eq. neumann with zero wall velocity) is implemented. */
typedef enum { MG_BC_NEUMANN = 0 } mg_bc_kind;
typedef struct {
    mg_bc_kind wall[6]; /* -x, +x, -y, +y, -z, +z */
} mg_bc;

typedef enum { MG_FP64 = 0, MG_MIXED = 1 } mg_precision;

/* Solver options; mg_default_opts fills the defaults given in brackets. */
typedef struct {
    int nu1;              /* pre-smoothing red-black sweeps per level [2] */
    int nu2;              /* post-smoothing sweeps, colours reversed [2] */
    int max_cycles;       /* cycle (or refinement-step) limit [100] */
    int check_every;      /* residual check every this many cycles [1] */
    int coarse_max_cells; /* largest coarsest grid solved densely [512] */
    mg_precision prec;    /* MG_FP64 or MG_MIXED [MG_FP64] */
    int inner_cycles;     /* V-cycles per preconditioner application (krylov = 1) or, with
                             krylov = 0 and MG_MIXED, FP32 V-cycles per FP64 refinement step [1] */
    int profile;          /* nonzero: time finest-grid kernels with CUDA events (mg_profile_read) [0] */
    int smoother;         /* red-black sweep kernels; every choice gives bit-identical results:
                             0 auto (currently 1, the fastest measured on GB300); 1 one pass per
                             colour; 2 one fused pass per sweep with register-staged planes on
                             levels of >= 32 x 8 x 8 cells (both precisions); 3 one fused pass per
                             sweep with TMA-staged planes on FP32 levels of >= 32 x 8 x 8 cells
                             with nx % 4 == 0, one pass per colour elsewhere [0] */
    int krylov;           /* 0: stationary V-cycles (refinement steps when mixed); 1: conjugate
                             gradients preconditioned by inner_cycles V-cycles from a zero guess
                             (flexible Polak-Ribiere form; FP64 Krylov vectors, the cycles in the
                             precision prec selects).  The conjugate gradients stop at a true
                             relative residual of 0.4 tol, not tol, so that their solution error
                             stays below 10 tol: on the 128^3, 256^3 and 512x256x128 workloads the
                             error of a CG iterate is 4 to 23 times its relative residual [0] */
    int coarse_graph;     /* 1: replay the coarse-grid part of each V-cycle (all levels below the
                             finest) as one CUDA graph captured on first use on a private stream;
                             0: launch its kernels one by one.  Identical results [1] */
    int coarse_tail;      /* 1: the smallest levels below the finest (each field of at most a few
                             thousand cells) are smoothed, restricted and prolonged by one CTA in
                             two launches around the coarsest solve instead of a launch per pass;
                             0: a launch per pass.  Identical results [1] */
    int precond;          /* preconditioner of the conjugate gradients (krylov = 1): 0 inner_cycles
                             multigrid V-cycles; 1 Jacobi (the inverse diagonal, z = D^-1 r; MG_FP64
                             only), the diagonally preconditioned CG the Poisson-solver section
                             compares multigrid with [0] */
    int pass_order;       /* plane order of the finest level's FP32 colour passes (colour-split
                             layout): 1 alternate descending and ascending passes, so that each
                             starts on the planes the previous kernel touched last, still in L2,
                             and run the restriction after them descending; 0 every pass
                             ascending.  Each colour pass updates cells that do not depend on one
                             another, so the results are identical [1] */
} mg_opts;

/* Solve statistics (host struct, filled when non-NULL). */
typedef struct {
    int cycles;              /* V-cycles (FP64), refinement steps (mixed) or CG iterations (krylov) */
    double rel_resid;        /* final ||b - A p||_2 / ||b||_2 over fluid cells, FP64 */
    double rhs_norm;         /* ||b||_2 after compatibility projection */
    double rhs_mean_removed; /* mean of the rhs over all fluid cells (with one connected fluid region,
                                the value subtracted; with several, each region's own mean is) */
    double resid_hist[256];  /* relative residual after each checked cycle */
    float ms_setup;          /* mg_setup wall time of this context (ms, host clock) */
    float ms_solve;          /* last solve's time (ms, CUDA events on the stream) */
} mg_stats;

typedef struct mg_ctx mg_ctx; /* opaque, owned by the library */

/* Fill *o with the defaults listed in mg_opts. */
void mg_default_opts(mg_opts *o);

/*
 * Face coefficients from the volume fraction (Eq. density with H(phi) = phi;
 * Poisson-solver section, face product (1/rho)*area on the finest grid):
 *   rho_c = rho_air + (rho_water - rho_air) * phi_c
 *   beta_f = 2 / (rho_L + rho_R)   (harmonic mean of 1/rho)   on open faces
 *   beta_f = 0 on walls and on faces touching a solid cell.
 * phi: device, nx*ny*nz doubles.  solid_mask: device, nx*ny*nz bytes, 1 =
 * solid, or NULL (no body).  beta_out[0..2]: device, nx*ny*nz doubles each
 * (x, y, z low-face layout), written.  Stream-ordered on `stream`.
 * Returns MG_OK, MG_ERR_ARG (bad grid, null or unaligned array, rho_air or
 * rho_water not > 0) or MG_ERR_CUDA (the launch failed).
 */
int mg_face_coeffs(const mg_grid *g, const double *phi, const uint8_t *solid_mask, double rho_air,
                   double rho_water, double *const beta_out[3], void *stream);

/*
 * Build the multigrid hierarchy (Poisson-solver section): copy the fine face
 * coefficients, restrict them face-wise to every coarser grid (mean of the 2x2
 * coplanar fine faces), form the inverse diagonals, the FP32 copies when
 * opt->prec == MG_MIXED, and the dense minimum-norm inverse of the coarsest
 * grid's operator (computed on the host in FP64).  Levels halve every axis
 * while all three are even and >= 8; the coarsest grid must then have at most
 * opt->coarse_max_cells cells (MG_ERR_ARG otherwise).
 * face_coeffs[0..2]: device, nx*ny*nz doubles each, copied (a later change of
 * phi needs a new mg_setup).  bc: host, NULL = all Neumann.  solid_mask: device
 * or NULL; it is implied by the zero faces and used only for validation.
 * opt: host or NULL (defaults).  stream: cudaStream_t or NULL.  The context
 * owns all its device memory (about 5.3 x the fine face arrays in FP64 plus,
 * when mixed, 2.4 x in FP32) until mg_destroy.  The fluid cells with at least
 * one open face may form several connected regions (e.g. sealed pockets): each
 * hierarchy build labels them on the GPU (union-find over runs of x-joined
 * cells), and every solve removes the rhs mean and pins p to zero mean on each
 * region separately, the minimum-norm solution of the singular Neumann
 * problem; at most 65536 regions (MG_ERR_ARG beyond).  Cells with no open face
 * hold p = 0.  Every reduction is summed in a fixed order (bitwise
 * reproducible) for up to 64 regions; beyond that the per-region sums use
 * atomics and may round differently from run to run.
 */
int mg_setup(mg_ctx **out, const mg_grid *g, const double *const face_coeffs[3], const mg_bc *bc,
             const uint8_t *solid_mask, const mg_opts *opt, void *stream);

/*
 * Rebuild the hierarchy of an existing context for new fine face coefficients
 * on the same grid (same work as mg_setup, no allocation): restriction,
 * inverse diagonals, FP32 copies and the coarsest dense inverse.  face_coeffs:
 * device, copied.  Synchronises with the context's stream once (the coarsest
 * operator, at most coarse_max_cells cells, is inverted on the host).
 * Returns MG_OK, MG_ERR_ARG (null context or array, unaligned array) or
 * MG_ERR_CUDA.
 */
int mg_update(mg_ctx *c, const double *const face_coeffs[3]);

/*
 * Open-area fractions of the faces from a body given by a signed distance psi
 * (Body Boundary Conditions section: psi > 0 outside the body, < 0 inside),
 * the fractional areas of Eq. integral2.  psi_nodes: device, the
 * (nz+1) x (ny+1) x (nx+1) grid nodes in C order, node (i,j,k) at (i h, j h,
 * k h).  The paper takes the area calculation from a cited reference; here
 * each face is split into four triangles about its centre (psi there = the
 * mean of its four corners), psi is taken as linear on each triangle, and the
 * face's fraction is the mean of the triangles' areas where psi > 0 (a closed
 * form per triangle; exact for a planar body).  area_out: device, the three
 * low-face arrays (layout as for face coefficients), values in [0, 1]; wall
 * faces 0.  Errors: MG_ERR_ARG for a bad grid or null/unaligned arrays.
 */
int mg_face_areas(const mg_grid *g, const double *psi_nodes, double *const area_out[3], void *stream);

/*
 * Fractional face areas for a context (Eq. integral2 solved by the method of
 * fractional areas): the face coefficients given to mg_setup / mg_update are
 * then 1/rho_f, and the operator uses area_f * (1/rho_f) on the finest faces
 * (the product the Poisson-solver section moves to the coarse grids); a face
 * is open where that product is > 0.  mg_divergence weights each open face's
 * flux by its area; mg_correct updates the velocity of open faces with
 * 1/rho_f; mg_project_adjoint uses the areas in its gradients.  area: device,
 * three low-face arrays in [0, 1] (mg_face_areas), copied; NULL returns to
 * whole faces.  Rebuilds the hierarchy (as mg_update).  Cells are not merged:
 * a cut cell of small open area stays a cell of small coefficients.  Returns
 * MG_OK, MG_ERR_ARG (null context, null or unaligned array), MG_ERR_OOM (the
 * area arrays are allocated on first use) or MG_ERR_CUDA.
 */
int mg_set_face_areas(mg_ctx *c, const double *const area[3]);

/*
 * Body velocity v* on the faces (Eq. bc2), for the body term of Eq. integral2:
 * mg_divergence and mg_project use u - v on every open face.  For a body
 * velocity of zero divergence (a rigid motion, sampled at the face centres),
 * its flux through the body surface inside a cut cell is minus its flux
 * through the cell's open face parts (Gauss's theorem), so this adds the body
 * term; in cells the body does not cut, the discrete divergence of a rigid
 * motion is zero.  v: device, three face arrays, copied; NULL: a static body.
 * Returns MG_OK, MG_ERR_ARG (null context, null or unaligned array),
 * MG_ERR_OOM (allocated on first use) or MG_ERR_CUDA.
 */
int mg_set_body_velocity(mg_ctx *c, const double *const v[3]);

/*
 * Stretched grids (grids stretched along the Cartesian axes, as in the
 * paper's runs): cell widths hx[nx], hy[ny], hz[nz] (device).  Multiplying
 * Eq. integral2 by the cell volume puts it on the index grid of unit spacing,
 * with per low face
 *     beta_out = beta / d   (d: the distance between the two cell centres),
 *     area_out = the face's two widths * frac (frac: open fractions, or NULL
 *                for whole faces).
 * A context built on beta_out with h = 1 and given area_out by
 * mg_set_face_areas then solves the stretched problem: mg_divergence returns
 * the cell volume times b, the pressure and mg_correct's velocity are the
 * physical ones, and the adjoint's face gradient is with respect to beta_out
 * (divide by d for 1/rho).  g->h is ignored.  beta, frac: device face arrays
 * (layout as for face coefficients); beta_out, area_out: device, written;
 * wall faces 0.  Errors: MG_ERR_ARG for a bad grid or null/unaligned arrays.
 */
int mg_stretched_metrics(const mg_grid *g, const double *hx, const double *hy, const double *hz,
                         const double *const beta[3], const double *const frac[3], double *const beta_out[3],
                         double *const area_out[3], void *stream);

/*
 * Terms of the momentum equations (Eq. navi) other than the pressure gradient:
 * the body force -g on the z-faces (g = 1/Fr^2); the viscous term
 * inv_re (1/rho_f) d/dx_j (2 mu S_ij), S_ij = (du_i/dx_j + du_j/dx_i)/2, with
 * mu = mu_air + (mu_water - mu_air) phi (Eq. density, H(phi) = phi; the
 * dimensionless viscosities, water 1, air the ratio eta) when inv_re = 1/Re
 * > 0; the convective term -d/dx_j (u_j u_i) when convection != 0.  The
 * sub-grid stress is not modelled.
 */
typedef struct {
    double g;          /* 1/Fr^2 */
    double inv_re;     /* 1/Re (0: no viscous term) */
    double mu_air;     /* dimensionless viscosity of air (eta = mu_g/mu_l), >= 0 */
    double mu_water;   /* dimensionless viscosity of water (1), >= 0 */
    int convection;    /* nonzero: include the convective term */
} mg_forces;

/*
 * R_i of Eq. navi without the pressure gradient and the sub-grid stress (the
 * terms the Runge-Kutta stages add as dt R_i), on every face:
 *   R_i = -d/dx_j (u_j u_i) + inv_re (1/rho_f) d/dx_j (2 mu S_ij) - delta_i3 g.
 * The paper does not give the discrete operators; these are the second-order
 * central conservative MAC forms: u_i u_i at cell centres from the mean of the
 * cell's two i-faces, u_j u_i at cell edges from the means of the two j-faces
 * and of the two i-faces that meet there; 2 mu S_ii at cell centres (mu of the
 * cell), 2 mu S_ij at edges (mu the mean of the four cells around the edge);
 * each divergence the difference of the two values that bracket the face,
 * over h; the edge viscosity sums its four cells in the order of their index.  Walls are free-slip: normal velocity 0 (the stored wall face, or
 * the unstored high wall), the tangential velocity mirrored into the ghost
 * row, so no momentum flux and no shear cross a wall.  Faces with beta = 0
 * (walls, faces at a solid) get R = 0 and enter the stencils of their
 * neighbours with their stored velocity.  phi: device, nx*ny*nz; beta: device
 * face arrays, 1/rho on open faces and 0 on closed ones (mg_face_coeffs); u:
 * device face velocities; R: device face arrays, written (must not alias the
 * inputs); work: device scratch of 12*nx*ny*nz doubles (the fluxes and stresses
 * each cell shares with its faces, computed once per cell), overwritten; f:
 * host.  Returns MG_OK, MG_ERR_ARG (bad grid, null, aliased or unaligned array,
 * forces not finite) or MG_ERR_CUDA.
 */
int mg_momentum_rhs(const mg_grid *g, const double *phi, const double *const beta[3], const double *const u[3],
                    const mg_forces *f, double *const R[3], double *work, void *stream);

/*
 * One step of the second-order Runge-Kutta time integration (Numerical Time
 * Integration section) around the projection:
 *   stage 1: beta from phi^k (Eq. density); u~ = u^k + dt R(u^k, phi^k);
 *            P* from Eq. poisson1; u* = u~ - dt beta G P* (Eq. runge1);
 *            phi* = phi^k - VOF(u^k, phi^k, dt)
 *   stage 2: beta from phi*; u~~ = (u* + u^k) + dt R(u*, phi*); P from
 *            Eq. poisson2; u^{k+1} = (u~~ - dt beta G P) / 2 (Eq. runge2);
 *            phi^{k+1} = phi^k - VOF((u* + u^k)/2, phi^k, dt)
 * R is mg_momentum_rhs with the forces f (each stage's R from that stage's
 * velocity, volume fraction and 1/rho: Heun's method on the projected
 * equations, second order in time).  VOF is the conservative first-order
 * upwind flux form of Eq. vof (Q = 0) through the open faces.  The two
 * projections use the context's solver options (and its face areas and body
 * velocity, if set).  phi, solid_mask: as for mg_face_coeffs; f: host; u:
 * device face arrays, u^k on entry, u^{k+1} on return; phi_out: device,
 * phi^{k+1} (must not alias phi); p_out: device, P of the second stage.
 * stats: of the second projection.  Errors: as for mg_project, and MG_ERR_ARG
 * for null or non-finite forces.
 */
int mg_rk2_step(mg_ctx *c, const double *phi, const uint8_t *solid_mask, double rho_air, double rho_water,
                const mg_forces *f, double dt, double *const u[3], double *phi_out, double *p_out, double tol,
                mg_stats *stats);


/*
 * Solve A p = b to ||b - A p|| / ||b|| <= tol (multigrid of the Poisson-solver
 * section).  rhs: device, read only; its mean over each connected fluid region
 * is removed first (compatibility of the Neumann problem, Eq. neumann) and
 * isolated cells are ignored.  p: device, in = initial guess, out = solution
 * with zero mean over each fluid region (isolated cells 0).  stats: host or
 * NULL.  Returns MG_OK, MG_ERR_INCOMPATIBLE (converged; a region's rhs mean was
 * above the threshold given at mg_status), MG_ERR_NOT_CONVERGED (p holds the
 * last iterate), MG_ERR_NAN, or an error.  rhs and p must not alias.
 */
int mg_solve(mg_ctx *c, const double *rhs, double *p, double tol, mg_stats *stats);

/*
 * One V(nu1,nu2)-cycle on the finest grid, p updated in place, with no mean
 * removal and no residual check: red-black Gauss-Seidel (red = (i+j+k) even
 * first on the way down, colours reversed on the way up), residual and
 * cell-centred full weighting (mean of the 8 children), recursion, exact
 * coarsest solve, trilinear prolongation.  The cycle runs in the precision of
 * the context's solves: FP64 for MG_FP64; for MG_MIXED one FP32 cycle, on
 * rhs and p rounded to FP32 (the same kernels and coefficients the mixed
 * solves use), its result widened back into p.  rhs, p: device FP64; rhs is
 * used as given (the caller makes it compatible).
 * Returns MG_OK, MG_ERR_ARG (null or unaligned array) or MG_ERR_CUDA.
 */
int mg_vcycle(mg_ctx *c, const double *rhs, double *p);

/*
 * Right-hand side of Eq. poisson1 for a static body: rhs_c = (D u)_c / dt with
 *   (D u)_c = h^-1 * sum_axis ( u_high - u_low ) over the OPEN faces of c
 * (closed faces carry the wall/body velocity, zero).  u[0..2]: device face
 * arrays; rhs: device, written.
 * Returns MG_OK, MG_ERR_ARG (null or unaligned array, dt not > 0) or
 * MG_ERR_CUDA.
 */
int mg_divergence(mg_ctx *c, const double *const u[3], double dt, double *rhs);

/*
 * Velocity correction of Eq. runge1: on open faces u_f = u*_f - dt beta_f
 * (p_R - p_L) / h; closed faces copy u*.  u_star, u: device face arrays (u
 * may alias u_star); p: device.
 * Returns MG_OK, MG_ERR_ARG (null or unaligned array) or MG_ERR_CUDA.
 */
int mg_correct(mg_ctx *c, const double *const u_star[3], const double *p, double dt, double *const u[3]);

/*
 * Projection: rhs = D u* / dt (mg_divergence), solve (mg_solve, p's incoming
 * value is the initial guess), correct (mg_correct).  u_star: device, read;
 * u: device, written (may alias u_star); p: device, in/out.  The divergence
 * of u over the fluid cells is then at the solve's tolerance.
 * Returns MG_OK, MG_ERR_INCOMPATIBLE (as for mg_solve: a nonzero body-velocity
 * divergence, for instance), MG_ERR_NOT_CONVERGED (u and p from the last
 * iterate), MG_ERR_NAN, MG_ERR_ARG (null or unaligned array, dt or tol not > 0)
 * or MG_ERR_CUDA.
 */
int mg_project(mg_ctx *c, const double *const u_star[3], double *const u[3], double *p, double dt, double tol,
               mg_stats *stats);

/*
 * Adjoint of the projection (derived from u = u* - B G A^+ D u*, B = diag(beta),
 * G the face gradient on open faces, G = -D^T): for the upstream gradient
 * w = dL/du,
 *   c = D (beta w),  A q = c (same hierarchy: A is self-adjoint),
 *   grad_u*_f    = w_f - (G q)_f                    (closed faces: w_f)
 *   grad_beta_f  = dt (G p)_f ((G q)_f - w_f)       (closed faces: 0)
 * w: device face arrays; p: device, the forward solution; grad_u: device,
 * written; grad_beta: device or NULL; q_out: device scratch of nx*ny*nz
 * doubles that receives q (also the initial guess; pass zeros), may be NULL
 * to use the context's buffer.  stats: host or NULL.
 * Returns MG_OK, MG_ERR_INCOMPATIBLE (as for mg_solve), MG_ERR_NOT_CONVERGED
 * (the gradients from the last iterate), MG_ERR_NAN, MG_ERR_ARG (null, aliased
 * or unaligned array, dt or tol not > 0) or MG_ERR_CUDA.
 */
int mg_project_adjoint(mg_ctx *c, const double *const w[3], const double *p, double dt, double tol,
                       double *const grad_u[3], double *const grad_beta[3], double *q_out, mg_stats *stats);

/*
 * Chain rule from face coefficients to phi (Eq. density):
 *   d beta_f / d rho_c = -beta_f^2 / 2,  d rho / d phi = rho_water - rho_air,
 *   grad_phi_c = -(rho_water - rho_air)/2 * sum_{open faces f of c} beta_f^2 grad_beta_f.
 * beta, grad_beta: device face arrays; grad_phi: device, written.
 * Returns MG_OK, MG_ERR_ARG (bad grid, null or unaligned array) or
 * MG_ERR_CUDA.
 */
int mg_phi_grad(const mg_grid *g, const double *const beta[3], const double *const grad_beta[3], double rho_air,
                double rho_water, double *grad_phi, void *stream);

/* Hierarchy introspection (tests): number of levels, dimensions of level l
 * (host int[3] = nx, ny, nz), and a copy of one of its FP64 arrays
 * (which: 0,1,2 = beta x,y,z; 3 = inverse diagonal 1/sum(beta)) into a device
 * buffer of that level's size. * Returns the number of levels, 0 for a null context.
 */
int mg_num_levels(const mg_ctx *c);
int mg_level_dims(const mg_ctx *c, int level, int dims[3]);
int mg_level_array(mg_ctx *c, int level, int which, double *out);

/* Instrumentation.  mg_kernel_launches: number of CUDA kernels this library has
 * launched in this process (all contexts).  mg_profile_read: for a context made
 * with opts.profile != 0, the number of timed launches and their summed device
 * time (ms, CUDA events on the context's stream) of one kernel group since the
 * last mg_profile_reset; the stream must be idle (any solve returns so).
 * Groups: 0 = one finest-grid red-black smoothing sweep (both colours, in the
 * precision the cycles run in), 1 = finest-grid residual + restriction, 2 =
 * finest-grid prolongation, 3 = FP64 finest-grid residual (norm, mixed cast,
 * or the conjugate-gradient update), 4 = conjugate-gradient operator apply
 * q = A d, 5 = conjugate-gradient dot products and direction update, 6 = all
 * levels below the finest of one V-cycle (coarse-grid correction), 7 =
 * hierarchy rebuild (mg_update). */
enum {
    MG_PROF_SMOOTH = 0, MG_PROF_RESTRICT = 1, MG_PROF_PROLONG = 2, MG_PROF_RESID64 = 3, MG_PROF_APPLY = 4,
    MG_PROF_KRYLOV = 5, MG_PROF_COARSE = 6, MG_PROF_UPDATE = 7, MG_PROF_GROUPS = 8
};
uint64_t mg_kernel_launches(void);

/*
 * Bounds-check build.  A library compiled with -DMGP_CHECK (build(check=True):
 * libmgproj_check.so) checks in its kernels, before the loads and stores, that
 * every index a thread is about to use -- a cell, its stencil neighbours within
 * the stencil's guards, a colour-split slot, a coarse cell, a row of the
 * coarsest inverse -- lies inside the array it indexes; a thread with an index
 * outside skips its accesses and records it (nothing traps).  mg_check_read
 * returns the record since the previous read and resets it: *enabled = 1 in a
 * check build (0 otherwise, with *first = *count = 0), *first = the kernel's
 * check id << 48 | the index (0: none), *count = the number of skipped
 * accesses.  Host pointers.  Returns MG_OK, MG_ERR_ARG (null pointer) or
 * MG_ERR_CUDA.
 */
int mg_check_read(int *enabled, uint64_t *first, uint64_t *count);
int mg_profile_read(mg_ctx *c, int group, int *count, double *ms_total);
void mg_profile_reset(mg_ctx *c);

/*
 * Allocation-free residual check.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- applications whose
 * device memory all belongs to a pool or arena they must not bypass, loops
 * where an allocation (which may synchronise the device) is not allowed, and
 * hosts that give plug-ins no allocator.  It needs no mg_ctx.
 *
 * For rhs b and pressure p on grid g with face coefficients beta it writes
 * out[0] = ||b0 - A p||_2 / ||b0||_2 (0 if ||b0|| = 0), out[1] = ||b0||_2,
 * out[2] = the mean of b over the live cells, out[3] = the number of live
 * cells, where b0 = b - mean on live cells (cells with an open face) and 0
 * elsewhere -- the same quantities mg_solve reports in mg_stats (rel_resid,
 * rhs_norm, rhs_mean_removed) for its initial iterate when the fluid forms one
 * connected region (this check removes one mean over all live cells).  beta:
 * the operator's face coefficients (with fractional face areas, area x 1/rho,
 * the product mg_set_face_areas forms; on a stretched grid, area x beta / d).
 * beta, rhs, p: device, read only; out: device, 4 doubles, written.
 * Stream-ordered on `stream`.
 *
 * Its only scratch memory is a static __device__ array of the library
 * (4 * MG_NOALLOC_MAX_PLANES + 2 doubles, 128 KB on every GPU that loads the
 * library, held until the process exits); grids with nz > MG_NOALLOC_MAX_PLANES
 * are rejected with MG_ERR_ARG.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture.  The address is cached per
 * device for the life of the process: after cudaDeviceReset on a device, do not
 * call this function on that device again.  All calls share the array:
 * calls that overlap on the GPU (e.g. on two streams) race and must be
 * serialised by the caller.  Nothing is allocated or freed.
 */
#define MG_NOALLOC_MAX_PLANES 4096
int mg_residual_norm_noalloc(const mg_grid *g, const double *const beta[3], const double *rhs, const double *p,
                             double *out, void *stream);

void mg_destroy(mg_ctx *c);

/* Message of the last failed call on this thread ("" if none). */
const char *mg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MGPROJ_H */
