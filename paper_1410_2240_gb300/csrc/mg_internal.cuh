// mg_internal.cuh -- internal declarations shared by the CUDA kernels and the C ABI host code.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mgproj.h"

namespace mg {

// Geometry of one grid level.  Cell (i,j,k) is at linear index (k*ny + j)*nx + i.
struct Dims {
    int nx, ny, nz;
    size_t n() const { return (size_t)nx * ny * nz; }
};

// Arrays of one multigrid level in one precision.
template <typename T>
struct LevelArrays {
    T *bx = nullptr, *by = nullptr, *bz = nullptr;  // low-face coefficients
    T *dinv = nullptr;                               // 1 / sum of the six face coefficients (0 if none open)
    T *b = nullptr;                                  // right-hand side (levels >= 1; level 0 owned elsewhere)
    T *p = nullptr;                                  // correction (levels >= 1)
};

// Number of CTAs of the grid-stride vector and reduction kernels (16 per SM on 152 SMs,
// enough loads in flight to keep HBM busy).  A reduction's partials buffer holds 2 * kRedBlocks
// doubles and, after them, the counter of the blocks that have finished (kRedPartials doubles in
// all, the counter zero between reductions).
constexpr int kRedBlocks = 2432;
constexpr int kRedPartials = 2 * kRedBlocks + 2;
constexpr int kRedThreads = 256;

// Device scalar slots (FP64) in ctx->dscal.
enum Scal {
    S_SUM_B = 0,   // sum of the rhs over live cells
    S_NB2 = 1,     // ||b0||^2 after mean removal
    S_RR = 2,      // ||b0 - A p||^2 of the last residual pass
    S_SUM_P = 3,   // sum of p over live cells (same pass)
    S_SCALE0 = 4,  // mixed refinement: scale of the FP32 residual (ping)
    S_SCALE1 = 5,  // (pong)
    S_NLIVE = 6,   // number of live fine cells (as double)
    S_RZ = 7,      // PCG: <r, z>
    S_RZN = 8,     // PCG: new <r, z>
    S_RZO = 9,     // PCG: <r_new, z_old> (flexible beta)
    S_SIGMA = 10,  // PCG: <d, A d>
    S_ERR = 11,    // set to nonzero by a kernel whose bounded wait expired
    S_TOPO = 12,   // set to 1 by a hierarchy build whose open faces differ from the last build's
    S_COUNT = 16
};

// bounds-check build (-DMGP_CHECK): the first recorded out-of-range index (kernel id << 48 |
// index) and the number of skipped accesses since the last read, then reset; returns 1 in a check
// build, 0 otherwise (first = count = 0), -1 if the device copy failed
int check_read(unsigned long long *first, unsigned long long *count);

// total kernels launched by this library in this process
unsigned long long launch_count();
void note_kernel_launch();

// set the message mg_last_error() returns on this thread
void set_last_error(const char *msg);

// Division of 32-bit unsigned integers by a divisor fixed for a launch: a multiply-high, a
// subtraction, an addition and two shifts instead of an emulated division (Granlund and
// Montgomery, "Division by invariant integers using multiplication", PLDI 1994, the round-up
// method; exact for every dividend below 2^32).
struct FastDiv {
    unsigned mult = 0, s1 = 0, s2 = 0;
};
inline FastDiv make_fastdiv(unsigned d)
{
    unsigned l = 0;
    while ((1ull << l) < d) l++;  // l = ceil(log2 d)
    const unsigned long long m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
    return FastDiv{(unsigned)m, l < 1 ? l : 1u, l > 1 ? l - 1 : 0u};
}

// Layout of the finest level's FP32 iterate and right-hand side.  half == 0: natural C order.
// half == n / 2 (all dims even): colour-split, the cells of colour (i + j + k) & 1 == 0 in
// [0, half) and of colour 1 in [half, n), cell c at slot c >> 1 of its colour's half.  Face
// coefficients and every FP64 field keep the natural order.
struct Split {
    size_t half = 0;
    int nx = 0, ny = 0;
    FastDiv fnx, fny;  // division by nx and ny (the row and plane of a natural index)
};

// The coarse tail: levels lev[0] (the largest) .. lev[nlev-1] (the coarsest) of the hierarchy,
// run by one CTA.  Each level's b and p are the ones a V-cycle on it would receive.
constexpr int kTailMaxLevels = 8;
template <typename T>
struct TailLevel {
    int nx, ny, nz;
    T h2, ih2;
    LevelArrays<T> L;
    FastDiv fhx, fny, fcx, fcy;  // division by (nx + 1) / 2, ny, nx / 2 and ny / 2
};
template <typename T>
struct TailArgs {
    int nlev, nu1, nu2;
    int zero0;  // nonzero: lev[0].p starts at zero (zeroed here, not by the caller)
    TailLevel<T> lev[kTailMaxLevels];
};

// ---- kernel launchers (mg_kernels.cu); all stream-ordered, return cudaError_t of the launch ----
cudaError_t launch_face_coeffs(Dims d, const double *phi, const uint8_t *solid, double rho_a, double drho,
                               double *bx, double *by, double *bz, cudaStream_t s);
// op (optional): also write the CG operator's arrays scaled by `scale` (op->dinv = the scaled sum);
// open (optional): per-cell open bits of the three low faces, updated, *changed = 1 where any changed
template <typename T>
cudaError_t launch_diag_inv(Dims d, const T *bx, const T *by, const T *bz, T *dinv, cudaStream_t s,
                            const LevelArrays<T> *op = nullptr, T scale = T(1), uint8_t *open = nullptr,
                            double *changed = nullptr);
cudaError_t launch_restrict_coeffs(Dims fine, const double *bx, const double *by, const double *bz, double *cbx,
                                   double *cby, double *cbz, cudaStream_t s);
// the FP32 copy of a level (faces and 1/sum of the narrowed faces) from its FP64 faces; with sf,
// the faces also in the colour-split layout sp
cudaError_t launch_level_f32(Dims d, const LevelArrays<double> &L, LevelArrays<float> &out, cudaStream_t s,
                             LevelArrays<float> *sf = nullptr, Split sp = {});

// one colour of a red-black sweep on planes [z0, z1) (z1 < 0: to the last plane); zero: the
// iterate is zero and is not read (the first pass of a cycle from a zero guess)
template <typename T>
cudaError_t launch_smooth(Dims d, T h2, const LevelArrays<T> &L, const T *b, T *p, int colour, cudaStream_t s,
                          int z0 = 0, int z1 = -1, bool zero = false);
// one colour of a red-black sweep on the colour-split layout (FP32, all dims even); urow (optional):
// the level's uniform-row values, arow (optional, nx % 8 == 0, replaces urow in the sweep): its
// banded-row records (launch_uniform_rows); rev: blocks take the planes in descending order; S
// (required where nx % 8 == 0): the face arrays of L in the colour-split layout
cudaError_t launch_smooth_split(Dims d, float h2, const LevelArrays<float> &L, const float *b, float *p, int colour,
                                cudaStream_t s, const float *urow = nullptr, const float4 *arow = nullptr,
                                int rev = 0, bool zero = false, const LevelArrays<float> *S = nullptr);
// urow[k*ny + j] = v if row (j,k) is interior (0 < j < ny-1, 0 < k < nz-1) and every face around
// it but its two x-walls equals v, else 0; arow
// (optional) = {vx, vy, vzl, vzh} if the row's x-, y-, low z- and high z-faces hold one value
// each, else zeros; count (optional, two counters, incremented): uniform rows, banded rows that
// are not uniform
cudaError_t launch_uniform_rows(Dims d, const float *bx, const float *by, const float *bz, float *urow,
                                cudaStream_t s, float4 *arow = nullptr, unsigned *count = nullptr);
// FP32 fused sweep with TMA-staged planes (mg_sweep_tma.cu)
bool tma_sweep_supported(Dims d);
cudaError_t launch_rb_sweep_tma(Dims d, float h2, const LevelArrays<float> &L, const float *b, const float *p_old,
                                float *p_new, int first, double *dscal, cudaStream_t s);

// one full red-black sweep (first colour, then the other) from p_old into p_new
template <typename T>
cudaError_t launch_rb_sweep(Dims d, T h2, const LevelArrays<T> &L, const T *b, const T *p_old, T *p_new, int first,
                            cudaStream_t s);
// b and p of the fine level in the layout sp (FP32 only may be split); bc natural; rev (FP32): blocks
// take the coarse planes in descending order
template <typename T>
cudaError_t launch_resid_restrict(Dims fine, T ih2, const LevelArrays<T> &L, const T *b, const T *p, T *bc,
                                  cudaStream_t s, Split sp = {}, const float *urow = nullptr, int rev = 0);
template <typename T>
// urow (optional, FP32): the fine level's uniform-row values (cells of uniform rows are all live)
cudaError_t launch_prolong(Dims fine, const T *ec, const T *dinv, T *p, cudaStream_t s, Split sp = {},
                           const float *urow = nullptr);
template <typename T>
cudaError_t launch_coarse_solve(int n, const double *M, const T *b, T *e, cudaStream_t s);
// the coarse tail's descent (pre-smoothing, restriction down to lev[nlev-1].b) and ascent
// (prolongation of lev[nlev-1].p, post-smoothing up to lev[0].p); the coarsest solve runs between
template <typename T>
cudaError_t launch_tail_down(const TailArgs<T> &a, cudaStream_t s);
template <typename T>
cudaError_t launch_tail_up(const TailArgs<T> &a, cudaStream_t s);

// connected components of the live cells (joined by open faces): label[c] = the smallest cell
// index of c's component (-1 on dead cells); ctr[0] = number of components, ctr[1] != 0 if a
// bounded loop gave up (both reset here)
cudaError_t launch_components(Dims d, const double *dinv, const double *bx, const double *by, const double *bz,
                              int *label, unsigned *ctr, cudaStream_t s);
// the component roots (label[c] == c) into roots[0..cap) in any order; *slot = their number
cudaError_t launch_component_roots(size_t n, const int *label, int *roots, unsigned *slot, unsigned cap,
                                   cudaStream_t s);
// Up to kCompOrdered components are summed in a fixed order (bitwise reproducible, one pass per
// eight components, per-block sums in part[8 * kRedBlocks]); more are summed with atomics (not
// reproducible bit for bit from run to run).
constexpr int kCompOrdered = 64;
// sums[m] = sum of v (v null: 1) over the live cells of component m (comp[c] = m)
cudaError_t launch_comp_sums(size_t n, const double *v, const int *comp, int ncomp, double *sums, double *part,
                             cudaStream_t s);
// label: root -> rank among sorted_roots (the component number); cnt[m] = cells of component m
cudaError_t launch_component_compact(size_t n, int *label, const int *sorted_roots, int ncomp, double *cnt,
                                     double *part, cudaStream_t s);
// out = v - the mean of v over its component on live cells (comp >= 0), 0 elsewhere; sums[m] =
// the component sums of v; dscal[slot_sq] = ||out||^2, dscal[slot_sum] = sum of v (slots < 0:
// not written)
cudaError_t launch_comp_center(size_t n, const double *v, const int *comp, int ncomp, double *sums,
                               const double *cnt, double *out, double *partials, double *dscal, int slot_sq,
                               int slot_sum, cudaStream_t s, double *part);

// reductions and fine-level helpers (FP64)
cudaError_t launch_count_live(Dims d, const double *dinv, double *partials, double *dscal, cudaStream_t s);
cudaError_t launch_rhs_prepare(Dims d, const double *rhs, const double *dinv, double *b0, double *partials,
                               double *dscal, cudaStream_t s);
cudaError_t launch_resid_norm(Dims d, double ih2, const LevelArrays<double> &L, const double *b, const double *p,
                              double *partials, double *dscal, cudaStream_t s);
cudaError_t launch_sub_mean_p(Dims d, const double *dinv, double *p, const double *dscal, cudaStream_t s);
// r32 / e32: the finest FP32 fields, in the layout sp
cudaError_t launch_resid_cast(Dims d, double ih2, const LevelArrays<double> &L, const double *b, const double *p,
                              float *r32, double *partials, double *dscal, int scale_in, int scale_out,
                              cudaStream_t s, Split sp = {});
cudaError_t launch_accumulate(Dims d, const double *dinv, const float *e32, double *p, const double *dscal,
                              int scale_slot, cudaStream_t s, Split sp = {});
// dst = (float)src into the layout sp / dst = (double)src out of it (natural-order FP64 side)
cudaError_t launch_to_f32_layout(size_t n, const double *src, float *dst, cudaStream_t s, Split sp = {});
cudaError_t launch_from_f32_layout(size_t n, const float *src, double *dst, cudaStream_t s, Split sp = {});

// multigrid-preconditioned CG (FP64 Krylov vectors)
// pnz (optional): a device word; with it, the pass first tests whether p is zero everywhere and,
// if so, takes r = b without loading p's stencil (the same values)
cudaError_t launch_pcg_resid(Dims d, double ih2, const LevelArrays<double> &L, const double *b, const double *p,
                             double *r, float *r32, double *partials, double *dscal, int scale_slot, cudaStream_t s,
                             Split sp = {}, unsigned *pnz = nullptr);
template <typename Z>
cudaError_t launch_pcg_dots(size_t n, const double *r, const Z *z, const Z *zo, double *partials, double *dscal,
                            int sz_slot, int so_slot, cudaStream_t s);
cudaError_t launch_pcg_dots32(size_t n, const float *r32, const float *z, const float *zo, double *partials,
                              double *dscal, int sr_slot, int sz_slot, int so_slot, cudaStream_t s);
// z = scale * dinv * r (the Jacobi preconditioner of the CG)
cudaError_t launch_jacobi(size_t n, double scale, const double *dinv, const double *r, double *z, cudaStream_t s);
// d = D, the CG direction divided by the scale of its preconditioned residual (dscal[sz_slot]);
// so_slot: the scale of the previous D (-1 on the first direction or without scales)
template <typename Z>
cudaError_t launch_pcg_dir(size_t n, const Z *z, double *d, double *dscal, int sz_slot, int so_slot, int first,
                           cudaStream_t s, Split sp, double *partials);
// op: face coefficients and diagonal pre-scaled by h^-2 (op.dinv holds the scaled diagonal)
cudaError_t launch_pcg_apply(Dims d, const LevelArrays<double> &op, const double *dv, double *q, double *partials,
                             double *dscal, cudaStream_t s);
// sd_slot: the scale of the direction dv (its k_pcg_dir's sz_slot; -1 without scales)
cudaError_t launch_pcg_update(size_t n, const double *dv, const double *q, double *p, double *r, float *r32,
                              double *partials, double *dscal, int scale_slot, int sd_slot, cudaStream_t s,
                              Split sp = {});

// projection and adjoint
cudaError_t launch_divergence(Dims d, double scale, const double *bx, const double *by, const double *bz,
                              const double *ux, const double *uy, const double *uz, double *rhs, cudaStream_t s);
// the face is open where b > 0; val (optional): its coefficient (1/rho) when b holds area * 1/rho
cudaError_t launch_correct(Dims d, double dt, double h, const double *bx, const double *by, const double *bz,
                           const double *p, const double *ux0, const double *uy0, const double *uz0, double *ux,
                           double *uy, double *uz, cudaStream_t s, const LevelArrays<double> *val = nullptr);
// fractional face areas (open fractions of the low faces) from psi at the (nx+1)(ny+1)(nz+1) nodes
cudaError_t launch_face_areas(Dims d, const double *psi, double *ax, double *ay, double *az, cudaStream_t s);
// stretched-grid metrics: bout = beta / (centre distance), aout = face widths * frac (frac null: 1)
cudaError_t launch_stretched_metrics(Dims d, const double *hx, const double *hy, const double *hz,
                                    const LevelArrays<double> &beta, const LevelArrays<double> &frac,
                                    const LevelArrays<double> &bout, const LevelArrays<double> &aout, cudaStream_t s);
// time step pieces: out = (a + b) + dt R, R three face arrays (b null: a + dt R);
// out = 0.5 (a + b); phi_out = phi - (dt/h) sum +-u phi_upwind over open faces
cudaError_t launch_rk_combine(size_t n, const LevelArrays<double> &a, const LevelArrays<double> &b,
                              const LevelArrays<double> &r, double dt, const LevelArrays<double> &out, cudaStream_t s);
// R = the momentum right-hand side of Eq. navi on the faces (convective if convect, viscous with
// mu = mu_air + (mu_water - mu_air) phi scaled by inv_re and beta = 1/rho, -g on the z-faces),
// 0 on closed faces (beta == 0); work: 12 nx*ny*nz doubles (the per-cell fluxes and stresses)
constexpr int kMomWork = 12;
cudaError_t launch_momentum_rhs(Dims d, double h, const double *phi, double mu_air, double mu_water, double inv_re,
                                double g, int convect, const LevelArrays<double> &beta, const LevelArrays<double> &u,
                                const LevelArrays<double> &r, double *work, cudaStream_t s);
cudaError_t launch_half(size_t n, const LevelArrays<double> &a, const LevelArrays<double> &b,
                        const LevelArrays<double> &out, cudaStream_t s);
cudaError_t launch_vof_upwind(Dims d, double s_dt_h, const LevelArrays<double> &mask, const LevelArrays<double> &u,
                              const double *phi, double *phi_out, cudaStream_t s);
// out = area * beta on faces of open area, 0 elsewhere (bx/by/bz of each)
cudaError_t launch_area_coeffs(size_t n, const LevelArrays<double> &area, const LevelArrays<double> &beta,
                               const LevelArrays<double> &out, cudaStream_t s);
// rhs = scale * sum over open faces (mask > 0) of +-area (u - v); area or v null: 1 or 0
cudaError_t launch_divergence_area(Dims d, double scale, const LevelArrays<double> &mask,
                                   const LevelArrays<double> &area, const LevelArrays<double> &u,
                                   const LevelArrays<double> &v, double *rhs, cudaStream_t s);
// rhs = scale * sum over the open faces (L > 0) of +-(B w): the divergence of the face products
cudaError_t launch_divergence_mul(Dims d, double scale, const LevelArrays<double> &L, const LevelArrays<double> &B,
                                  const double *wx, const double *wy, const double *wz, double *rhs, cudaStream_t s);
cudaError_t launch_adjoint_faces(Dims d, double h, double dt, const double *bx, const double *by,
                                 const double *bz, const double *p, const double *q, const double *wx,
                                 const double *wy, const double *wz, double *gux, double *guy, double *guz,
                                 double *gbx, double *gby, double *gbz, cudaStream_t s,
                                 const LevelArrays<double> *area = nullptr);
cudaError_t launch_phi_grad(Dims d, double neg_half_drho, const double *bx, const double *by, const double *bz,
                            const double *gbx, const double *gby, const double *gbz, double *gphi,
                            cudaStream_t s);

}  // namespace mg
