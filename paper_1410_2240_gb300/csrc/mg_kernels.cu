// mg_kernels.cu -- CUDA kernels (sm_103a) of the variable-density pressure projection.
//
// Every kernel works on one grid level stored in C order [k][j][i] (x fastest).
// Face arrays hold the LOW face of each cell: bx[c] couples cells c-1 and c in x;
// bx[.][.][0] is the wall (0).  The high wall face is not stored (closed).
// A "live" cell has at least one open face (dinv > 0); other cells (solid or
// isolated) hold p = 0 and are excluded from means and norms.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>
#include <type_traits>

#include "mg_internal.cuh"

namespace mg {

static std::atomic<unsigned long long> g_launches{0};
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void note_kernel_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

constexpr int kRowThreads = 128;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; the result is valid in thread 0.  NT = blockDim.x.
template <int NT>
__device__ double block_sum(double v)
{
    __shared__ double sh[NT / 32];
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (l < NT / 32) ? sh[l] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// A scalar every thread of a block needs, computed by thread 0 and shared: FP64 divisions and
// square roots of the CG's scalars would otherwise run in every thread, on the FP64 unit these
// passes are bound by (tens of operations per thread, one to two per cell).  f() is called in
// thread 0 only; the value is the one each thread would have computed.
template <typename F>
__device__ __forceinline__ double block_scalar(F f)
{
    __shared__ double v;
    if (threadIdx.x == 0) v = f();
    __syncthreads();
    return v;
}

// Sums the per-block partial pairs in a fixed order (deterministic) into dscal.
__global__ void k_finish2(const double *__restrict__ partials, int nblocks, double *__restrict__ dscal, int slot0,
                          int slot1)
{
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
    }
    a = block_sum<kRedThreads>(a);
    b = block_sum<kRedThreads>(b);
    if (threadIdx.x == 0) {
        if (slot0 >= 0) dscal[slot0] = a;
        if (slot1 >= 0) dscal[slot1] = b;
    }
}

// The end of a grid-wide reduction in the reducing kernel itself: every block stores its pair of
// block sums (valid in thread 0); the last block to finish -- a counter in the word after the
// 2 * kRedBlocks partials, reset by that block -- sums the pairs in k_finish2's order and writes
// dscal[slot0], dscal[slot1] (slots < 0: not written).  The same sums as a separate k_finish2
// launch, one launch fewer.  Returns true in the last block (all its threads).
__device__ bool reduce_finish(double a, double b, double *partials, double *dscal, int slot0, int slot1)
{
    __shared__ bool last;
    unsigned *ctr = reinterpret_cast<unsigned *>(partials + 2 * kRedBlocks);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
        __threadfence();
        last = atomicAdd(ctr, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double x = 0.0, y = 0.0;
    // two strides per iteration, both loads issued before either sum: half the chain of
    // dependent L2 round trips, the same additions in the same order
    const int nb = (int)gridDim.x;
    for (int i = threadIdx.x; i < nb; i += 2 * blockDim.x) {
        const int i2 = i + (int)blockDim.x;
        const double x0 = __ldcg(partials + 2 * i), y0 = __ldcg(partials + 2 * i + 1);
        const double x1 = i2 < nb ? __ldcg(partials + 2 * i2) : 0.0, y1 = i2 < nb ? __ldcg(partials + 2 * i2 + 1) : 0.0;
        x += x0;
        y += y0;
        if (i2 < nb) {
            x += x1;
            y += y1;
        }
    }
    x = block_sum<kRedThreads>(x);
    y = block_sum<kRedThreads>(y);
    if (threadIdx.x == 0) {
        if (slot0 >= 0) dscal[slot0] = x;
        if (slot1 >= 0) dscal[slot1] = y;
        *ctr = 0u;
    }
    return true;
}

// The last block of a grid to get here (the counter after the partials, reset by that block):
// true in all its threads.  For kernels that need one block to act after every block has read
// something, with nothing to sum.
__device__ bool last_block(double *partials)
{
    __shared__ bool last;
    unsigned *ctr = reinterpret_cast<unsigned *>(partials + 2 * kRedBlocks);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ctr, 1u) == gridDim.x - 1;
        if (last) *ctr = 0u;
    }
    __syncthreads();
    return last;
}

__device__ __forceinline__ void cell_of(unsigned idx, int nx, int ny, int &i, int &j, int &k)
{
    const unsigned t = idx / (unsigned)nx;
    i = (int)(idx - t * (unsigned)nx);
    k = (int)(t / (unsigned)ny);
    j = (int)(t - (unsigned)k * (unsigned)ny);
}

// ---------------------------------------------------------------------------
// Face coefficients (Eq. density, H(phi) = phi; face product (1/rho)*area):
// rho = rho_a + drho*phi, beta = 2/(rho_L + rho_R) on open faces.  Rounded as
// separate IEEE operations (no contraction) so that it is reproducible.
// ---------------------------------------------------------------------------
// Set-up kernels walk kRun cells up a z-column per thread.  A quotient x / den depends on den
// alone, so each keeps its last divisor and quotient and divides again only when the divisor's
// bits change: in a uniform region (pure air, pure water, constant coefficients) that is once
// per run instead of once per cell, and the results are those of dividing every time.
constexpr int kRun = 16;
// a compile-time bool as a value (a generic lambda's case)
template <bool B>
struct BoolTag {
    static constexpr bool value = B;
};
// Kernels that share face products along rows (k_phi_grad, k_divergence_mul): blocks of at most
// kPhiThreads threads over rows of at most kPhiW cells, kPhiRun planes per block.
constexpr int kPhiW = 256, kPhiThreads = 512, kPhiRun = 8;

__device__ __forceinline__ bool same_bits(double a, double b)
{
    return __double_as_longlong(a) == __double_as_longlong(b);
}
__device__ __forceinline__ bool same_bits(float a, float b) { return __float_as_int(a) == __float_as_int(b); }

// a / b as a call: the compiler cannot run a call speculatively, so a memo that skips the
// division really skips it (an inlined division is if-converted and runs on every lane, and on
// this part's narrow FP64 unit it costs as much as the rest of the pass)
template <typename T>
__device__ __noinline__ T div_call(T a, T b)
{
    return a / b;
}

// float -> double on the integer pipe.  The hardware conversion issues on the FP64 unit, which
// bounds the CG kernels that widen an FP32 field per cell.  From the IEEE 754 binary32 and binary64
// layouts: the sign is kept, the exponent rebiased (127 -> 1023), the 23-bit fraction shifted into
// the top of the 52-bit one; zeros, infinities and NaNs map field by field.  Subnormal floats (never
// produced by the scaled cycles, but possible) take the hardware conversion.  Exact: every float is
// a double.
__device__ __noinline__ double f2d_slow(float x) { return (double)x; }
__device__ __forceinline__ double widen(float x)
{
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    const unsigned long long sgn = (unsigned long long)(b >> 31) << 63;
    if (e == 0u) return m ? f2d_slow(x) : __longlong_as_double((long long)sgn);
    const unsigned long long ee = (e == 0xffu) ? 0x7ffull : (unsigned long long)(e + 896u);
    return __longlong_as_double((long long)(sgn | (ee << 52) | ((unsigned long long)m << 29)));
}
__device__ __forceinline__ double widen(double x) { return x; }

// x > 0 and x == 0 decided on the integer pipe (an FP64 comparison occupies the FP64 unit, the
// limiting resource of the FP64 passes).  pos_bits(x) equals x > 0 for every x but a NaN with a
// clear sign bit; the coefficients, inverse diagonals and live masks it is applied to are never
// NaN for finite input.  zero_bits(x) equals x == 0 for every x.
__device__ __forceinline__ bool pos_bits(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool pos_bits(float x) { return __float_as_int(x) > 0; }
__device__ __forceinline__ bool zero_bits(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ bool zero_bits(float x) { return (__float_as_int(x) << 1) == 0; }

// ---------------------------------------------------------------------------
// Bounds-check build (-DMGP_CHECK).  Before its loads and stores a kernel checks that every index
// it is about to use, within the guards of its stencil, lies inside the array it indexes
// (nx*ny*nz cells, a colour half, a coarse level); a thread with an index outside skips its
// accesses and records the kernel and the index (the first such record and a count, read by
// mg_check_read).  Nothing traps.  In the normal build MG_CK is the constant true and every check
// folds away.
// ---------------------------------------------------------------------------
enum CheckKernel : unsigned {
    CK_SMOOTH = 1, CK_SMOOTH_SPLIT, CK_SMOOTH_SPLIT4, CK_RESTRICT, CK_RESTRICT_PAIRS, CK_PROLONG, CK_COARSE_SOLVE,
    CK_TAIL, CK_RESID, CK_SPLIT_SLOT, CK_PCG_APPLY, CK_DIVERGENCE, CK_CORRECT, CK_ADJOINT, CK_PHI_GRAD,
    CK_FACE_COEFFS, CK_DIAG_INV, CK_MOMENTUM, CK_LABEL, CK_VOF, CK_NARROW, CK_POW2
};
#ifdef MGP_CHECK
__device__ unsigned long long g_check_first = 0;  // kernel id << 48 | (index & (2^48 - 1)); 0: none
__device__ unsigned long long g_check_count = 0;
__device__ __noinline__ void ck_record(unsigned kid, long long idx)
{
    atomicAdd(&g_check_count, 1ull);
    atomicCAS(&g_check_first, 0ull,
              ((unsigned long long)kid << 48) | ((unsigned long long)idx & 0xffffffffffffull));
}
// [lo, hi] inside [0, n)
__device__ __forceinline__ bool ck_in(long long lo, long long hi, long long n, unsigned kid)
{
    if (lo >= 0 && hi < n) return true;
    ck_record(kid, lo < 0 ? lo : hi);
    return false;
}
#define MG_CK(lo, hi, n, kid) ck_in((long long)(lo), (long long)(hi), (long long)(n), (unsigned)(kid))
#else
#define MG_CK(lo, hi, n, kid) true
#endif
// double -> float, rounded to nearest (ties to even), on the integer pipe: the hardware conversion
// issues on the FP64 unit, the limiting resource of the FP64 passes that hand an FP32 copy to the
// cycles.  From the IEEE 754 layouts: the exponent rebiased (1023 -> 127), the 52-bit fraction cut
// to its top 23 bits and rounded by the 29 bits cut off (above half, or exactly half with an odd
// result, adds one unit; a carry into the exponent is the correct rounding, up to infinity).
// Zeros map exactly; results that would be subnormal, and infinities and NaNs, take the hardware
// conversion.  The check build compares every result with the hardware conversion.
__device__ __noinline__ float d2f_slow(double x) { return __double2float_rn(x); }
__device__ __forceinline__ float narrow(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sgn = (unsigned)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7ffull);
    const unsigned long long m = b & 0xfffffffffffffull;
    float f;
    if (e == 0 && m == 0) {
        f = __uint_as_float(sgn);
    } else if (e - 896 <= 0 || e - 896 >= 255) {
        f = d2f_slow(x);
    } else {
        const unsigned mant = (unsigned)(m >> 29), rest = (unsigned)(m & 0x1fffffffull);
        unsigned u = sgn | ((unsigned)(e - 896) << 23) | mant;
        if (rest > 0x10000000u || (rest == 0x10000000u && (mant & 1u))) u += 1u;
        f = __uint_as_float(u);
    }
#ifdef MGP_CHECK
    if (__float_as_uint(f) != __float_as_uint(__double2float_rn(x)) && !(isnan(x) && isnan(f)))
        ck_record(CK_NARROW, (long long)(b >> 16));
#endif
    return f;
}

// Products that only some lanes or launches need, as calls: the compiler cannot run a call
// speculatively, so a branch around one is not if-converted into an FP64 instruction that every
// warp issues (predicated off, it still occupies the FP64 unit).
__device__ __noinline__ double dmul_call(double x, double f) { return __dmul_rn(x, f); }
__device__ __noinline__ double sq_mul_call(double b, double g) { return __dmul_rn(__dmul_rn(b, b), g); }

// x * f for f = 2^e, bit for bit the product __dmul_rn(x, f), on the integer pipe where x and the
// product are normal numbers: e added to the exponent field (the FP64 unit is the limiting
// resource of the FP64 set-up and projection passes).  Zeros, subnormals, infinities, NaNs and
// products outside the normal range take the multiply (a call).  The check build compares every
// result with the multiply.
__device__ __forceinline__ double mul_pow2(double x, double f, int e)
{
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const int ex = (hi >> 20) & 0x7ff;
    double y;
    if ((unsigned)(ex - 1) < 2046u && (unsigned)(ex + e - 1) < 2046u)
        y = __hiloint2double(hi + e * (1 << 20), lo);
    else
        y = dmul_call(x, f);
#ifdef MGP_CHECK
    if (__double_as_longlong(y) != __double_as_longlong(__dmul_rn(x, f)) && !isnan(x))
        ck_record(CK_POW2, (long long)((unsigned long long)__double_as_longlong(x) >> 16));
#endif
    return y;
}
// a power-of-two factor (ok: f = 2^e) or any other (ok = 0: a multiply)
struct Scale2 {
    double f;
    int e, ok;
};
__device__ __forceinline__ double mul_s2(double x, const Scale2 &s) { return s.ok ? mul_pow2(x, s.f, s.e) : dmul_call(x, s.f); }

// cell c = (i, j, k) and the neighbours its guards admit (i > 0: c - 1, i < nx - 1: c + 1, ...)
// inside the nx*ny*nz cells
__device__ __forceinline__ bool ck_cell(long long c, int i, int j, int k, int nx, int ny, int nz, unsigned kid)
{
    const long long n = (long long)nx * ny * nz, sxy = (long long)nx * ny;
    (void)n;
    (void)sxy;
    return MG_CK(c, c, n, kid) && (i == 0 || MG_CK(c - 1, c - 1, n, kid)) &&
           (i >= nx - 1 || MG_CK(c + 1, c + 1, n, kid)) && (j == 0 || MG_CK(c - nx, c - nx, n, kid)) &&
           (j >= ny - 1 || MG_CK(c + nx, c + nx, n, kid)) && (k == 0 || MG_CK(c - sxy, c - sxy, n, kid)) &&
           (k >= nz - 1 || MG_CK(c + sxy, c + sxy, n, kid));
}

inline dim3 run_grid(int nx, int ny, int nz)
{
    return dim3((unsigned)((nx + kRowThreads - 1) / kRowThreads), (unsigned)ny, (unsigned)((nz + kRun - 1) / kRun));
}

// beta_f = 2 / (rho_L + rho_R), rho = rho_a + drho phi (each operation rounded separately); 0 on
// walls and on faces touching a solid cell.  The density of the cell below is carried up the run.
__global__ void k_face_coeffs(int nx, int ny, int nz, const double *__restrict__ phi,
                              const uint8_t *__restrict__ solid, double rho_a, double drho, double *__restrict__ bx,
                              double *__restrict__ by, double *__restrict__ bz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nx) return;
    const int k0 = blockIdx.z * kRun, k1 = min(k0 + kRun, nz);
    const size_t sxy = (size_t)nx * ny;
    // divisor memo per face direction (2 / 1 = 2 exactly)
    double dx_last = 1.0, qx_last = 2.0, dy_last = 1.0, qy_last = 2.0, dz_last = 1.0, qz_last = 2.0;
    size_t c = (size_t)k0 * sxy + (size_t)j * nx + i;
    bool s_below = k0 > 0 && solid && solid[c - sxy];
    double r_below = k0 > 0 ? __dadd_rn(rho_a, __dmul_rn(drho, phi[c - sxy])) : 0.0;
    // a cell's inputs (phi and the solid flags of the cell and its x- and y- neighbours), all
    // loaded at once; the next cell's are loaded before this one's faces are formed and stored
    struct In {
        double pc, px, py;
        bool sc, sx, sy;
    };
    auto load = [&](size_t cc) {
        In v;
        v.pc = phi[cc];
        v.px = i > 0 ? phi[cc - 1] : 0.0;
        v.py = j > 0 ? phi[cc - nx] : 0.0;
        v.sc = solid && solid[cc];
        v.sx = solid && i > 0 && solid[cc - 1];
        v.sy = solid && j > 0 && solid[cc - nx];
        return v;
    };
    In cur = load(c);
    for (int k = k0; k < k1; k++, c += sxy) {
        const In nxt = k + 1 < k1 ? load(c + sxy) : cur;
        const bool sc = cur.sc;
        const double rc = __dadd_rn(rho_a, __dmul_rn(drho, cur.pc));
        double v = 0.0;
        if (i > 0 && !sc && !cur.sx) {
            const double den = __dadd_rn(__dadd_rn(rho_a, __dmul_rn(drho, cur.px)), rc);
            if (!same_bits(den, dx_last)) {
                dx_last = den;
                qx_last = div_call(2.0, den);
            }
            v = qx_last;
        }
        bx[c] = v;
        v = 0.0;
        if (j > 0 && !sc && !cur.sy) {
            const double den = __dadd_rn(__dadd_rn(rho_a, __dmul_rn(drho, cur.py)), rc);
            if (!same_bits(den, dy_last)) {
                dy_last = den;
                qy_last = div_call(2.0, den);
            }
            v = qy_last;
        }
        by[c] = v;
        v = 0.0;
        if (k > 0 && !sc && !s_below) {
            const double den = __dadd_rn(r_below, rc);
            if (!same_bits(den, dz_last)) {
                dz_last = den;
                qz_last = div_call(2.0, den);
            }
            v = qz_last;
        }
        bz[c] = v;
        s_below = sc;
        r_below = rc;
        cur = nxt;
    }
}

// dinv = 1 / (sum of the six face coefficients), summed x-, x+, y-, y+, z-, z+; 0 if none is
// open.  Optionally (op != null) the CG operator's arrays scaled by `scale` = h^-2: op->dinv =
// scale * sum, op->bx/by/bz = scale * the faces (mul_s2: the products, on the integer pipe when
// h^-2 is a power of two).  kRun cells per thread with the divisor memo above.
template <typename T>
// open (optional): per cell the open bits of its three low faces (x 1, y 2, z 4), kept from the
// last call; where they change, *changed = 1 (the fluid regions must be labelled again)
__global__ void k_diag_inv(int nx, int ny, int nz, const T *__restrict__ bx, const T *__restrict__ by,
                           const T *__restrict__ bz, T *__restrict__ dinv, LevelArrays<T> op, Scale2 scale,
                           uint8_t *__restrict__ open, double *__restrict__ changed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nx) return;
    const int k0 = blockIdx.z * kRun, k1 = min(k0 + kRun, nz);
    const size_t sxy = (size_t)nx * ny;
    T s_last = T(1), q_last = T(1);
    size_t c = (size_t)k0 * sxy + (size_t)j * nx + i;
    T bz_lo = bz[c];
    // a cell's loads at once; the next cell's issued before this one's stores
    struct In {
        T x0, x1, y0, y1, zh;
        uint8_t ob;
    };
    auto load = [&](size_t cc, int kk) {
        In v;
        v.x0 = bx[cc];
        v.x1 = (i < nx - 1) ? bx[cc + 1] : T(0);
        v.y0 = by[cc];
        v.y1 = (j < ny - 1) ? by[cc + nx] : T(0);
        v.zh = (kk < nz - 1) ? bz[cc + sxy] : T(0);
        v.ob = open ? open[cc] : 0;
        return v;
    };
    In cur = load(c, k0);
    for (int k = k0; k < k1; k++, c += sxy) {
        const In nxt = k + 1 < k1 ? load(c + sxy, k + 1) : cur;
        const T bz_hi = cur.zh;
        T s = cur.x0;
        s += cur.x1;
        s += cur.y0;
        s += cur.y1;
        s += bz_lo;
        s += bz_hi;
        if (op.dinv) {
            op.dinv[c] = mul_s2(s, scale);
            op.bx[c] = mul_s2(cur.x0, scale);
            op.by[c] = mul_s2(cur.y0, scale);
            op.bz[c] = mul_s2(bz_lo, scale);
        }
        if (open) {
            const uint8_t bits = (uint8_t)((pos_bits(cur.x0) ? 1 : 0) | (pos_bits(cur.y0) ? 2 : 0) | (pos_bits(bz_lo) ? 4 : 0));
            if (cur.ob != bits) {
                open[c] = bits;
                *changed = 1.0;
            }
        }
        cur = nxt;
        bz_lo = bz_hi;
        T q = T(0);
        if (s > T(0)) {
            if (!same_bits(s, s_last)) {
                s_last = s;
                q_last = div_call(T(1), s);
            }
            q = q_last;
        }
        dinv[c] = q;
    }
}

// Coarse face coefficient = mean of the 2x2 coplanar fine faces it covers.
__global__ void k_restrict_coeffs(int nx, int ny, int nz, const double *__restrict__ bx,
                                  const double *__restrict__ by, const double *__restrict__ bz,
                                  double *__restrict__ cbx, double *__restrict__ cby, double *__restrict__ cbz)
{
    const int NX = nx / 2, NY = ny / 2;
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y, K = blockIdx.z;
    if (I >= NX) return;
    const size_t sxy = (size_t)nx * ny;
    const size_t f = (size_t)(2 * K) * sxy + (size_t)(2 * J) * nx + 2 * I;  // fine cell (2I, 2J, 2K)
    const size_t C = ((size_t)K * NY + J) * NX + I;
    cbx[C] = 0.25 * (((bx[f] + bx[f + nx]) + bx[f + sxy]) + bx[f + sxy + nx]);
    cby[C] = 0.25 * (((by[f] + by[f + 1]) + by[f + sxy]) + by[f + sxy + 1]);
    cbz[C] = 0.25 * (((bz[f] + bz[f + 1]) + bz[f + nx]) + bz[f + nx + 1]);
}

// Inverse diagonal of a smoothing update: FP64 levels use the stored 1/sum(beta); FP32 levels
// form 1/sum from the six face coefficients already loaded (sum in the order of k_diag_inv),
// which saves reading dinv.
template <typename T>
__device__ __forceinline__ T inv_diag(T stored, T bxl, T bxh, T byl, T byh, T bzl, T bzh)
{
    if (sizeof(T) == 8) return stored;
    const T sum = ((((bxl + bxh) + byl) + byh) + bzl) + bzh;
    return sum > T(0) ? T(1) / sum : T(0);
}

// ---------------------------------------------------------------------------
// Red-black Gauss-Seidel, one colour ((i+j+k) mod 2 == colour).  Each thread
// owns the one cell of that colour in an x-pair of a row:
//     p_c = dinv_c * (sum_f beta_f p_nb - h^2 b_c),  sum order x-,x+,y-,y+,z-,z+,
// products accumulated with fused multiply-adds in that order.
// ---------------------------------------------------------------------------
// one cell's update (shared by k_smooth and the coarse tail, so both round alike).  STORED: take
// 1/sum from L.dinv also in FP32, where the hierarchy stores exactly inv_diag's value.  ZERO: the
// iterate is zero (the first pass of a cycle from a zero guess): the neighbours are not read, the
// products with +0 give the +0 sum the loads of a zeroed array would
template <typename T, bool STORED = false, bool ZERO = false>
__device__ __forceinline__ void smooth_cell(int i, int j, int k, int nx, int ny, int nz, T h2, const LevelArrays<T> &L,
                                            const T *b, T *p)
{
    const size_t sxy = (size_t)nx * ny;
    const size_t c = (size_t)k * sxy + (size_t)j * nx + i;
    T s = T(0);
    const T bxl = L.bx[c], bxh = (i < nx - 1) ? L.bx[c + 1] : T(0);
    const T byl = L.by[c], byh = (j < ny - 1) ? L.by[c + nx] : T(0);
    const T bzl = L.bz[c], bzh = (k < nz - 1) ? L.bz[c + sxy] : T(0);
    auto nb = [&](size_t q) { return ZERO ? T(0) : p[q]; };
    if (i > 0) s = fma(bxl, nb(c - 1), s);
    if (i < nx - 1) s = fma(bxh, nb(c + 1), s);
    if (j > 0) s = fma(byl, nb(c - nx), s);
    if (j < ny - 1) s = fma(byh, nb(c + nx), s);
    if (k > 0) s = fma(bzl, nb(c - sxy), s);
    if (k < nz - 1) s = fma(bzh, nb(c + sxy), s);
    const T d = (STORED || sizeof(T) == 8) ? L.dinv[c] : inv_diag<T>(T(0), bxl, bxh, byl, byh, bzl, bzh);
    p[c] = d * fma(-h2, b[c], s);
}

template <typename T, bool ZERO>
__global__ void k_smooth(int nx, int ny, int nz, T h2, LevelArrays<T> L, const T *__restrict__ b,
                         T *__restrict__ p, int colour, int z0)
{
    const int j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z + z0;
    const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ((j + k + colour) & 1);
    if (i >= nx || j >= ny) return;
    if (!ck_cell(((long long)k * ny + j) * nx + i, i, j, k, nx, ny, nz, CK_SMOOTH)) return;
    smooth_cell<T, true, ZERO>(i, j, k, nx, ny, nz, h2, L, b, p);
}

// Colour-split layout (Split in mg_internal.cuh): slot of natural cell c in a row of parity
// q = (j + k) & 1, whose colour is (c & 1) ^ q (rows start at even indices).
__device__ __forceinline__ size_t split_slot(size_t c, int q, size_t half)
{
    return (((int)(c & 1) ^ q) ? half : 0) + (c >> 1);
}
__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv &f)
{
    const unsigned t = __umulhi(n, f.mult);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}
// parity (j + k) & 1 of the row holding natural index c
__device__ __forceinline__ int row_parity(unsigned c, const Split &sp)
{
    const unsigned row = fdiv(c, sp.fnx), k = fdiv(row, sp.fny), j = row - k * (unsigned)sp.ny;
    return (int)((j + k) & 1u);
}

// Uniform rows.  Away from the interface and the body, every face coefficient around an x-row of
// cells holds one value (pure air or pure water).  urow[k*ny + j] = that value v when the row is
// interior (0 < j < ny-1, 0 < k < nz-1) and every face of every cell of row (j,k) except the two x-walls (bx at i = 0 and the high face of i = nx-1,
// both walls, stored as 0) equals v bitwise, else 0; one warp per row.  A pass that reads urow[r]
// != 0 takes its face values from it instead of loading them: the same values, so the same results.
// On a grid stretched in z the metric factors differ per axis, and a row away from the interface
// holds four values instead: vx on its x-faces, vy on its low and high y-faces, vzl on its low and
// vzh on its high z-faces.  arow[r] (optional) = {vx, vy, vzl, vzh} for such a "banded" row, else
// zeros; count[0] and count[1] (optional) receive the numbers of uniform rows and of banded rows
// that are not uniform.
__global__ void k_uniform_rows(int nx, int ny, int nz, const float *__restrict__ bx, const float *__restrict__ by,
                               const float *__restrict__ bz, float *__restrict__ urow, float4 *__restrict__ arow,
                               unsigned *__restrict__ count)
{
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * warps + (threadIdx.x >> 5);
    if (r >= ny * nz) return;
    const int j = r % ny, k = r / ny;
    const size_t sxy = (size_t)nx * ny, c0 = (size_t)r * nx;
    const bool inner = j > 0 && k > 0 && j < ny - 1 && k < nz - 1;
    const float vy = by[c0], vx = nx > 1 ? bx[c0 + 1] : vy, vzl = bz[c0], vzh = inner ? bz[c0 + sxy] : 0.f;
    const int bxv = __float_as_int(vx), byv = __float_as_int(vy), bzl = __float_as_int(vzl),
              bzh = __float_as_int(vzh);
    bool ok = inner && vx > 0.f && vy > 0.f && vzl > 0.f && vzh > 0.f;
    if (ok)  // warp-uniform; the loads of a lane's cells are independent of one another
        for (int i = lane; i < nx; i += 32) {
            const size_t c = c0 + i;
            const bool cell = (i == 0 || __float_as_int(bx[c]) == bxv) & (__float_as_int(by[c]) == byv) &
                              (__float_as_int(by[c + nx]) == byv) & (__float_as_int(bz[c]) == bzl) &
                              (__float_as_int(bz[c + sxy]) == bzh);
            ok = ok & cell;
        }
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) {
        const bool uni = ok && bxv == byv && bzl == byv && bzh == byv;
        urow[r] = uni ? vy : 0.f;
        if (arow) arow[r] = ok ? make_float4(vx, vy, vzl, vzh) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (count && ok) atomicAdd(&count[uni ? 0 : 1], 1u);
    }
}

// One colour of red-black Gauss-Seidel on the colour-split layout (FP32, all dims even): the
// cell's six neighbours are the other colour's slots m-1+(i&1), m+(i&1), m -+ nx/2, m -+ nx*ny/2
// (m = c >> 1), read contiguously; b and the result are the own colour's slot m.  A pass moves
// the face coefficients (none on uniform rows), half of p and half of b instead of all of p and
// b.  Same arithmetic, in the same order, as k_smooth<float>.  Used where nx % 8 != 0
// (k_smooth_split4 otherwise).
__global__ void k_smooth_split(int nx, int ny, int nz, float h2, LevelArrays<float> L, const float *__restrict__ b,
                               float *__restrict__ p, int colour, const float *__restrict__ urow, int rev, int zero)
{
    const int j = rev ? ny - 1 - (int)blockIdx.y : (int)blockIdx.y, k = rev ? nz - 1 - (int)blockIdx.z : (int)blockIdx.z;
    const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ((j + k + colour) & 1);
    if (i >= nx) return;
    const size_t sxy = (size_t)nx * ny, half = sxy * nz / 2;
    const size_t c = (size_t)k * sxy + (size_t)j * nx + i;
    const size_t m = c >> 1, hx = nx / 2, hxy = sxy / 2;
    const float *__restrict__ o = p + (colour ? 0 : half);  // the other colour
    const int odd = i & 1;
    const size_t own = (colour ? half : 0) + m;
    if (!(ck_cell((long long)c, i, j, k, nx, ny, nz, CK_SMOOTH_SPLIT) && MG_CK(m, m, half, CK_SMOOTH_SPLIT) &&
          (i == 0 || MG_CK(m - 1 + odd, m - 1 + odd, half, CK_SMOOTH_SPLIT)) &&
          (i >= nx - 1 || MG_CK(m + odd, m + odd, half, CK_SMOOTH_SPLIT)) &&
          (j == 0 || MG_CK((long long)m - (long long)hx, m, half, CK_SMOOTH_SPLIT)) &&
          (j >= ny - 1 || MG_CK(m, m + hx, half, CK_SMOOTH_SPLIT)) &&
          (k == 0 || MG_CK((long long)m - (long long)hxy, m, half, CK_SMOOTH_SPLIT)) &&
          (k >= nz - 1 || MG_CK(m, m + hxy, half, CK_SMOOTH_SPLIT))))
        return;
    // the neighbours and b are loaded before the row's uniform value is known, so a uniform row
    // waits for one memory round trip, not two
    const float v = urow ? urow[(size_t)k * ny + j] : 0.f;
    // zero: the iterate is zero (first pass of a cycle from a zero guess), nothing to read
    const float pxm = (!zero && i > 0) ? o[m - 1 + odd] : 0.f, pxp = (!zero && i < nx - 1) ? o[m + odd] : 0.f;
    const float pym = (!zero && j > 0) ? o[m - hx] : 0.f, pyp = (!zero && j < ny - 1) ? o[m + hx] : 0.f;
    const float pzm = (!zero && k > 0) ? o[m - hxy] : 0.f, pzp = (!zero && k < nz - 1) ? o[m + hxy] : 0.f;
    const float bv = b[own];
    float bxl, bxh, byl, byh, bzl, bzh;
    if (v != 0.f) {  // uniform row: the stored values, x-walls 0
        bxl = i > 0 ? v : 0.f;
        bxh = i < nx - 1 ? v : 0.f;
        byl = byh = bzl = bzh = v;
    } else {
        bxl = L.bx[c];
        bxh = (i < nx - 1) ? L.bx[c + 1] : 0.f;
        byl = L.by[c];
        byh = (j < ny - 1) ? L.by[c + nx] : 0.f;
        bzl = L.bz[c];
        bzh = (k < nz - 1) ? L.bz[c + sxy] : 0.f;
    }
    float s = 0.f;
    if (i > 0) s = fmaf(bxl, pxm, s);
    if (i < nx - 1) s = fmaf(bxh, pxp, s);
    if (j > 0) s = fmaf(byl, pym, s);
    if (j < ny - 1) s = fmaf(byh, pyp, s);
    if (k > 0) s = fmaf(bzl, pzm, s);
    if (k < nz - 1) s = fmaf(bzh, pzp, s);
    p[own] = inv_diag<float>(0.f, bxl, bxh, byl, byh, bzl, bzh) * fmaf(-h2, bv, s);
}

// The same colour pass, four consecutive cells of the colour per thread (nx % 8 == 0): the cells'
// slots mb..mb+3 are float4-aligned in the colour-split arrays, so the x-neighbours (one float4
// and one scalar), the y and z neighbours, b and the results move as float4.  Four independent
// updates per thread keep more loads in flight than one, which the pass needs once uniform rows
// have removed most of its bytes.  Each cell's arithmetic is k_smooth_split's, in its order.
// OFF = (j + k + colour) & 1, the x offset of the colour in the row (uniform across a warp).
// BAND: the row's record is {vx, vy, vzl, vzh} of a banded row (all four equal on a uniform row,
// zeros elsewhere), else {v, v, v, v} from urow.  A row with a record is interior (0 < j < ny-1,
// 0 < k < nz-1: k_uniform_rows), so its update needs no y or z wall tests, which keeps the
// record path short; the neighbours are loaded before the record is known, under the wall tests
// any row needs.  Rows without a record take their faces from S, the colour-split copies of the
// face arrays: a cell's low faces are the own colour's slots, its high faces the low faces of its
// +x, +y and +z neighbours, i.e. the other colour's slots of its x-neighbour (as for p), mb + hx
// and mb + hxy; six float4 and one scalar, each value used.
template <int OFF, bool BAND, bool ZERO>
__device__ __forceinline__ void split4_body(int nx, int ny, int nz, float h2, const LevelArrays<float> &S,
                                            const float *__restrict__ b, float *__restrict__ p, int colour, float4 rv,
                                            int g, int j, int k)
{
    const float v = rv.x;
    const int G = nx / 8;
    const size_t sxy = (size_t)nx * ny, half = sxy * nz / 2, hx = nx / 2, hxy = sxy / 2;
    const size_t mb = ((size_t)k * sxy + (size_t)j * nx) / 2 + 4 * g;
    const float *__restrict__ o = p + (colour ? 0 : half);
    float *own = p + (colour ? half : 0);
    const float *bo = b + (colour ? half : 0);
    const size_t so = colour ? half : 0, sn = colour ? 0 : half;  // own and other colour in S
    {
        const long long n = (long long)sxy * nz, m = (long long)mb;
        (void)n;
        (void)m;
        if (!(MG_CK(m, m + 3, half, CK_SMOOTH_SPLIT4) &&
              (OFF ? (g >= G - 1 || MG_CK(m + 4, m + 4, half, CK_SMOOTH_SPLIT4))
                   : (g == 0 || MG_CK(m - 1, m - 1, half, CK_SMOOTH_SPLIT4))) &&
              (j == 0 || MG_CK(m - (long long)hx, m - (long long)hx + 3, half, CK_SMOOTH_SPLIT4)) &&
              (j >= ny - 1 || MG_CK(m + hx, m + hx + 3, half, CK_SMOOTH_SPLIT4)) &&
              (k == 0 || MG_CK(m - (long long)hxy, m - (long long)hxy + 3, half, CK_SMOOTH_SPLIT4)) &&
              (k >= nz - 1 || MG_CK(m + hxy, m + hxy + 3, half, CK_SMOOTH_SPLIT4)) &&
              (v != 0.f || (MG_CK(so + m, so + m + 3, n, CK_SMOOTH_SPLIT4) &&
                            MG_CK(sn + m, sn + m + 3 + ((OFF && g < G - 1) ? 1 : 0), n, CK_SMOOTH_SPLIT4) &&
                            (j >= ny - 1 || MG_CK(sn + m + hx, sn + m + hx + 3, n, CK_SMOOTH_SPLIT4)) &&
                            (k >= nz - 1 || MG_CK(sn + m + hxy, sn + m + hxy + 3, n, CK_SMOOTH_SPLIT4))))))
            return;
    }
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // ZERO: the other colour is zero (first pass of a cycle from a zero guess), nothing to read
    const float4 ox = ZERO ? zero4 : *reinterpret_cast<const float4 *>(o + mb);
    const float oxe = ZERO ? 0.f : (OFF ? ((g < G - 1) ? o[mb + 4] : 0.f) : ((g > 0) ? o[mb - 1] : 0.f));
    const float4 oym = (!ZERO && j > 0) ? *reinterpret_cast<const float4 *>(o + mb - hx) : zero4;
    const float4 oyp = (!ZERO && j < ny - 1) ? *reinterpret_cast<const float4 *>(o + mb + hx) : zero4;
    const float4 ozm = (!ZERO && k > 0) ? *reinterpret_cast<const float4 *>(o + mb - hxy) : zero4;
    const float4 ozp = (!ZERO && k < nz - 1) ? *reinterpret_cast<const float4 *>(o + mb + hxy) : zero4;
    // b of this colour is read next a sweep later: loaded evict-first, so that it leaves L2 to the
    // iterate the next pass reads
    const float4 bv = __ldcs(reinterpret_cast<const float4 *>(bo + mb));
    const float xs[6] = {OFF ? 0.f : oxe, ox.x, ox.y, ox.z, ox.w, OFF ? oxe : 0.f};  // slots mb-1 .. mb+4
    const float oy0[4] = {oym.x, oym.y, oym.z, oym.w}, oy1[4] = {oyp.x, oyp.y, oyp.z, oyp.w};
    const float oz0[4] = {ozm.x, ozm.y, ozm.z, ozm.w}, oz1[4] = {ozp.x, ozp.y, ozp.z, ozp.w};
    const float bb[4] = {bv.x, bv.y, bv.z, bv.w};
    float out[4];
    if (v != 0.f) {
        // a row with a record: the diagonal is 6v, or 5v at an x-wall (the sums of inv_diag, in its
        // order: 0 + v = v + 0 = v), so two divisions serve the thread's four cells; on a banded
        // row the same with vx, vy, vzl, vzh in their places
        const float vx = BAND ? rv.x : v, vy = BAND ? rv.y : v, vzl = BAND ? rv.z : v, vzh = BAND ? rv.w : v;
        float inv6, inv5;
        if (BAND) {
            inv6 = 1.f / ((((((vx + vx) + vy) + vy) + vzl) + vzh));
            inv5 = 1.f / ((((vx + vy) + vy) + vzl) + vzh);
        } else {
            const float s5 = (((v + v) + v) + v) + v;
            inv6 = 1.f / (s5 + v);
            inv5 = 1.f / s5;
        }
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const int i = 8 * g + 2 * t + OFF;
            const float pxm = xs[t + OFF], pxp = xs[t + 1 + OFF];  // slots mb+t-1+OFF, mb+t+OFF
            float s = 0.f;
            if (i > 0) s = fmaf(vx, pxm, s);
            if (i < nx - 1) s = fmaf(vx, pxp, s);
            s = fmaf(vy, oy0[t], s);
            s = fmaf(vy, oy1[t], s);
            s = fmaf(vzl, oz0[t], s);
            s = fmaf(vzh, oz1[t], s);
            const float dinv = (i > 0 && i < nx - 1) ? inv6 : inv5;
            out[t] = dinv * fmaf(-h2, bb[t], s);
        }
    } else {
        const float4 xl = *reinterpret_cast<const float4 *>(S.bx + so + mb);
        const float4 yl = *reinterpret_cast<const float4 *>(S.by + so + mb);
        const float4 zl = *reinterpret_cast<const float4 *>(S.bz + so + mb);
        const float4 xh = *reinterpret_cast<const float4 *>(S.bx + sn + mb);
        const float xe = (OFF && g < G - 1) ? S.bx[sn + mb + 4] : 0.f;
        const float4 yh = (j < ny - 1) ? *reinterpret_cast<const float4 *>(S.by + sn + mb + hx) : zero4;
        const float4 zh = (k < nz - 1) ? *reinterpret_cast<const float4 *>(S.bz + sn + mb + hxy) : zero4;
        const float fxl[4] = {xl.x, xl.y, xl.z, xl.w}, fxh[5] = {xh.x, xh.y, xh.z, xh.w, xe};
        const float fyl[4] = {yl.x, yl.y, yl.z, yl.w}, fyh[4] = {yh.x, yh.y, yh.z, yh.w};
        const float fzl[4] = {zl.x, zl.y, zl.z, zl.w}, fzh[4] = {zh.x, zh.y, zh.z, zh.w};
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const int i = 8 * g + 2 * t + OFF;
            // high x-face: the other colour's slot mb+t+OFF, the x-neighbour's low face
            const float bxl = fxl[t], bxh = i < nx - 1 ? fxh[t + OFF] : 0.f;
            const float byl = fyl[t], byh = fyh[t], bzl = fzl[t], bzh = fzh[t];
            const float pxm = xs[t + OFF], pxp = xs[t + 1 + OFF];
            float s = 0.f;
            if (i > 0) s = fmaf(bxl, pxm, s);
            if (i < nx - 1) s = fmaf(bxh, pxp, s);
            if (j > 0) s = fmaf(byl, oy0[t], s);
            if (j < ny - 1) s = fmaf(byh, oy1[t], s);
            if (k > 0) s = fmaf(bzl, oz0[t], s);
            if (k < nz - 1) s = fmaf(bzh, oz1[t], s);
            out[t] = inv_diag<float>(0.f, bxl, bxh, byl, byh, bzl, bzh) * fmaf(-h2, bb[t], s);
        }
    }
    *reinterpret_cast<float4 *>(own + mb) = make_float4(out[0], out[1], out[2], out[3]);
}
template <bool BAND, bool ZERO>
__global__ void k_smooth_split4(int nx, int ny, int nz, float h2, LevelArrays<float> S, const float *__restrict__ b,
                                float *__restrict__ p, int colour, const float *__restrict__ urow,
                                const float4 *__restrict__ arow, int rev)
{
    // rev: the blocks take the planes (and rows) in descending order, so that a pass that follows
    // an ascending one starts on the data that pass touched last (still in L2)
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int by = rev ? (int)gridDim.y - 1 - (int)blockIdx.y : (int)blockIdx.y;
    // the planes of the four quarters interleaved in the block order (0, nz/4, nz/2, 3nz/4, 1, ...):
    // the rows without a record gather in a band of planes (an interface), and interleaving runs
    // their face-loading blocks alongside blocks of record rows instead of all together
    const int zb = rev ? (int)gridDim.z - 1 - (int)blockIdx.z : (int)blockIdx.z;
    const int qz = nz / 4;
    const int k = (nz & 3) ? zb : (zb & 3) * qz + (zb >> 2);
    const int j = by * blockDim.y + threadIdx.y;
    if (g >= nx / 8 || j >= ny) return;
    float4 rv;
    if (BAND) {
        rv = arow[(size_t)k * ny + j];
    } else {
        const float v = urow ? urow[(size_t)k * ny + j] : 0.f;
        rv = make_float4(v, v, v, v);
    }
    if ((j + k + colour) & 1) split4_body<1, BAND, ZERO>(nx, ny, nz, h2, S, b, p, colour, rv, g, j, k);
    else split4_body<0, BAND, ZERO>(nx, ny, nz, h2, S, b, p, colour, rv, g, j, k);
}

// r = b - h^-2 sum_f beta_f (p_nb - p_c) at one fine cell (sum order x-,x+,y-,y+,z-,z+).
template <typename T>
__device__ __forceinline__ T residual_at(int i, int j, int k, size_t c, int nx, int ny, int nz, size_t sxy, T ih2,
                                         const LevelArrays<T> &L, const T *b, const T *p)
{
    if (!ck_cell((long long)c, i, j, k, nx, ny, nz, CK_RESID)) return T(0);
    const T pc = p[c];
    T s = T(0);
    if (i > 0) s = fma(L.bx[c], p[c - 1] - pc, s);
    if (i < nx - 1) s = fma(L.bx[c + 1], p[c + 1] - pc, s);
    if (j > 0) s = fma(L.by[c], p[c - nx] - pc, s);
    if (j < ny - 1) s = fma(L.by[c + nx], p[c + nx] - pc, s);
    if (k > 0) s = fma(L.bz[c], p[c - sxy] - pc, s);
    if (k < nz - 1) s = fma(L.bz[c + sxy], p[c + sxy] - pc, s);
    return fma(-s, ih2, b[c]);
}

// FP64 residual for the solver's convergence checks.  Where p and its in-domain neighbours are
// all zero (bitwise, either sign) every product beta (0 - 0) is a signed zero, the sum stays +0
// and residual_at returns b[c] exactly (for finite coefficients): the test runs on the integer
// pipe and skips the FP64 arithmetic, which dominates this pass on a zero initial guess.
__device__ __forceinline__ double residual64_at(int i, int j, int k, size_t c, int nx, int ny, int nz, size_t sxy,
                                                double ih2, const LevelArrays<double> &L,
                                                const double *__restrict__ b, const double *__restrict__ p)
{
    unsigned long long z = __double_as_longlong(p[c]);
    if (i > 0) z |= __double_as_longlong(p[c - 1]);
    if (i < nx - 1) z |= __double_as_longlong(p[c + 1]);
    if (j > 0) z |= __double_as_longlong(p[c - nx]);
    if (j < ny - 1) z |= __double_as_longlong(p[c + nx]);
    if (k > 0) z |= __double_as_longlong(p[c - sxy]);
    if (k < nz - 1) z |= __double_as_longlong(p[c + sxy]);
    if ((z << 1) == 0ull) return b[c];
    return residual_at<double>(i, j, k, c, nx, ny, nz, sxy, ih2, L, b, p);
}

// Residual and cell-centred full weighting: coarse b = mean of the 8 children's residuals.
template <typename T>
__device__ __forceinline__ void restrict_cell(int I, int J, int K, int nx, int ny, int nz, T ih2,
                                              const LevelArrays<T> &L, const T *b, const T *p, T *bc)
{
    const int NX = nx / 2, NY = ny / 2;
    const size_t sxy = (size_t)nx * ny;
    if (!MG_CK(((long long)K * NY + J) * NX + I, ((long long)K * NY + J) * NX + I, (long long)NX * NY * (nz / 2),
               CK_RESTRICT))
        return;
    T s = T(0);
#pragma unroll
    for (int dk = 0; dk < 2; dk++)
#pragma unroll
        for (int dj = 0; dj < 2; dj++)
#pragma unroll
            for (int di = 0; di < 2; di++) {
                const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
                const size_t c = (size_t)k * sxy + (size_t)j * nx + i;
                s += residual_at<T>(i, j, k, c, nx, ny, nz, sxy, ih2, L, b, p);
            }
    bc[((size_t)K * NY + J) * NX + I] = T(0.125) * s;
}

template <typename T>
__global__ void k_resid_restrict(int nx, int ny, int nz, T ih2, LevelArrays<T> L, const T *__restrict__ b,
                                 const T *__restrict__ p, T *__restrict__ bc)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y, K = blockIdx.z;
    if (I >= nx / 2 || J >= ny / 2) return;
    restrict_cell<T>(I, J, K, nx, ny, nz, ih2, L, b, p, bc);
}

template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

// The same residual + full weighting for FP32, reading each coarse cell's 2x2x2 children as four
// x-pairs: every row it touches (the children's rows, their y and z neighbour rows, the x halo
// cells, the face rows) is loaded once as a pair, 44 loads per coarse cell instead of 112
// stride-2 scalar loads, which made the per-cell form bound by L1 wavefronts.  Each child's
// residual takes residual_at's terms and conditions in residual_at's order, and the 8 are summed
// in the same order, so the result is identical.  Arrays 16-byte aligned, fine dims even.
template <bool SPLIT>
__global__ void k_resid_restrict_pairs(int nx, int ny, int nz, float ih2, LevelArrays<float> L,
                                       const float *__restrict__ b, const float *__restrict__ p,
                                       float *__restrict__ bc, size_t half, const float *__restrict__ urow,
                                       int rev)
{
    const int NX = nx / 2, NY = ny / 2;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int Jb = blockIdx.y * blockDim.y + threadIdx.y;
    const int J = rev ? NY - 1 - Jb : Jb;
    // coarse planes of the four quarters interleaved in the block order, as in the colour passes
    const int NZ = nz / 2, zb = rev ? NZ - 1 - (int)blockIdx.z : (int)blockIdx.z;
    const int K = (NZ & 3) ? zb : (zb & 3) * (NZ / 4) + (zb >> 2);
    if (I >= NX || Jb >= NY) return;
    const size_t sxy = (size_t)nx * ny;
    const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * K;
    const bool xhi = i0 + 2 < nx, ylo = j0 > 0, yhi = j0 + 2 < ny, zlo = k0 > 0, zhi = k0 + 2 < nz;
    {
        // the lowest and highest fine cells any load reaches: (i0 - 1, j0 - 1 | j0, k0 - 1 | k0) ...
        // (i0 + 2, j0 + 2, k0 + 1) within the guards, and the coarse cell
        const long long n = (long long)sxy * nz;
        const long long lo = ((long long)(k0 - (zlo ? 1 : 0)) * ny + j0 - (ylo ? 1 : 0)) * nx + i0 - (i0 > 0 ? 1 : 0);
        const long long hi = ((long long)(k0 + (zhi ? 2 : 1)) * ny + j0 + (yhi ? 2 : 1)) * nx + i0 + (xhi ? 2 : 1);
        (void)n;
        (void)lo;
        (void)hi;
        if (!(MG_CK(lo, hi, n, CK_RESTRICT_PAIRS) &&
              MG_CK(((long long)K * NY + J) * NX + I, ((long long)K * NY + J) * NX + I, (long long)NX * NY * (nz / 2),
                    CK_RESTRICT_PAIRS) &&
              (!SPLIT || MG_CK(lo >> 1, hi >> 1, (long long)half, CK_RESTRICT_PAIRS))))
            return;
    }
    auto ld2 = [](const float *a, size_t c) { return *reinterpret_cast<const float2 *>(a + c); };
    // p and b pairs: natural, or the two colours' slots c >> 1 (row parity q decides the order)
    auto ldf2 = [&](const float *a, size_t c, int q) {
        if (!SPLIT) return ld2(a, c);
        const size_t m = c >> 1;
        return q ? make_float2(a[half + m], a[m]) : make_float2(a[m], a[half + m]);
    };
    auto ldf = [&](const float *a, size_t c, int q) { return SPLIT ? a[split_slot(c, q, half)] : a[c]; };
    const float2 zero2 = make_float2(0.f, 0.f);
    // row base of fine row (j, k) at x = i0, and its parity
    auto row = [&](int j, int k) { return (size_t)k * sxy + (size_t)j * nx + i0; };
    auto par = [](int j, int k) { return (j + k) & 1; };
    float2 pc[2][2], bb[2][2], fx[2][2];
    float pxm[2][2], pxp[2][2], fxp[2][2];
    float2 fy[2][3], fz[2][3];      // fy[dk][row j0, j0+1, j0+2], fz[dj][plane k0, k0+1, k0+2]
    float2 pym[2], pyp[2], pzm[2], pzp[2];  // pym[dk] = p(j0-1, k0+dk) ...; pzm[dj] = p(j0+dj, k0-1) ...
    // the four fine rows uniform with one value: every face this cell reads is that value (the
    // uniform rows' y+ and z+ faces included), x-walls 0
    float v = 0.f;
    if (urow) {
        const float u00 = urow[(size_t)k0 * ny + j0], u10 = urow[(size_t)k0 * ny + j0 + 1];
        const float u01 = urow[(size_t)(k0 + 1) * ny + j0], u11 = urow[(size_t)(k0 + 1) * ny + j0 + 1];
        if (u00 != 0.f && u00 == u10 && u00 == u01 && u00 == u11) v = u00;
    }
    const float2 v2 = make_float2(v, v);
#pragma unroll
    for (int dk = 0; dk < 2; dk++)
#pragma unroll
        for (int dj = 0; dj < 2; dj++) {
            const size_t c = row(j0 + dj, k0 + dk);
            const int q = par(j0 + dj, k0 + dk);
            pc[dj][dk] = ldf2(p, c, q);
            bb[dj][dk] = ldf2(b, c, q);
            pxm[dj][dk] = i0 > 0 ? ldf(p, c - 1, q) : 0.f;
            pxp[dj][dk] = xhi ? ldf(p, c + 2, q) : 0.f;
            if (v != 0.f) {
                fx[dj][dk] = make_float2(i0 > 0 ? v : 0.f, v);
                fxp[dj][dk] = xhi ? v : 0.f;
            } else {
                fx[dj][dk] = ld2(L.bx, c);
                fxp[dj][dk] = xhi ? L.bx[c + 2] : 0.f;
            }
        }
#pragma unroll
    for (int dk = 0; dk < 2; dk++) {
        if (v != 0.f) {
            fy[dk][0] = fy[dk][1] = fy[dk][2] = v2;
        } else {
            fy[dk][0] = ld2(L.by, row(j0, k0 + dk));
            fy[dk][1] = ld2(L.by, row(j0 + 1, k0 + dk));
            fy[dk][2] = yhi ? ld2(L.by, row(j0 + 2, k0 + dk)) : zero2;
        }
        pym[dk] = ylo ? ldf2(p, row(j0 - 1, k0 + dk), par(j0 - 1, k0 + dk)) : zero2;
        pyp[dk] = yhi ? ldf2(p, row(j0 + 2, k0 + dk), par(j0 + 2, k0 + dk)) : zero2;
    }
#pragma unroll
    for (int dj = 0; dj < 2; dj++) {
        if (v != 0.f) {
            fz[dj][0] = fz[dj][1] = fz[dj][2] = v2;
        } else {
            fz[dj][0] = ld2(L.bz, row(j0 + dj, k0));
            fz[dj][1] = ld2(L.bz, row(j0 + dj, k0 + 1));
            fz[dj][2] = zhi ? ld2(L.bz, row(j0 + dj, k0 + 2)) : zero2;
        }
        pzm[dj] = zlo ? ldf2(p, row(j0 + dj, k0 - 1), par(j0 + dj, k0 - 1)) : zero2;
        pzp[dj] = zhi ? ldf2(p, row(j0 + dj, k0 + 2), par(j0 + dj, k0 + 2)) : zero2;
    }
    auto comp = [](float2 v, int d) { return d ? v.y : v.x; };
    float sum = 0.f;
#pragma unroll
    for (int dk = 0; dk < 2; dk++)
#pragma unroll
        for (int dj = 0; dj < 2; dj++)
#pragma unroll
            for (int di = 0; di < 2; di++) {
                const int i = i0 + di, j = j0 + dj, k = k0 + dk;
                const float pcv = comp(pc[dj][dk], di);
                float s = 0.f;
                if (i > 0) s = fmaf(comp(fx[dj][dk], di), (di ? pc[dj][dk].x : pxm[dj][dk]) - pcv, s);
                if (i < nx - 1) s = fmaf(di ? fxp[dj][dk] : fx[dj][dk].y, (di ? pxp[dj][dk] : pc[dj][dk].y) - pcv, s);
                if (j > 0) s = fmaf(comp(fy[dk][dj], di), comp(dj ? pc[0][dk] : pym[dk], di) - pcv, s);
                if (j < ny - 1) s = fmaf(comp(fy[dk][dj + 1], di), comp(dj ? pyp[dk] : pc[1][dk], di) - pcv, s);
                if (k > 0) s = fmaf(comp(fz[dj][dk], di), comp(dk ? pc[dj][0] : pzm[dj], di) - pcv, s);
                if (k < nz - 1) s = fmaf(comp(fz[dj][dk + 1], di), comp(dk ? pzp[dj] : pc[dj][1], di) - pcv, s);
                sum += fmaf(-s, ih2, comp(bb[dj][dk], di));
            }
    bc[((size_t)K * NY + J) * NX + I] = 0.125f * sum;
}

// Trilinear cell-centred prolongation added to p (cells with no open face keep p): weights 3/4
// (parent) and 1/4 (next coarse cell on the fine cell's side) per axis; that index clamps at
// walls.  One thread per coarse cell handles its 2x2x2 children as four x-pairs: the 3x3x3 coarse
// neighbourhood is loaded once and every fine load is issued before the dead-cell test, so a
// thread keeps 8 pair loads in flight (one load per thread, then a dependent one, leaves the pass
// bound by memory latency).  A child's 8 products w_z w_y w_x e are summed with fma, z outermost
// and x innermost, the parent before the neighbour on each axis.  p and dinv are aligned to a
// pair (16-byte aligned arrays, even nx).
// the trilinear corrections of coarse cell (I,J,K)'s 8 children, corr[dz][dy][dx]
template <typename T>
__device__ __forceinline__ void prolong_corr(int I, int J, int K, int NX, int NY, int NZ, const T *ec, T corr[2][2][2])
{
    // neighbourhood index 0 = lower neighbour (clamped), 1 = parent, 2 = upper neighbour (clamped)
    const int Is[3] = {max(I - 1, 0), I, min(I + 1, NX - 1)};
    const int Js[3] = {max(J - 1, 0), J, min(J + 1, NY - 1)};
    const int Ks[3] = {max(K - 1, 0), K, min(K + 1, NZ - 1)};
    if (!(MG_CK(((long long)Ks[0] * NY + Js[0]) * NX + Is[0], ((long long)Ks[2] * NY + Js[2]) * NX + Is[2],
                (long long)NX * NY * NZ, CK_PROLONG))) {
        for (int q = 0; q < 8; q++) (&corr[0][0][0])[q] = T(0);
        return;
    }
    T e[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int bb = 0; bb < 3; bb++)
#pragma unroll
            for (int d = 0; d < 3; d++) e[a][bb][d] = ec[((size_t)Ks[a] * NY + Js[bb]) * NX + Is[d]];
    const T w[2] = {T(0.75), T(0.25)};
#pragma unroll
    for (int dz = 0; dz < 2; dz++)
#pragma unroll
        for (int dy = 0; dy < 2; dy++)
#pragma unroll
            for (int dx = 0; dx < 2; dx++) {
                // parent first, then the neighbour on the child's side
                const int ka[2] = {1, dz ? 2 : 0}, jb[2] = {1, dy ? 2 : 0}, id[2] = {1, dx ? 2 : 0};
                T s = T(0);
#pragma unroll
                for (int a = 0; a < 2; a++)
#pragma unroll
                    for (int bb = 0; bb < 2; bb++)
#pragma unroll
                        for (int d = 0; d < 2; d++) s = fma(w[a] * w[bb] * w[d], e[ka[a]][jb[bb]][id[d]], s);
                corr[dz][dy][dx] = s;
            }
}

// urow (optional, the finest FP32 level): a fine row with a uniform value has every cell live, so
// its inverse diagonals are not read
template <typename T, bool SPLIT>
__global__ void k_prolong(int nx, int ny, int nz, const T *__restrict__ ec, const T *__restrict__ dinv,
                          T *__restrict__ p, size_t half, const float *__restrict__ urow)
{
    using P2 = typename Pair<T>::type;
    const int NX = nx / 2, NY = ny / 2, NZ = nz / 2;
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
    // on the colour-split finest level, coarse planes of the four quarters interleaved in the block
    // order, as in its colour passes and restriction
    const int zb = blockIdx.z;
    const int K = (SPLIT && (NZ & 3) == 0) ? (zb & 3) * (NZ / 4) + (zb >> 2) : zb;
    if (I >= NX || J >= NY) return;
    {
        const long long n = (long long)nx * ny * nz;
        const long long c0 = ((long long)(2 * K) * ny + 2 * J) * nx + 2 * I;
        const long long c1 = ((long long)(2 * K + 1) * ny + 2 * J + 1) * nx + 2 * I + 1;
        (void)n;
        (void)c0;
        (void)c1;
        if (!(MG_CK(c0, c1, n, CK_PROLONG) && (!SPLIT || MG_CK(c0 >> 1, c1 >> 1, (long long)half, CK_PROLONG))))
            return;
    }
    P2 dv[2][2], pv[2][2];
#pragma unroll
    for (int dz = 0; dz < 2; dz++)
#pragma unroll
        for (int dy = 0; dy < 2; dy++) {
            const size_t c = ((size_t)(2 * K + dz) * ny + (2 * J + dy)) * nx + 2 * I;
            if (urow && urow[(size_t)(2 * K + dz) * ny + 2 * J + dy] != 0.f) {
                dv[dz][dy].x = T(1);
                dv[dz][dy].y = T(1);
            } else {
                dv[dz][dy] = *reinterpret_cast<const P2 *>(dinv + c);
            }
            if (SPLIT) {  // the pair's two colours at slot c >> 1 of each half
                const size_t m = c >> 1;
                const bool q = (2 * J + dy + 2 * K + dz) & 1;
                pv[dz][dy].x = p[(q ? half : 0) + m];
                pv[dz][dy].y = p[(q ? 0 : half) + m];
            } else {
                pv[dz][dy] = *reinterpret_cast<const P2 *>(p + c);
            }
        }
    T corr[2][2][2];
    prolong_corr<T>(I, J, K, NX, NY, NZ, ec, corr);
#pragma unroll
    for (int dz = 0; dz < 2; dz++)
#pragma unroll
        for (int dy = 0; dy < 2; dy++) {
            T out[2];
#pragma unroll
            for (int dx = 0; dx < 2; dx++) {
                const T dval = dx ? dv[dz][dy].y : dv[dz][dy].x;
                const T pold = dx ? pv[dz][dy].y : pv[dz][dy].x;
                out[dx] = zero_bits(dval) ? pold : pold + corr[dz][dy][dx];
            }
            const size_t c = ((size_t)(2 * K + dz) * ny + (2 * J + dy)) * nx + 2 * I;
            if (SPLIT) {
                const size_t m = c >> 1;
                const bool q = (2 * J + dy + 2 * K + dz) & 1;
                p[(q ? half : 0) + m] = out[0];
                p[(q ? 0 : half) + m] = out[1];
            } else {
                P2 o;
                o.x = out[0];
                o.y = out[1];
                *reinterpret_cast<P2 *>(p + c) = o;
            }
        }
}

// ---------------------------------------------------------------------------
// Fused red-black sweep: both colours in one pass over HBM.
//
// The CTA owns a TX x TY tile of columns and a chunk of z-planes and marches up
// the chunk with a two-plane wavefront: at step s it updates the FIRST colour on
// plane s, then the SECOND colour on plane s-1 (whose first-colour neighbours on
// planes s-2, s-1 and s are final by then).  It reads the iterate from p_old and
// writes every cell of its tile to p_new, so CTAs never see each other's writes:
// the first colour on a one-cell ring around the tile (and on one plane below
// and above the chunk) is recomputed from p_old, exactly as the neighbouring CTA
// computes it.  Per cell the arithmetic is that of k_smooth, so the result is
// bit-identical to two colour passes.  Threads: one per column of the tile plus a
// two-cell halo; ring 2 only loads, ring 1 also updates the first colour.
// Shared memory holds three rotating planes of (p, bx, by): the x+ and y+ face
// coefficients of a cell are its neighbour's low faces.
// ---------------------------------------------------------------------------
template <typename T, int TX, int TY>
__global__ void __launch_bounds__((TX + 4) * (TY + 4))
k_rb_sweep(int nx, int ny, int nz, int zc, T h2, LevelArrays<T> L, const T *__restrict__ b,
           const T *__restrict__ p_old, T *__restrict__ p_new, int first)
{
    constexpr int W = TX + 4, H = TY + 4;
    __shared__ T sp[3][H][W];
    __shared__ T sbx[3][H][W];
    __shared__ T sby[3][H][W];
    const int lx = threadIdx.x % W, ly = threadIdx.x / W;
    const int i = blockIdx.x * TX + lx - 2, j = blockIdx.y * TY + ly - 2;
    const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, nz);
    const bool dom = (i >= 0 && i < nx && j >= 0 && j < ny);
    const bool ring1 = dom && lx >= 1 && lx <= TX + 2 && ly >= 1 && ly <= TY + 2;
    const bool inner = dom && lx >= 2 && lx < TX + 2 && ly >= 2 && ly < TY + 2;
    const size_t sxy = (size_t)nx * ny;
    const size_t col = dom ? (size_t)j * nx + i : 0;
    const int second = first ^ 1;
    const bool xlo = i > 0, xhi = i < nx - 1, ylo = j > 0, yhi = j < ny - 1;

    // column registers: iterate at planes s-2 .. s+1, coefficients at planes s-1 .. s+1
    T q_m2 = T(0), q_m1 = T(0), q_0 = T(0), q_p1 = T(0);
    T bx_m1 = T(0), by_m1 = T(0), bz_m1 = T(0), di_m1 = T(0), b_m1 = T(0);
    T bx_0 = T(0), by_0 = T(0), bz_0 = T(0), di_0 = T(0), b_0 = T(0);
    T bx_p1 = T(0), by_p1 = T(0), bz_p1 = T(0), di_p1 = T(0), b_p1 = T(0);

    auto load_plane = [&](int z, T &q, T &bxv, T &byv, T &bzv, T &div, T &bv) {
        q = bxv = byv = bzv = div = bv = T(0);
        if (!dom || z < 0 || z >= nz) return;
        const size_t c = (size_t)z * sxy + col;
        q = p_old[c];
        bxv = L.bx[c];
        byv = L.by[c];
        if (ring1) {
            bzv = L.bz[c];
            if (sizeof(T) == 8) div = L.dinv[c];
            bv = b[c];
        }
    };
    // prologue: planes z0-2 (iterate only) and z0-1
    {
        T t0, t1, t2, t3, t4;
        load_plane(z0 - 2, q_m1, t0, t1, t2, t3, t4);
        load_plane(z0 - 1, q_0, bx_0, by_0, bz_0, di_0, b_0);
    }
    int cur = 0;
    for (int s = z0 - 1; s <= z1; s++) {
        const int prv = (cur + 2) % 3;  // buffer of plane s-1
        load_plane(s + 1, q_p1, bx_p1, by_p1, bz_p1, di_p1, b_p1);
        sp[cur][ly][lx] = q_0;
        sbx[cur][ly][lx] = bx_0;
        sby[cur][ly][lx] = by_0;
        __syncthreads();
        // first colour on plane s
        if (ring1 && s >= 0 && s < nz && ((i + j + s) & 1) == first) {
            const T bxh = xhi ? sbx[cur][ly][lx + 1] : T(0), byh = yhi ? sby[cur][ly + 1][lx] : T(0);
            const T bzh = (s < nz - 1) ? bz_p1 : T(0);
            T acc = T(0);
            if (xlo) acc = fma(bx_0, sp[cur][ly][lx - 1], acc);
            if (xhi) acc = fma(bxh, sp[cur][ly][lx + 1], acc);
            if (ylo) acc = fma(by_0, sp[cur][ly - 1][lx], acc);
            if (yhi) acc = fma(byh, sp[cur][ly + 1][lx], acc);
            if (s > 0) acc = fma(bz_0, q_m1, acc);
            if (s < nz - 1) acc = fma(bz_p1, q_p1, acc);
            q_0 = inv_diag<T>(di_0, bx_0, bxh, by_0, byh, bz_0, bzh) * fma(-h2, b_0, acc);
            sp[cur][ly][lx] = q_0;
        }
        __syncthreads();
        // second colour on plane s-1, then plane s-1 is final for this tile
        const int z = s - 1;
        if (inner && z >= z0 && z < z1) {
            if (((i + j + z) & 1) == second) {
                const T bxh = xhi ? sbx[prv][ly][lx + 1] : T(0), byh = yhi ? sby[prv][ly + 1][lx] : T(0);
                const T bzh = (z < nz - 1) ? bz_0 : T(0);
                T acc = T(0);
                if (xlo) acc = fma(bx_m1, sp[prv][ly][lx - 1], acc);
                if (xhi) acc = fma(bxh, sp[prv][ly][lx + 1], acc);
                if (ylo) acc = fma(by_m1, sp[prv][ly - 1][lx], acc);
                if (yhi) acc = fma(byh, sp[prv][ly + 1][lx], acc);
                if (z > 0) acc = fma(bz_m1, q_m2, acc);
                if (z < nz - 1) acc = fma(bz_0, q_0, acc);
                q_m1 = inv_diag<T>(di_m1, bx_m1, bxh, by_m1, byh, bz_m1, bzh) * fma(-h2, b_m1, acc);
            }
            p_new[(size_t)z * sxy + col] = q_m1;
        }
        q_m2 = q_m1; q_m1 = q_0; q_0 = q_p1;
        bx_m1 = bx_0; by_m1 = by_0; bz_m1 = bz_0; di_m1 = di_0; b_m1 = b_0;
        bx_0 = bx_p1; by_0 = by_p1; bz_0 = bz_p1; di_0 = di_p1; b_0 = b_p1;
        cur = (cur + 1) % 3;
    }
}

// Exact coarsest-grid solve e = M b with the dense minimum-norm inverse M (FP64 always).
// One warp per row (coalesced row reads, shuffle reduction); b staged in shared memory.
template <typename T>
__global__ void k_coarse_solve(int n, const double *__restrict__ M, const T *__restrict__ b, T *__restrict__ e)
{
    extern __shared__ double sb[];
    for (int i = threadIdx.x; i < n; i += blockDim.x) sb[i] = (double)b[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    for (int r = blockIdx.x * warps + warp; r < n; r += gridDim.x * warps) {
        if (!MG_CK((long long)r * n, (long long)r * n + n - 1, (long long)n * n, CK_COARSE_SOLVE)) continue;
        const double *row = M + (size_t)r * n;
        double s = 0.0;
        for (int q = lane; q < n; q += 32) s = fma(row[q], sb[q], s);
        s = warp_sum(s);
        if (lane == 0) e[r] = (T)s;
    }
}

// ---------------------------------------------------------------------------
// Coarse tail.  On the smallest levels (a few thousand cells) every colour pass, restriction and
// prolongation is a launch far longer than its work.  One CTA runs them in sequence instead,
// phases separated by __syncthreads (a level's fields stay in the SM's L1 between phases).  The
// per-cell arithmetic is the per-pass kernels' own (smooth_cell, restrict_cell, prolong_corr) and
// every cell of a pass is independent of the others, so the results are identical.  The fields
// are written and read within the kernel, so they are read through plain pointers (never the
// read-only path).
// ---------------------------------------------------------------------------
// threads of the descent (its residual-restriction needs more registers) and of the ascent
constexpr int kTailDownThreads = 512, kTailUpThreads = 1024;

template <typename T>
__device__ void tail_colour(const TailLevel<T> &v, int colour)
{
    const int hx = (v.nx + 1) / 2, total = hx * v.ny * v.nz;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int jk = (int)fdiv(t, v.fhx), k = (int)fdiv(jk, v.fny);
        const int u = t - jk * hx, j = jk - k * v.ny;
        const int i = 2 * u + ((j + k + colour) & 1);
        if (i < v.nx && ck_cell(((long long)k * v.ny + j) * v.nx + i, i, j, k, v.nx, v.ny, v.nz, CK_TAIL))
            smooth_cell<T, true>(i, j, k, v.nx, v.ny, v.nz, v.h2, v.L, v.L.b, v.L.p);
    }
    __syncthreads();
}

template <typename T>
__device__ void tail_restrict(const TailLevel<T> &f, T *bc)
{
    const int NX = f.nx / 2, NY = f.ny / 2, total = NX * NY * (f.nz / 2);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int JK = (int)fdiv(t, f.fcx), K = (int)fdiv(JK, f.fcy);
        const int I = t - JK * NX, J = JK - K * NY;
        restrict_cell<T>(I, J, K, f.nx, f.ny, f.nz, f.ih2, f.L, f.L.b, f.L.p, bc);
    }
    __syncthreads();
}

template <typename T>
__device__ void tail_prolong(const TailLevel<T> &f, const T *ec)
{
    const int NX = f.nx / 2, NY = f.ny / 2, NZ = f.nz / 2, total = NX * NY * NZ;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int JK = (int)fdiv(t, f.fcx), K = (int)fdiv(JK, f.fcy);
        const int I = t - JK * NX, J = JK - K * NY;
        T corr[2][2][2];
        prolong_corr<T>(I, J, K, NX, NY, NZ, ec, corr);
#pragma unroll
        for (int dz = 0; dz < 2; dz++)
#pragma unroll
            for (int dy = 0; dy < 2; dy++)
#pragma unroll
                for (int dx = 0; dx < 2; dx++) {
                    const size_t c = ((size_t)(2 * K + dz) * f.ny + (2 * J + dy)) * f.nx + 2 * I + dx;
                    if (!MG_CK(c, c, (long long)f.nx * f.ny * f.nz, CK_TAIL)) continue;
                    if (!zero_bits(f.L.dinv[c])) f.L.p[c] = f.L.p[c] + corr[dz][dy][dx];
                }
    }
    __syncthreads();
}

// descent: on each level but the coarsest, zero p (below the first), nu1 sweeps red then
// black, residual restricted to the next level's b
template <typename T>
__global__ void __launch_bounds__(kTailDownThreads) k_tail_down(TailArgs<T> a)
{
    for (int l = 0; l < a.nlev - 1; l++) {
        const TailLevel<T> v = a.lev[l];
        if (l > 0 || a.zero0) {
            const int n = v.nx * v.ny * v.nz;
            for (int t = threadIdx.x; t < n; t += blockDim.x) v.L.p[t] = T(0);
            __syncthreads();
        }
        for (int it = 0; it < a.nu1; it++) {
            tail_colour<T>(v, 0);
            tail_colour<T>(v, 1);
        }
        tail_restrict<T>(v, a.lev[l + 1].L.b);
    }
}

// ascent: from the level above the coarsest up, prolong the coarser correction, nu2 sweeps
// black then red
template <typename T>
__global__ void __launch_bounds__(kTailUpThreads) k_tail_up(TailArgs<T> a)
{
    for (int l = a.nlev - 2; l >= 0; l--) {
        const TailLevel<T> v = a.lev[l];
        tail_prolong<T>(v, a.lev[l + 1].L.p);
        for (int it = 0; it < a.nu2; it++) {
            tail_colour<T>(v, 1);
            tail_colour<T>(v, 0);
        }
    }
}

// ---------------------------------------------------------------------------
// Fine-level reductions (FP64, grid-stride, per-block partial pairs)
// ---------------------------------------------------------------------------
__global__ void k_count_live(unsigned n, const double *__restrict__ dinv, double *__restrict__ partials, double *dscal)
{
    double a = 0.0;
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x)
        a += pos_bits(dinv[idx]) ? 1.0 : 0.0;
    reduce_finish(block_sum<kRedThreads>(a), 0.0, partials, dscal, S_NLIVE, -1);
}

// pass 1 of the rhs preparation: sum of rhs over live cells
__global__ void k_sum_live(unsigned n, const double *__restrict__ v, const double *__restrict__ dinv,
                           double *__restrict__ partials, double *dscal)
{
    double a = 0.0;
    // the value loaded whatever the test (no wait on dinv); a starts at +0 and stays off -0, so
    // adding +0 for a dead cell leaves it unchanged
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const double x = v[idx];
        a += pos_bits(dinv[idx]) ? x : 0.0;
    }
    reduce_finish(block_sum<kRedThreads>(a), 0.0, partials, dscal, S_SUM_B, -1);
}

// pass 2: b0 = rhs - mean on live cells, 0 elsewhere; partial ||b0||^2
__global__ void k_rhs_center(unsigned n, const double *__restrict__ rhs, const double *__restrict__ dinv,
                             double *__restrict__ b0, double *dscal, double *__restrict__ partials)
{
    const double mean = block_scalar([&] { return dscal[S_SUM_B] / dscal[S_NLIVE]; });
    double a = 0.0;
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const double x = rhs[idx];  // loaded whatever the test
        const double v = pos_bits(dinv[idx]) ? x - mean : 0.0;
        b0[idx] = v;
        a += v * v;
    }
    reduce_finish(block_sum<kRedThreads>(a), 0.0, partials, dscal, S_NB2, -1);
}

// ||b - A p||^2 and sum of p over live cells
__global__ void k_resid_norm(int nx, int ny, int nz, double ih2, LevelArrays<double> L,
                             const double *__restrict__ b, const double *__restrict__ p, double *__restrict__ partials,
                             double *dscal)
{
    const unsigned n = (unsigned)nx * ny * nz;
    const size_t sxy = (size_t)nx * ny;
    double rr = 0.0, sp = 0.0;
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_of(idx, nx, ny, i, j, k);
        const double r = residual64_at(i, j, k, idx, nx, ny, nz, sxy, ih2, L, b, p);
        rr += r * r;
        if (pos_bits(L.dinv[idx])) sp += p[idx];
    }
    rr = block_sum<kRedThreads>(rr);
    sp = block_sum<kRedThreads>(sp);
    reduce_finish(rr, sp, partials, dscal, S_RR, S_SUM_P);
}

// p -= mean of p over live cells (mean = dscal[S_SUM_P] / dscal[S_NLIVE]); dead cells 0
__global__ void k_sub_mean_p(unsigned n, const double *__restrict__ dinv, double *__restrict__ p,
                             const double *__restrict__ dscal)
{
    const double mean = block_scalar([&] { return dscal[S_SUM_P] / dscal[S_NLIVE]; });
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const double x = p[idx];  // loaded whatever the test
        p[idx] = pos_bits(dinv[idx]) ? x - mean : 0.0;
    }
}

// Mixed refinement: r = b - A p in FP64, stored as FP32 r / scale_in; partial ||r||^2.
__global__ void k_resid_cast(int nx, int ny, int nz, double ih2, LevelArrays<double> L,
                             const double *__restrict__ b, const double *__restrict__ p, float *__restrict__ r32,
                             double *dscal, int scale_in, int scale_out, double *__restrict__ partials, size_t half)
{
    const unsigned n = (unsigned)nx * ny * nz;
    const size_t sxy = (size_t)nx * ny;
    const double inv_scale = block_scalar([&] { return 1.0 / dscal[scale_in]; });
    double rr = 0.0, sp = 0.0;
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_of(idx, nx, ny, i, j, k);
        const double r = residual64_at(i, j, k, idx, nx, ny, nz, sxy, ih2, L, b, p);
        rr += r * r;
        if (pos_bits(L.dinv[idx])) sp += p[idx];
        const size_t slot = half ? split_slot(idx, (j + k) & 1, half) : idx;
        if (MG_CK(slot, slot, (long long)n, CK_SPLIT_SLOT)) r32[slot] = narrow(r * inv_scale);
    }
    rr = block_sum<kRedThreads>(rr);
    sp = block_sum<kRedThreads>(sp);
    // the last block also sets the next scale: the RMS of this residual over the live cells (1 if 0)
    if (reduce_finish(rr, sp, partials, dscal, S_RR, S_SUM_P) && threadIdx.x == 0 && scale_out >= 0) {
        const double rms = sqrt(dscal[S_RR] / dscal[S_NLIVE]);
        dscal[scale_out] = (rms > 0.0 && isfinite(rms)) ? rms : 1.0;
    }
}

__global__ void k_scale_from_nb2(double *dscal, int slot)
{
    const double rms = sqrt(dscal[S_NB2] / dscal[S_NLIVE]);
    dscal[slot] = (rms > 0.0 && isfinite(rms)) ? rms : 1.0;
}

// p += scale * e32 (the FP32 cycle leaves e32 = 0 on dead cells, so no mask is read); e32 in
// the layout (half, nx, ny)
__global__ void k_accumulate(unsigned n, const float *__restrict__ e32, double *__restrict__ p,
                             const double *__restrict__ dscal, int scale_slot, Split sp)
{
    const double s = dscal[scale_slot];
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const size_t e = sp.half ? split_slot(idx, row_parity(idx, sp), sp.half) : idx;
        if (!MG_CK(e, e, (long long)n, CK_SPLIT_SLOT)) continue;
        p[idx] = fma(s, widen(e32[e]), p[idx]);
    }
}

// The FP32 copy of one level: the narrowed faces (natural layout; on the finest level with a
// colour-split layout, also in that layout, sf != null) and 1/sum of the narrowed faces, summed
// in k_diag_inv's order with its divisor memo (so the value k_diag_inv gives on the narrowed
// faces), from one read of the FP64 faces.  Grid and runs as k_diag_inv.
__global__ void k_level_f32(int nx, int ny, int nz, const double *__restrict__ bx, const double *__restrict__ by,
                            const double *__restrict__ bz, LevelArrays<float> out, LevelArrays<float> sf,
                            size_t half)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nx) return;
    const int k0 = blockIdx.z * kRun, k1 = min(k0 + kRun, nz);
    const size_t sxy = (size_t)nx * ny;
    float s_last = 1.0f, q_last = 1.0f;
    size_t c = (size_t)k0 * sxy + (size_t)j * nx + i;
    float bz_lo = narrow(bz[c]);
    // a cell's loads at once; the next cell's issued before this one's stores
    struct In {
        double x0, x1, y0, y1, zh;
    };
    auto load = [&](size_t cc, int kk) {
        In v;
        v.x0 = bx[cc];
        v.x1 = (i < nx - 1) ? bx[cc + 1] : 0.0;
        v.y0 = by[cc];
        v.y1 = (j < ny - 1) ? by[cc + nx] : 0.0;
        v.zh = (kk < nz - 1) ? bz[cc + sxy] : 0.0;
        return v;
    };
    In cur = load(c, k0);
    for (int k = k0; k < k1; k++, c += sxy) {
        const In nxt = k + 1 < k1 ? load(c + sxy, k + 1) : cur;
        const float bz_hi = narrow(cur.zh);
        const float x = narrow(cur.x0), y = narrow(cur.y0);
        out.bx[c] = x;
        out.by[c] = y;
        out.bz[c] = bz_lo;
        if (sf.bx) {
            const size_t e = split_slot(c, (j + k) & 1, half);
            sf.bx[e] = x;
            sf.by[e] = y;
            sf.bz[e] = bz_lo;
        }
        float t = x;
        t += narrow(cur.x1);
        t += y;
        t += narrow(cur.y1);
        t += bz_lo;
        t += bz_hi;
        bz_lo = bz_hi;
        cur = nxt;
        float q = 0.0f;
        if (t > 0.0f) {
            if (!same_bits(t, s_last)) {
                s_last = t;
                q_last = div_call(1.0f, t);
            }
            q = q_last;
        }
        out.dinv[c] = q;
    }
}

// FP64 natural-order field <-> the finest FP32 field in the layout sp (one FP32 V-cycle on a
// caller's FP64 rhs and iterate)
__global__ void k_to_f32_layout(unsigned n, const double *__restrict__ src, float *__restrict__ dst, Split sp)
{
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x)
    {
        const size_t e = sp.half ? split_slot(idx, row_parity(idx, sp), sp.half) : idx;
        if (MG_CK(e, e, (long long)n, CK_SPLIT_SLOT)) dst[e] = narrow(src[idx]);
    }
}
__global__ void k_from_f32_layout(unsigned n, const float *__restrict__ src, double *__restrict__ dst, Split sp)
{
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x)
    {
        const size_t e = sp.half ? split_slot(idx, row_parity(idx, sp), sp.half) : idx;
        if (MG_CK(e, e, (long long)n, CK_SPLIT_SLOT)) dst[idx] = widen(src[e]);
    }
}

// ---------------------------------------------------------------------------
// Projection (Eq. poisson1 right-hand side; Eq. runge1 correction) and adjoint
// ---------------------------------------------------------------------------
__global__ void k_divergence(int nx, int ny, int nz, Scale2 scale, const double *__restrict__ bx,
                             const double *__restrict__ by, const double *__restrict__ bz,
                             const double *__restrict__ ux, const double *__restrict__ uy,
                             const double *__restrict__ uz, double *__restrict__ rhs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const size_t sxy = (size_t)nx * ny;
    const size_t c = (size_t)k * sxy + (size_t)j * nx + i;
    if (!ck_cell((long long)c, i, j, k, nx, ny, nz, CK_DIVERGENCE)) return;
    // every load first (a velocity's load does not wait for its face's coefficient)
    const bool xh = i < nx - 1, yh = j < ny - 1, zh = k < nz - 1;
    const double bx0 = bx[c], bx1 = xh ? bx[c + 1] : 0.0, by0 = by[c], by1 = yh ? by[c + nx] : 0.0;
    const double bz0 = bz[c], bz1 = zh ? bz[c + sxy] : 0.0;
    const double ux0 = ux[c], ux1 = xh ? ux[c + 1] : 0.0, uy0 = uy[c], uy1 = yh ? uy[c + nx] : 0.0;
    const double uz0 = uz[c], uz1 = zh ? uz[c + sxy] : 0.0;
    double d = 0.0;
    if (pos_bits(bx1)) d += ux1;
    if (pos_bits(bx0)) d -= ux0;
    if (pos_bits(by1)) d += uy1;
    if (pos_bits(by0)) d -= uy0;
    if (pos_bits(bz1)) d += uz1;
    if (pos_bits(bz0)) d -= uz0;
    rhs[c] = mul_s2(d, scale);  // scale * d
}

// ---------------------------------------------------------------------------
// Fractional face areas (Body Boundary Conditions section, Eq. integral2).  psi is given at the
// nodes ((nz+1) x (ny+1) x (nx+1), > 0 outside the body).  A face is split into four triangles
// about its centre (psi there = the mean of the four corners), psi is linear on each, and the open
// fraction is the mean of the triangles' fractions where psi > 0; a triangle with one corner f > 0
// and two g1, g2 <= 0 has f^2 / ((f - g1)(f - g2)), one with two corners > 0 and one g <= 0 has
// 1 - g^2 / ((g - f1)(g - f2)).  Each operation rounded separately.
// ---------------------------------------------------------------------------
__device__ double tri_open(double a, double b, double c)
{
    const bool pa = pos_bits(a), pb = pos_bits(b), pc = pos_bits(c);
    const int np = (int)pa + (int)pb + (int)pc;
    if (np == 0) return 0.0;
    if (np == 3) return 1.0;
    if (np == 1) {
        const double f = pa ? a : (pb ? b : c);
        const double g1 = pa ? b : a, g2 = pc ? b : c;
        return div_call(__dmul_rn(f, f), __dmul_rn(__dsub_rn(f, g1), __dsub_rn(f, g2)));
    }
    const double g = !pa ? a : (!pb ? b : c);
    const double f1 = !pa ? b : a, f2 = !pc ? b : c;
    return __dsub_rn(1.0, div_call(__dmul_rn(g, g), __dmul_rn(__dsub_rn(g, f1), __dsub_rn(g, f2))));
}

// corners in cyclic order around the face: f00, f10, f11, f01
__device__ double face_open(double f00, double f10, double f01, double f11)
{
    const double fc = __dmul_rn(__dadd_rn(__dadd_rn(f00, f10), __dadd_rn(f01, f11)), 0.25);
    const double t0 = tri_open(f00, f10, fc), t1 = tri_open(f10, f11, fc);
    const double t2 = tri_open(f11, f01, fc), t3 = tri_open(f01, f00, fc);
    return __dmul_rn(__dadd_rn(__dadd_rn(__dadd_rn(t0, t1), t2), t3), 0.25);
}

// open fractions of the low faces of every cell; wall faces 0
__global__ void k_face_areas(int nx, int ny, int nz, const double *__restrict__ psi, double *__restrict__ ax,
                             double *__restrict__ ay, double *__restrict__ az)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const size_t NX = (size_t)nx + 1, NXY = NX * ((size_t)ny + 1);
    auto P = [&](int ii, int jj, int kk) { return psi[(size_t)kk * NXY + (size_t)jj * NX + (size_t)ii]; };
    const size_t c = ((size_t)k * ny + j) * nx + i;
    ax[c] = i == 0 ? 0.0 : face_open(P(i, j, k), P(i, j + 1, k), P(i, j, k + 1), P(i, j + 1, k + 1));
    ay[c] = j == 0 ? 0.0 : face_open(P(i, j, k), P(i + 1, j, k), P(i, j, k + 1), P(i + 1, j, k + 1));
    az[c] = k == 0 ? 0.0 : face_open(P(i, j, k), P(i + 1, j, k), P(i, j + 1, k), P(i + 1, j + 1, k));
}

// Stretched grids: cell widths hx[i], hy[j], hz[k].  Eq. integral2 times the cell volume on the
// index grid (unit spacing): beta_idx = beta / d with d the distance between the two cell centres,
// area = the face's two widths times the open fraction (frac, or 1); walls 0.  Each operation
// rounded separately.
__global__ void k_stretched_metrics(int nx, int ny, int nz, const double *__restrict__ hx,
                                    const double *__restrict__ hy, const double *__restrict__ hz,
                                    LevelArrays<double> beta, LevelArrays<double> frac, LevelArrays<double> bout,
                                    LevelArrays<double> aout)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const size_t c = ((size_t)k * ny + j) * nx + i;
    if (i == 0) {
        bout.bx[c] = 0.0;
        aout.bx[c] = 0.0;
    } else {
        const double d = __dmul_rn(0.5, __dadd_rn(hx[i - 1], hx[i]));
        bout.bx[c] = div_call(beta.bx[c], d);
        aout.bx[c] = __dmul_rn(__dmul_rn(hy[j], hz[k]), frac.bx ? frac.bx[c] : 1.0);
    }
    if (j == 0) {
        bout.by[c] = 0.0;
        aout.by[c] = 0.0;
    } else {
        const double d = __dmul_rn(0.5, __dadd_rn(hy[j - 1], hy[j]));
        bout.by[c] = div_call(beta.by[c], d);
        aout.by[c] = __dmul_rn(__dmul_rn(hx[i], hz[k]), frac.by ? frac.by[c] : 1.0);
    }
    if (k == 0) {
        bout.bz[c] = 0.0;
        aout.bz[c] = 0.0;
    } else {
        const double d = __dmul_rn(0.5, __dadd_rn(hz[k - 1], hz[k]));
        bout.bz[c] = div_call(beta.bz[c], d);
        aout.bz[c] = __dmul_rn(__dmul_rn(hx[i], hy[j]), frac.bz ? frac.bz[c] : 1.0);
    }
}

// ---------------------------------------------------------------------------
// The Runge-Kutta time step (Numerical Time Integration section).  R = the body force, -g on the
// open z-faces (beta_z > 0), 0 elsewhere; each operation rounded separately in the order written.
// ---------------------------------------------------------------------------
// out = (a + b) + dt R   (b null: a + dt R)
__global__ void k_rk_combine(size_t n, LevelArrays<double> a, LevelArrays<double> b, LevelArrays<double> r, double dt,
                             LevelArrays<double> out)
{
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const double sx = b.bx ? __dadd_rn(a.bx[c], b.bx[c]) : a.bx[c];
        const double sy = b.by ? __dadd_rn(a.by[c], b.by[c]) : a.by[c];
        const double sz = b.bz ? __dadd_rn(a.bz[c], b.bz[c]) : a.bz[c];
        out.bx[c] = __dadd_rn(sx, __dmul_rn(dt, r.bx[c]));
        out.by[c] = __dadd_rn(sy, __dmul_rn(dt, r.by[c]));
        out.bz[c] = __dadd_rn(sz, __dmul_rn(dt, r.bz[c]));
    }
}

// ---------------------------------------------------------------------------
// Momentum right-hand side R_i of Eq. navi without the pressure gradient and the sub-grid
// stress: R_i = -d/dx_j (u_j u_i) + (1/rho_f)/Re d/dx_j (2 mu S_ij) - delta_i3 g, with mu from
// Eq. density and 1/rho_f the face coefficient.  Second-order central conservative MAC form:
// u_i u_i at the cell centres (mean of the cell's two i-faces), u_j u_i at the edges (means of
// the two j-faces and of the two i-faces meeting there), 2 mu S_ii at the centres, 2 mu S_ij at
// the edges (mu: mean of the four cells around the edge, in cell-index order), each divergence
// the difference of the two values bracketing the face over h.  Free-slip walls: normal velocity
// 0 (the stored wall face, or the unstored high wall), tangential velocity mirrored into the
// ghost row; closed faces get R = 0.  Separately rounded operations in a fixed order.
//
// Two passes.  k_mom_parts computes, once per cell, the quantities every face shares: for each
// axis a the centre flux C_a = U_a^2 (U_a the cell's mean a-velocity) and stress T_a = 2 mu
// dU_a/dx_a, and for each plane (a, b), a < b, at the cell's low edge the flux F_ab = (mean u_b)
// (mean u_a) and the shear S_ab = mu_edge (du_a/dx_b + du_b/dx_a).  k_mom_combine forms each
// open face's R from the values bracketing it.  A face's F_ab and S_ab are the same numbers
// whichever of the four faces at the edge uses them (the product and the sum commute exactly), so
// R is bitwise the per-face evaluation, with a third of its FP64 operations.
// ---------------------------------------------------------------------------
struct MomArgs {
    int nx, ny, nz, convect;
    double ih, mu_air, dmu, inv_re, g;
    const double *phi;
    LevelArrays<double> beta, u, r;
    double *w;  // 12 arrays of n: C_x, C_y, C_z, T_x, T_y, T_z, F_xy, F_xz, F_yz, S_xy, S_xz, S_yz
};

__device__ __forceinline__ int clamp_idx(int v, int hi) { return v < 0 ? 0 : (v > hi ? hi : v); }

// velocity of axis AX on its face (i, j, k): 0 at the high wall of its own axis, the other two
// indices mirrored into the domain
template <int AX>
__device__ __forceinline__ double mom_vel(const MomArgs &m, int i, int j, int k)
{
    if ((AX == 0 && i >= m.nx) || (AX == 1 && j >= m.ny) || (AX == 2 && k >= m.nz)) return 0.0;
    i = clamp_idx(i, m.nx - 1);
    j = clamp_idx(j, m.ny - 1);
    k = clamp_idx(k, m.nz - 1);
    const double *u = AX == 0 ? m.u.bx : (AX == 1 ? m.u.by : m.u.bz);
    return u[((size_t)k * m.ny + j) * m.nx + i];
}

__device__ __forceinline__ double mom_mu(const MomArgs &m, int i, int j, int k)
{
    i = clamp_idx(i, m.nx - 1);
    j = clamp_idx(j, m.ny - 1);
    k = clamp_idx(k, m.nz - 1);
    return __dadd_rn(m.mu_air, __dmul_rn(m.dmu, m.phi[((size_t)k * m.ny + j) * m.nx + i]));
}

// centre flux and stress of axis A at cell (i, j, k) (mu: the cell's viscosity)
template <int A>
__device__ __forceinline__ void mom_centre(const MomArgs &m, int i, int j, int k, double mu, double &C, double &T)
{
    constexpr int ai = A == 0, aj = A == 1, ak = A == 2;
    const double u0 = mom_vel<A>(m, i, j, k), u1 = mom_vel<A>(m, i + ai, j + aj, k + ak);
    const double U = __dmul_rn(0.5, __dadd_rn(u0, u1));
    C = __dmul_rn(U, U);
    T = __dmul_rn(__dmul_rn(2.0, mu), __dmul_rn(__dsub_rn(u1, u0), m.ih));
}

// flux and shear of plane (A, B), A < B, at the low edge of cell (i, j, k); mc, ma, mb, mab: the
// viscosities of the cell and of its neighbours below along A, along B, along both
template <int A, int B>
__device__ __forceinline__ void mom_edge(const MomArgs &m, int i, int j, int k, double mc, double ma, double mb,
                                         double mab, double &F, double &S)
{
    constexpr int ai = A == 0, aj = A == 1, ak = A == 2, bi = B == 0, bj = B == 1, bk = B == 2;
    const double ua0 = mom_vel<A>(m, i - bi, j - bj, k - bk), ua1 = mom_vel<A>(m, i, j, k);
    const double ub0 = mom_vel<B>(m, i - ai, j - aj, k - ak), ub1 = mom_vel<B>(m, i, j, k);
    F = __dmul_rn(__dmul_rn(0.5, __dadd_rn(ub0, ub1)), __dmul_rn(0.5, __dadd_rn(ua0, ua1)));
    const double me = __dmul_rn(0.25, __dadd_rn(__dadd_rn(__dadd_rn(mab, mb), ma), mc));
    S = __dmul_rn(me, __dadd_rn(__dmul_rn(__dsub_rn(ua1, ua0), m.ih), __dmul_rn(__dsub_rn(ub1, ub0), m.ih)));
}

__global__ void k_mom_parts(MomArgs m)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
    if (i >= m.nx || j >= m.ny) return;
    const size_t n = (size_t)m.nx * m.ny * m.nz, c = ((size_t)k * m.ny + j) * m.nx + i;
    if (!MG_CK(c, c, (long long)n, CK_MOMENTUM)) return;
    const double mc = mom_mu(m, i, j, k), mx = mom_mu(m, i - 1, j, k), my = mom_mu(m, i, j - 1, k),
                 mz = mom_mu(m, i, j, k - 1), mxy = mom_mu(m, i - 1, j - 1, k), mxz = mom_mu(m, i - 1, j, k - 1),
                 myz = mom_mu(m, i, j - 1, k - 1);
    double C, T, F, S;
    mom_centre<0>(m, i, j, k, mc, C, T);
    m.w[c] = C;
    m.w[3 * n + c] = T;
    mom_centre<1>(m, i, j, k, mc, C, T);
    m.w[n + c] = C;
    m.w[4 * n + c] = T;
    mom_centre<2>(m, i, j, k, mc, C, T);
    m.w[2 * n + c] = C;
    m.w[5 * n + c] = T;
    // in cell-index order: the cell below along both axes, below along the higher axis, below along
    // the lower axis, the cell itself
    mom_edge<0, 1>(m, i, j, k, mc, mx, my, mxy, F, S);
    m.w[6 * n + c] = F;
    m.w[9 * n + c] = S;
    mom_edge<0, 2>(m, i, j, k, mc, mx, mz, mxz, F, S);
    m.w[7 * n + c] = F;
    m.w[10 * n + c] = S;
    mom_edge<1, 2>(m, i, j, k, mc, my, mz, myz, F, S);
    m.w[8 * n + c] = F;
    m.w[11 * n + c] = S;
}

// edge value of plane (A, B) (either order) at the low edge of cell (i, j, k), which may lie on the
// high wall of the other axis (one past the last cell): there the normal velocity of the wall and
// the mirrored tangential velocity make both the flux and the shear zero
template <int A, int B>
__device__ __forceinline__ void mom_edge_at(const MomArgs &m, size_t n, int i, int j, int k, double &F, double &S)
{
    constexpr int lo = A < B ? A : B, hi = A < B ? B : A;
    constexpr int slot = (lo == 0 && hi == 1) ? 0 : ((lo == 0) ? 1 : 2);
    if (i >= m.nx || j >= m.ny || k >= m.nz) {
        F = 0.0;
        S = 0.0;
        return;
    }
    const size_t c = ((size_t)k * m.ny + j) * m.nx + i;
    F = m.w[(6 + slot) * n + c];
    S = m.w[(9 + slot) * n + c];
}

template <int A>
__device__ __forceinline__ double mom_face(const MomArgs &m, size_t n, int i, int j, int k, size_t c, double beta)
{
    constexpr int ai = A == 0, aj = A == 1;
    const size_t cm = c - (ai ? 1 : (aj ? (size_t)m.nx : (size_t)m.nx * m.ny));
    double conv = __dmul_rn(__dsub_rn(m.w[A * n + c], m.w[A * n + cm]), m.ih);
    double visc = __dsub_rn(m.w[(3 + A) * n + c], m.w[(3 + A) * n + cm]);
    auto tangential = [&](auto bcon) {
        constexpr int B = decltype(bcon)::value;
        constexpr int bi = B == 0, bj = B == 1, bk = B == 2;
        double F0, S0, F1, S1;
        mom_edge_at<A, B>(m, n, i, j, k, F0, S0);
        mom_edge_at<A, B>(m, n, i + bi, j + bj, k + bk, F1, S1);
        conv = __dadd_rn(conv, __dmul_rn(__dsub_rn(F1, F0), m.ih));
        visc = __dadd_rn(visc, __dsub_rn(S1, S0));
    };
    if (A == 0) {
        tangential(std::integral_constant<int, 1>());
        tangential(std::integral_constant<int, 2>());
    } else if (A == 1) {
        tangential(std::integral_constant<int, 0>());
        tangential(std::integral_constant<int, 2>());
    } else {
        tangential(std::integral_constant<int, 0>());
        tangential(std::integral_constant<int, 1>());
    }
    double r = m.convect ? -conv : 0.0;
    r = __dadd_rn(r, __dmul_rn(__dmul_rn(m.inv_re, beta), __dmul_rn(visc, m.ih)));
    if (A == 2) r = __dsub_rn(r, m.g);
    return r;
}

// one thread per cell: R on its three low faces
__global__ void k_mom_combine(MomArgs m)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
    if (i >= m.nx || j >= m.ny) return;
    const size_t n = (size_t)m.nx * m.ny * m.nz, c = ((size_t)k * m.ny + j) * m.nx + i;
    if (!MG_CK(c, c, (long long)n, CK_MOMENTUM)) return;
    const double bx = m.beta.bx[c], by = m.beta.by[c], bz = m.beta.bz[c];
    // an open face is interior (its low neighbour exists), so c - e_a is a cell
    m.r.bx[c] = (i > 0 && pos_bits(bx)) ? mom_face<0>(m, n, i, j, k, c, bx) : 0.0;
    m.r.by[c] = (j > 0 && pos_bits(by)) ? mom_face<1>(m, n, i, j, k, c, by) : 0.0;
    m.r.bz[c] = (k > 0 && pos_bits(bz)) ? mom_face<2>(m, n, i, j, k, c, bz) : 0.0;
}

// out = 0.5 (a + b)   (b null: 0.5 a)
__global__ void k_half(size_t n, LevelArrays<double> a, LevelArrays<double> b, LevelArrays<double> out)
{
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        out.bx[c] = __dmul_rn(0.5, b.bx ? __dadd_rn(a.bx[c], b.bx[c]) : a.bx[c]);
        out.by[c] = __dmul_rn(0.5, b.by ? __dadd_rn(a.by[c], b.by[c]) : a.by[c]);
        out.bz[c] = __dmul_rn(0.5, b.bz ? __dadd_rn(a.bz[c], b.bz[c]) : a.bz[c]);
    }
}

// phi_out = phi - s * sum over open faces of +-u_f phi_up(f)  (s = dt / h; first-order upwind, the
// order x+, x-, y+, y-, z+, z-; closed faces carry no flux)
__global__ void k_vof_upwind(int nx, int ny, int nz, double s, LevelArrays<double> mask, LevelArrays<double> u,
                             const double *__restrict__ phi, double *__restrict__ phi_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const size_t sxy = (size_t)nx * ny;
    const size_t c = (size_t)k * sxy + (size_t)j * nx + i;
    if (!ck_cell((long long)c, i, j, k, nx, ny, nz, CK_VOF)) return;
    auto upw = [&](double uf, size_t lo, size_t hi) { return __dmul_rn(uf, pos_bits(uf) ? phi[lo] : phi[hi]); };
    double d = 0.0;
    if (i < nx - 1 && pos_bits(mask.bx[c + 1])) d = __dadd_rn(d, upw(u.bx[c + 1], c, c + 1));
    if (pos_bits(mask.bx[c])) d = __dsub_rn(d, upw(u.bx[c], c - 1, c));
    if (j < ny - 1 && pos_bits(mask.by[c + nx])) d = __dadd_rn(d, upw(u.by[c + nx], c, c + nx));
    if (pos_bits(mask.by[c])) d = __dsub_rn(d, upw(u.by[c], c - nx, c));
    if (k < nz - 1 && pos_bits(mask.bz[c + sxy])) d = __dadd_rn(d, upw(u.bz[c + sxy], c, c + sxy));
    if (pos_bits(mask.bz[c])) d = __dsub_rn(d, upw(u.bz[c], c - sxy, c));
    phi_out[c] = __dsub_rn(phi[c], __dmul_rn(s, d));
}

// the operator's coefficient of a face: area * 1/rho where the area is > 0, else 0
__global__ void k_area_coeffs(size_t n, LevelArrays<double> area, LevelArrays<double> beta, LevelArrays<double> out)
{
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        out.bx[c] = pos_bits(area.bx[c]) ? __dmul_rn(area.bx[c], beta.bx[c]) : 0.0;
        out.by[c] = pos_bits(area.by[c]) ? __dmul_rn(area.by[c], beta.by[c]) : 0.0;
        out.bz[c] = pos_bits(area.bz[c]) ? __dmul_rn(area.bz[c], beta.bz[c]) : 0.0;
    }
}

// b = scale * sum over the open faces (mask > 0) of +-w_f (u_f - v_f), order x+, x-, y+, y-, z+, z-;
// w = the face's area (or 1 without areas), v = the body velocity (or none)
__global__ void k_divergence_area(int nx, int ny, int nz, double scale, LevelArrays<double> mask,
                                  LevelArrays<double> area, LevelArrays<double> u, LevelArrays<double> v,
                                  double *__restrict__ rhs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const size_t sxy = (size_t)nx * ny;
    const size_t c = (size_t)k * sxy + (size_t)j * nx + i;
    auto flux = [&](const double *a, const double *uu, const double *vv, size_t f) {
        const double du = vv ? __dsub_rn(uu[f], vv[f]) : uu[f];
        return a ? __dmul_rn(a[f], du) : du;
    };
    double d = 0.0;
    if (i < nx - 1 && pos_bits(mask.bx[c + 1])) d = __dadd_rn(d, flux(area.bx, u.bx, v.bx, c + 1));
    if (pos_bits(mask.bx[c])) d = __dsub_rn(d, flux(area.bx, u.bx, v.bx, c));
    if (j < ny - 1 && pos_bits(mask.by[c + nx])) d = __dadd_rn(d, flux(area.by, u.by, v.by, c + nx));
    if (pos_bits(mask.by[c])) d = __dsub_rn(d, flux(area.by, u.by, v.by, c));
    if (k < nz - 1 && pos_bits(mask.bz[c + sxy])) d = __dadd_rn(d, flux(area.bz, u.bz, v.bz, c + sxy));
    if (pos_bits(mask.bz[c])) d = __dsub_rn(d, flux(area.bz, u.bz, v.bz, c));
    rhs[c] = __dmul_rn(scale, d);
}

// u_f = u*_f - dt beta_f (p_c - p_nb) / h on open low faces; closed faces copy u*.
// x / h, rounded once: a multiply by ih = 1/h when h is a power of two (then x * (1/h) is exact
// and equal to the quotient; mul_pow2), an IEEE division otherwise
__device__ __forceinline__ double div_h(double x, double h, const Scale2 &ih)
{
    return ih.ok ? mul_pow2(x, ih.f, ih.e) : div_call(x, h);
}

// The face is open where b > 0; its coefficient is val (1/rho when b holds area * 1/rho), or b
// itself when val is null.
__global__ void k_correct(int nx, int ny, int nz, double dt, double h, Scale2 ih,
                          const double *__restrict__ bx, const double *__restrict__ by, const double *__restrict__ bz,
                          const double *__restrict__ p, const double *ux0, const double *uy0, const double *uz0,
                          double *ux, double *uy, double *uz, LevelArrays<double> val)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const size_t sxy = (size_t)nx * ny;
    const size_t c = (size_t)k * sxy + (size_t)j * nx + i;
    if (!ck_cell((long long)c, i, j, k, nx, ny, nz, CK_CORRECT)) return;
    // every load first; each face's update formed and kept where the face is open (the same
    // operations as forming it there alone)
    const double pc = p[c], pxl = i > 0 ? p[c - 1] : 0.0, pyl = j > 0 ? p[c - nx] : 0.0;
    const double pzl = k > 0 ? p[c - sxy] : 0.0;
    const double b0 = bx[c], b1 = by[c], b2 = bz[c];
    const double u0 = ux0[c], u1 = uy0[c], u2 = uz0[c];
    const double v0 = val.bx ? val.bx[c] : b0, v1 = val.by ? val.by[c] : b1, v2 = val.bz ? val.bz[c] : b2;
    auto upd = [&](double u, double bv, double pn) {
        return __dsub_rn(u, div_h(__dmul_rn(__dmul_rn(dt, bv), __dsub_rn(pc, pn)), h, ih));
    };
    ux[c] = (i > 0 && pos_bits(b0)) ? upd(u0, v0, pxl) : u0;
    uy[c] = (j > 0 && pos_bits(b1)) ? upd(u1, v1, pyl) : u1;
    uz[c] = (k > 0 && pos_bits(b2)) ? upd(u2, v2, pzl) : u2;
}

// rhs_c = scale * the sum over the open faces of c (L's coefficient > 0) of +-(B_f w_f), x+ added
// and x- subtracted, then y, then z: the divergence (as k_divergence) of the face products B w,
// each rounded once (the adjoint's right-hand side D(beta w)).  Blocks as k_phi_grad: each face's
// product formed once, the x+ and y+ ones taken from the neighbours through shared memory (formed
// again only at the block's right edge and top row), the z+ one carried up the column.
__global__ void k_divergence_mul(int nx, int ny, int nz, Scale2 scale, LevelArrays<double> L, LevelArrays<double> B,
                                 const double *__restrict__ wx, const double *__restrict__ wy,
                                 const double *__restrict__ wz, double *__restrict__ rhs)
{
    __shared__ double sh[2][2][kPhiThreads];  // [plane parity][x- / y- product][thread]
    const int W = blockDim.x, R = blockDim.y;
    const int i = blockIdx.x * W + threadIdx.x, j = blockIdx.y * R + threadIdx.y;
    const int t = threadIdx.y * W + threadIdx.x;
    const bool in = i < nx && j < ny;
    const int k0 = blockIdx.z * kPhiRun, k1 = min(k0 + kPhiRun, nz);
    const size_t sxy = (size_t)nx * ny;
    size_t c = in ? (size_t)k0 * sxy + (size_t)j * nx + i : 0;
    const bool ok0 = in && ck_cell((long long)c, i, j, k0, nx, ny, nz, CK_DIVERGENCE);
    double tz_lo = ok0 ? __dmul_rn(B.bz[c], wz[c]) : 0.0;
    bool oz_lo = ok0 && pos_bits(L.bz[c]);
    for (int k = k0; k < k1; k++, c += sxy) {
        const bool ok = in && ck_cell((long long)c, i, j, k, nx, ny, nz, CK_DIVERGENCE);
        double tx = 0.0, ty = 0.0, tz_hi = 0.0;
        bool ox0 = false, ox1 = false, oy0 = false, oy1 = false, oz1 = false;
        if (ok) {
            tx = __dmul_rn(B.bx[c], wx[c]);
            ty = __dmul_rn(B.by[c], wy[c]);
            ox0 = pos_bits(L.bx[c]);
            oy0 = pos_bits(L.by[c]);
            ox1 = i < nx - 1 && pos_bits(L.bx[c + 1]);
            oy1 = j < ny - 1 && pos_bits(L.by[c + nx]);
            if (k < nz - 1) {
                tz_hi = __dmul_rn(B.bz[c + sxy], wz[c + sxy]);
                oz1 = pos_bits(L.bz[c + sxy]);
            }
        }
        double(*buf)[kPhiThreads] = sh[k & 1];
        buf[0][t] = tx;
        buf[1][t] = ty;
        __syncthreads();  // one barrier per plane: a buffer is written again two planes later
        if (ok) {
            double tx_hi = 0.0, ty_hi = 0.0;
            if (i < nx - 1) tx_hi = threadIdx.x < W - 1 ? buf[0][t + 1] : dmul_call(B.bx[c + 1], wx[c + 1]);
            if (j < ny - 1) ty_hi = threadIdx.y < R - 1 ? buf[1][t + W] : dmul_call(B.by[c + nx], wy[c + nx]);
            double d = 0.0;
            if (ox1) d = __dadd_rn(d, tx_hi);
            if (ox0) d = __dsub_rn(d, tx);
            if (oy1) d = __dadd_rn(d, ty_hi);
            if (oy0) d = __dsub_rn(d, ty);
            if (oz1) d = __dadd_rn(d, tz_hi);
            if (oz_lo) d = __dsub_rn(d, tz_lo);
            rhs[c] = mul_s2(d, scale);  // scale * d
        }
        tz_lo = tz_hi;
        oz_lo = oz1;
    }
}

// grad_u = w - G q (open faces) / w (closed);  grad_beta = dt (G p)((G q) - w) (open) / 0 (closed)
// has_a: the face's open area a multiplies G q (fractional areas)
__device__ __forceinline__ void adj_face(double b, double pc, double pn, double qc, double qn, double w, double h,
                                         const Scale2 &ih, double dt, bool has_a, double a, double &gu, double &gb)
{
    double gq = div_h(__dsub_rn(qc, qn), h, ih);
    const double gp = div_h(__dsub_rn(pc, pn), h, ih);
    if (has_a) gq = dmul_call(a, gq);
    const double go = __dsub_rn(w, gq);
    // (Gq - w) is -gu exactly: a rounded difference changes sign with its operands' order
    const double bo = __dmul_rn(__dmul_rn(dt, gp), -go);
    const bool open = pos_bits(b);
    gu = open ? go : w;
    gb = open ? bo : 0.0;
}

__global__ void k_adjoint_faces(int nx, int ny, int nz, double h, Scale2 ih, double dt,
                                const double *__restrict__ bx,
                                const double *__restrict__ by, const double *__restrict__ bz,
                                const double *__restrict__ p, const double *__restrict__ q,
                                const double *__restrict__ wx, const double *__restrict__ wy,
                                const double *__restrict__ wz, double *gux, double *guy, double *guz, double *gbx,
                                double *gby, double *gbz, LevelArrays<double> area)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const size_t sxy = (size_t)nx * ny;
    const size_t c = (size_t)k * sxy + (size_t)j * nx + i;
    if (!ck_cell((long long)c, i, j, k, nx, ny, nz, CK_ADJOINT)) return;
    // every load first
    const double pc = p[c], qc = q[c];
    const double pxl = i > 0 ? p[c - 1] : 0.0, qxl = i > 0 ? q[c - 1] : 0.0;
    const double pyl = j > 0 ? p[c - nx] : 0.0, qyl = j > 0 ? q[c - nx] : 0.0;
    const double pzl = k > 0 ? p[c - sxy] : 0.0, qzl = k > 0 ? q[c - sxy] : 0.0;
    const double b0 = bx[c], b1 = by[c], b2 = bz[c], w0 = wx[c], w1 = wy[c], w2 = wz[c];
    const double a0 = area.bx ? area.bx[c] : 1.0, a1 = area.by ? area.by[c] : 1.0, a2 = area.bz ? area.bz[c] : 1.0;
    double gu, gb;
    adj_face(b0, pc, pxl, qc, qxl, w0, h, ih, dt, area.bx != nullptr, a0, gu, gb);
    gux[c] = gu;
    if (gbx) gbx[c] = gb;
    adj_face(b1, pc, pyl, qc, qyl, w1, h, ih, dt, area.by != nullptr, a1, gu, gb);
    guy[c] = gu;
    if (gby) gby[c] = gb;
    adj_face(b2, pc, pzl, qc, qzl, w2, h, ih, dt, area.bz != nullptr, a2, gu, gb);
    guz[c] = gu;
    if (gbz) gbz[c] = gb;
}

// grad_phi_c = -(drho/2) sum over the six faces of beta_f^2 grad_beta_f (order x-,x+,y-,y+,z-,z+).
// A block of W x R threads covers R rows of W cells (W: nx rounded up to a warp multiple, at most
// kPhiW) and walks kPhiRun planes up z.  Each face's product (beta_f beta_f) grad_beta_f is formed
// once: every cell forms those of its x- and y- faces and of the z- face of the cell above; the
// x+ and y+ products are the neighbours' (shared memory, two buffers by plane parity), formed again
// only at the block's right edge and top row, and the z+ product is carried up as the next cell's
// z- product.  The same products summed in the same order as forming all six per cell (0 + t is
// t but for -0; NaN payloads aside).
__global__ void k_phi_grad(int nx, int ny, int nz, double neg_half_drho, const double *__restrict__ bx,
                           const double *__restrict__ by, const double *__restrict__ bz,
                           const double *__restrict__ gbx, const double *__restrict__ gby,
                           const double *__restrict__ gbz, double *__restrict__ gphi)
{
    __shared__ double sh[2][2][kPhiThreads];  // [plane parity][x- / y- product][thread]
    const int W = blockDim.x, R = blockDim.y;
    const int i = blockIdx.x * W + threadIdx.x, j = blockIdx.y * R + threadIdx.y;
    const int t = threadIdx.y * W + threadIdx.x;
    const bool in = i < nx && j < ny;
    const int k0 = blockIdx.z * kPhiRun, k1 = min(k0 + kPhiRun, nz);
    const size_t sxy = (size_t)nx * ny;
    auto prod = [](double b, double g) { return __dmul_rn(__dmul_rn(b, b), g); };
    size_t c = in ? (size_t)k0 * sxy + (size_t)j * nx + i : 0;
    const bool ok0 = in && ck_cell((long long)c, i, j, k0, nx, ny, nz, CK_PHI_GRAD);
    double tz_lo = ok0 ? prod(bz[c], gbz[c]) : 0.0;
    for (int k = k0; k < k1; k++, c += sxy) {
        const bool ok = in && ck_cell((long long)c, i, j, k, nx, ny, nz, CK_PHI_GRAD);
        double tx = 0.0, ty = 0.0, tz_hi = 0.0;
        if (ok) {
            tx = prod(bx[c], gbx[c]);
            ty = prod(by[c], gby[c]);
            if (k < nz - 1) tz_hi = prod(bz[c + sxy], gbz[c + sxy]);
        }
        double(*buf)[kPhiThreads] = sh[k & 1];
        buf[0][t] = tx;
        buf[1][t] = ty;
        __syncthreads();  // one barrier per plane: a buffer is written again two planes later
        if (ok) {
            double tx_hi = 0.0, ty_hi = 0.0;
            if (i < nx - 1) tx_hi = threadIdx.x < W - 1 ? buf[0][t + 1] : sq_mul_call(bx[c + 1], gbx[c + 1]);
            if (j < ny - 1) ty_hi = threadIdx.y < R - 1 ? buf[1][t + W] : sq_mul_call(by[c + nx], gby[c + nx]);
            double s = (__double_as_longlong(tx) << 1) == 0 ? 0.0 : tx;  // 0 + tx
            if (i < nx - 1) s = __dadd_rn(s, tx_hi);
            s = __dadd_rn(s, ty);
            if (j < ny - 1) s = __dadd_rn(s, ty_hi);
            s = __dadd_rn(s, tz_lo);
            if (k < nz - 1) s = __dadd_rn(s, tz_hi);
            gphi[c] = __dmul_rn(neg_half_drho, s);
        }
        tz_lo = tz_hi;
    }
}

// ---------------------------------------------------------------------------
// Multigrid-preconditioned CG (flexible form).  FP64 Krylov vectors; the
// preconditioned vector z is FP64 (plain FP64 solves) or s * e32 with the FP32
// cycle's output e32 and the scale s the FP32 right-hand side was divided by.
// Device scalars (Scal): S_RZ <r,z>, S_RZN / S_RZO new <r,z> and <r,z_old>,
// S_SIGMA <d, A d>, S_RR ||r||^2.
// ---------------------------------------------------------------------------

// r = b - A p (FP64), as residual_at forms it: differences of neighbouring p first, so a large
// smooth offset in p (a hydrostatic pressure) cancels before any product.  Optionally r32 = r /
// scale, scale = RMS of b (first pass) written to scale_slot.  Cell indices by multiply-shift
// division (fnx, fny).
// *flag |= 1 if any p[i] is nonzero (either sign of zero counts as zero); the caller clears it
__global__ void k_nonzero(unsigned n, const double *__restrict__ p, unsigned *__restrict__ flag)
{
    bool any = false;
    const unsigned n2 = n / 2, stride = gridDim.x * blockDim.x;
    const double2 *p2 = reinterpret_cast<const double2 *>(p);
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < n2; v += stride) {
        const double2 x = p2[v];
        any |= ((__double_as_longlong(x.x) | __double_as_longlong(x.y)) << 1) != 0;
    }
    for (unsigned idx = 2 * n2 + blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride)
        any |= (__double_as_longlong(p[idx]) << 1) != 0;
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(flag, 1u);
}

// pnz (optional): the k_nonzero flag of p; 0 means p is zero everywhere, and each cell's
// residual is then b exactly (residual64_at's zero case) with no stencil loaded: the same values
// for a fraction of the loads (the first residual of a solve from a zero guess)
__global__ void k_pcg_resid(int nx, int ny, int nz, double ih2, LevelArrays<double> L, const double *__restrict__ b,
                            const double *__restrict__ p, double *__restrict__ r, float *__restrict__ r32,
                            double *__restrict__ dscal, int scale_slot, double *__restrict__ partials, size_t half,
                            FastDiv fnx, FastDiv fny, const unsigned *__restrict__ pnz)
{
    const bool pzero = pnz && *pnz == 0u;
    const unsigned n = (unsigned)nx * ny * nz;
    const size_t sxy = (size_t)nx * ny;
    const double inv_scale = block_scalar([&] {
        if (!r32) return 1.0;
        const double rms = sqrt(dscal[S_NB2] / dscal[S_NLIVE]);
        const double sc = (rms > 0.0 && isfinite(rms)) ? rms : 1.0;
        if (blockIdx.x == 0) dscal[scale_slot] = sc;
        return 1.0 / sc;
    });
    double rr = 0.0, sp = 0.0;
    // one loop per case of the (grid-uniform) zero test: the zero case's loop holds no stencil
    // arithmetic at all (a select inside one loop would still issue it)
    auto run = [&](auto zero_tag) {
        constexpr bool PZ = decltype(zero_tag)::value;
        for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
            const unsigned t = fdiv(idx, fnx), kk = fdiv(t, fny);
            const int i = (int)(idx - t * (unsigned)nx), k = (int)kk, j = (int)(t - kk * (unsigned)ny);
            const double v = PZ ? b[idx] : residual64_at(i, j, k, idx, nx, ny, nz, sxy, ih2, L, b, p);
            r[idx] = v;
            if (r32) {
                const size_t slot = half ? split_slot(idx, (j + k) & 1, half) : idx;
                if (MG_CK(slot, slot, (long long)n, CK_SPLIT_SLOT)) r32[slot] = narrow(v * inv_scale);
            }
            rr += v * v;
            if (!PZ && pos_bits(L.dinv[idx])) sp += p[idx];
        }
    };
    if (pzero)
        run(BoolTag<true>{});
    else
        run(BoolTag<false>{});
    rr = block_sum<kRedThreads>(rr);
    sp = block_sum<kRedThreads>(sp);
    reduce_finish(rr, sp, partials, dscal, S_RR, S_SUM_P);
}

// <r, z> and <r, z_old> with z = sz * Z, z_old = so * Zo (Z double: scales 1)
template <typename Z>
__global__ void k_pcg_dots(unsigned n, const double *__restrict__ r, const Z *__restrict__ z, const Z *__restrict__ zo,
                           double *dscal, int sz_slot, int so_slot, double *__restrict__ partials)
{
    const double sz = sz_slot >= 0 ? dscal[sz_slot] : 1.0;
    const double so = so_slot >= 0 ? dscal[so_slot] : 1.0;
    double a = 0.0, c = 0.0;
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const double rv = r[idx];
        a = fma(rv, (double)z[idx], a);
        if (zo) c = fma(rv, (double)zo[idx], c);
    }
    a = block_sum<kRedThreads>(a) * sz;
    c = block_sum<kRedThreads>(c) * so;
    reduce_finish(a, c, partials, dscal, S_RZN, S_RZO);
}

// Mixed-precision variant: <r, z> = sr sz <r32, e32> from the FP32 copy r32 = r / sr that the
// preconditioner read.  Products and short per-thread sums are FP32, block sums FP64: the CG
// scalars need only the accuracy of the FP32 preconditioner they weigh.
__global__ void k_pcg_dots32(unsigned n, const float *__restrict__ r32, const float *__restrict__ z,
                             const float *__restrict__ zo, double *dscal, int sr_slot, int sz_slot,
                             int so_slot, double *__restrict__ partials)
{
    const double sr = dscal[sr_slot];
    double a = 0.0, c = 0.0;
    const unsigned n4 = n / 4, stride = gridDim.x * blockDim.x;
    const float4 *r4 = reinterpret_cast<const float4 *>(r32);
    const float4 *z4 = reinterpret_cast<const float4 *>(z);
    const float4 *o4 = reinterpret_cast<const float4 *>(zo);
    // widened on the integer pipe (exact, as the conversion instruction, which runs on the FP64 unit)
    auto dot4 = [](float4 x, float4 y) { return widen(fmaf(x.w, y.w, fmaf(x.z, y.z, fmaf(x.y, y.y, x.x * y.x)))); };
    // float4 groups v and v + stride per iteration, all loads issued first; the sums in the same
    // order as one group per iteration
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < n4; v += 2 * stride) {
        const unsigned w = v + stride;
        const bool has_w = w < n4;
        const float4 rv = r4[v], zv = z4[v], rw = has_w ? r4[w] : zero4, zw = has_w ? z4[w] : zero4;
        const float4 ov = zo ? o4[v] : zero4, ow = (zo && has_w) ? o4[w] : zero4;
        a += dot4(rv, zv);
        if (zo) c += dot4(rv, ov);
        if (has_w) {
            a += dot4(rw, zw);
            if (zo) c += dot4(rw, ow);
        }
    }
    for (unsigned idx = 4 * n4 + blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
        a += widen(r32[idx] * z[idx]);
        if (zo) c += widen(r32[idx] * zo[idx]);
    }
    a = block_sum<kRedThreads>(a) * sr * dscal[sz_slot];
    c = block_sum<kRedThreads>(c) * (so_slot >= 0 ? sr * dscal[so_slot] : 0.0);
    reduce_finish(a, c, partials, dscal, S_RZN, S_RZO);
}

// The search direction d = sz Z + beta d_old, beta = (<r,z> - <r,z_old>) / <r_old, z_old> (first:
// beta = 0), with z = sz Z the preconditioned residual, is kept divided by its z's scale: D = d / sz
// = Z + (beta so / sz) D_old (so: the scale of D_old), one FP64 operation per cell.  The CG
// update then moves p and r by <r,z> / (sz <D, A D>) times D and A D (k_pcg_update), the same
// step.  Without scales (sz_slot, so_slot < 0) D = d.
template <typename Z>
__global__ void k_pcg_dir(unsigned n, const Z *__restrict__ z, double *__restrict__ d, double *dscal,
                          int sz_slot, int so_slot, int first, Split sp, double *__restrict__ partials)
{
    const double beta = block_scalar([&] {
        return first ? 0.0
                     : (dscal[S_RZN] - dscal[S_RZO]) / dscal[S_RZ] *
                           (so_slot >= 0 ? dscal[so_slot] / dscal[sz_slot] : 1.0);
    });
    const unsigned n2 = n / 2, stride = gridDim.x * blockDim.x;
    double2 *d2 = reinterpret_cast<double2 *>(d);
    // the two Z indices of pair v (colour-split Z: the pair's colours sit at slot v of each half)
    auto zidx = [&](unsigned v, size_t &i0, size_t &i1) {
        i0 = 2 * (size_t)v;
        i1 = 2 * (size_t)v + 1;
        if (sp.half) {
            const int q = row_parity(2 * v, sp);
            i0 = (q ? sp.half : 0) + v;
            i1 = (q ? 0 : sp.half) + v;
            return MG_CK(i0, i0, (long long)n, CK_SPLIT_SLOT) && MG_CK(i1, i1, (long long)n, CK_SPLIT_SLOT);
        }
        return true;
    };
    // pairs v and v + stride per iteration, both pairs' loads issued before either update
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < n2; v += 2 * stride) {
        const unsigned w = v + stride;
        const bool has_w = w < n2;
        size_t a0, a1, b0 = 0, b1 = 0;
        const bool ok_v = zidx(v, a0, a1), ok_w = has_w && zidx(w, b0, b1);
        const Z za0 = ok_v ? z[a0] : Z(0), za1 = ok_v ? z[a1] : Z(0);
        const Z zb0 = ok_w ? z[b0] : Z(0), zb1 = ok_w ? z[b1] : Z(0);
        double2 dv = (first || !ok_v) ? make_double2(0.0, 0.0) : d2[v];
        double2 dw = (first || !ok_w) ? make_double2(0.0, 0.0) : d2[w];
        if (ok_v) {
            dv.x = fma(beta, dv.x, widen(za0));
            dv.y = fma(beta, dv.y, widen(za1));
            d2[v] = dv;
        }
        if (ok_w) {
            dw.x = fma(beta, dw.x, widen(zb0));
            dw.y = fma(beta, dw.y, widen(zb1));
            d2[w] = dw;
        }
    }
    for (unsigned idx = 2 * n2 + blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride)
        d[idx] = fma(beta, first ? 0.0 : d[idx], widen(z[idx]));
    // every block has read <r, z> above: the last one moves the new <r, z> into its place
    if (last_block(partials) && threadIdx.x == 0) dscal[S_RZ] = dscal[S_RZN];
}

// Jacobi preconditioner: z = (scale * dinv) * r, dead cells 0
__global__ void k_jacobi(unsigned n, double scale, const double *__restrict__ dinv, const double *__restrict__ r,
                         double *__restrict__ z)
{
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x)
        z[idx] = (scale * dinv[idx]) * r[idx];
}

// q = A d and <d, q>, with A d = sum_f (h^-2 beta_f) d_nb - (h^-2 diag) d_c on arrays pre-scaled
// by h^-2 (L, diag; exact for a power-of-two h): 8 FP64 operations per cell instead of 15 for the
// difference form.  Its rounding error is larger for smooth d (relative ~1e-12 at 256^3), which
// only perturbs the recursive residual; convergence is confirmed on the true residual in
// difference form.
__global__ void k_pcg_apply(int nx, int ny, int nz, LevelArrays<double> L, const double *__restrict__ diag,
                            const double *__restrict__ d, double *__restrict__ q, double *__restrict__ partials,
                            double *dscal)
{
    const unsigned n = (unsigned)nx * ny * nz;
    const size_t sxy = (size_t)nx * ny;
    double dq = 0.0;
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_of(idx, nx, ny, i, j, k);
        if (!ck_cell(idx, i, j, k, nx, ny, nz, CK_PCG_APPLY)) continue;
        const double dc = d[idx];
        double s = -diag[idx] * dc;
        if (i > 0) s = fma(L.bx[idx], d[idx - 1], s);
        if (i < nx - 1) s = fma(L.bx[idx + 1], d[idx + 1], s);
        if (j > 0) s = fma(L.by[idx], d[idx - nx], s);
        if (j < ny - 1) s = fma(L.by[idx + nx], d[idx + nx], s);
        if (k > 0) s = fma(L.bz[idx], d[idx - sxy], s);
        if (k < nz - 1) s = fma(L.bz[idx + sxy], d[idx + sxy], s);
        const double qv = s;
        q[idx] = qv;
        dq = fma(dc, qv, dq);
    }
    reduce_finish(block_sum<kRedThreads>(dq), 0.0, partials, dscal, S_SIGMA, -1);
}

// alpha = <r,z>/<d,Ad>; p += alpha d; r -= alpha q; ||r||^2; optionally r32 = r / scale with
// scale = RMS of the previous residual (written to scale_slot).  Two elements per iteration.
__global__ void k_pcg_update(unsigned n, const double *__restrict__ d, const double *__restrict__ q,
                             double *__restrict__ p, double *__restrict__ r, float *__restrict__ r32,
                             double *dscal, int scale_slot, int sd_slot, double *__restrict__ partials,
                             Split sp)
{
    // d holds D = (direction) / sd (k_pcg_dir): alpha = <r,z> / <d, A d> times sd
    const double alpha =
        block_scalar([&] { return dscal[S_RZ] / (dscal[S_SIGMA] * (sd_slot >= 0 ? dscal[sd_slot] : 1.0)); });
    const double inv_scale = block_scalar([&] {
        if (!r32) return 1.0;
        const double rms = sqrt(dscal[S_RR] / dscal[S_NLIVE]);
        const double sc = (rms > 0.0 && isfinite(rms)) ? rms : 1.0;
        if (blockIdx.x == 0) dscal[scale_slot] = sc;
        return 1.0 / sc;
    });
    const float inv_scale32 = (float)inv_scale;
    double rr = 0.0;
    const unsigned n2 = n / 2, stride = gridDim.x * blockDim.x;
    const double2 *d2 = reinterpret_cast<const double2 *>(d);
    const double2 *q2 = reinterpret_cast<const double2 *>(q);
    double2 *p2 = reinterpret_cast<double2 *>(p);
    double2 *rv2 = reinterpret_cast<double2 *>(r);
    float2 *r32v = reinterpret_cast<float2 *>(r32);
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < n2; v += stride) {
        const double2 dv = d2[v], qv = q2[v];
        double2 pv = p2[v], rv = rv2[v];
        pv.x = fma(alpha, dv.x, pv.x);
        pv.y = fma(alpha, dv.y, pv.y);
        rv.x = fma(-alpha, qv.x, rv.x);
        rv.y = fma(-alpha, qv.y, rv.y);
        p2[v] = pv;
        rv2[v] = rv;
        if (r32) {
            const float r0 = narrow(rv.x) * inv_scale32, r1 = narrow(rv.y) * inv_scale32;
            if (sp.half) {  // colour-split r32: the pair's colours at slot v of each half
                const int qp = row_parity(2 * v, sp);
                r32[(qp ? sp.half : 0) + v] = r0;
                r32[(qp ? 0 : sp.half) + v] = r1;
            } else {
                r32v[v] = make_float2(r0, r1);
            }
        }
        rr = fma(rv.x, rv.x, rr);
        rr = fma(rv.y, rv.y, rr);
    }
    for (unsigned idx = 2 * n2 + blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
        p[idx] = fma(alpha, d[idx], p[idx]);
        const double rv = fma(-alpha, q[idx], r[idx]);
        r[idx] = rv;
        if (r32) r32[idx] = narrow(rv) * inv_scale32;
        rr = fma(rv, rv, rr);
    }
    reduce_finish(block_sum<kRedThreads>(rr), 0.0, partials, dscal, S_RR, -1);
}


// ---------------------------------------------------------------------------
// Connected components of the live cells (cells joined by open faces) and the mean removal of
// the Neumann problem per component (Eq. neumann with Eq. pois: A is singular with one constant
// per component in its null space, so the rhs is projected to zero mean on each component and p
// is pinned to zero mean on each).  Union-find over x-runs:
//   1. each live cell points to the first cell of its run of cells joined by open x-faces;
//   2. each open y- or z-face joins the roots of its two cells (the larger root is hooked under
//      the smaller with atomicMin; a hook that finds the root hooked meanwhile continues with the
//      new parent), except where the face to the left already joined the same two runs;
//   3. every cell takes its root; a root is the smallest cell index of its component.
// Every parent has a smaller index than its child, so the pointers form no cycle and every loop
// below ends; each is still bounded by kCcBudget steps and reports exceeding it in *err.
// ---------------------------------------------------------------------------
constexpr unsigned kCcBudget = 1u << 26;

__device__ __forceinline__ int cc_load(const int *label, int x)
{
    if (!MG_CK(x, x, 0x7fffffffll, CK_LABEL)) return x;
    return *(const volatile int *)(label + x);
}

__device__ __forceinline__ int cc_find(const int *label, int x, unsigned &budget)
{
    int y = cc_load(label, x);
    while (y != x && budget) {
        budget--;
        x = y;
        y = cc_load(label, x);
    }
    return x;
}

__device__ void cc_union(int *label, int a, int b, unsigned *err)
{
    unsigned budget = kCcBudget;
    a = cc_find(label, a, budget);
    b = cc_find(label, b, budget);
    while (a != b && budget) {
        budget--;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(label + b, a);
        if (old == b) return;  // b was a root: now under a
        // b had been hooked under old meanwhile (and is now under min(old, a)): join old and a
        b = cc_find(label, old, budget);
        a = cc_find(label, a, budget);
    }
    if (a != b) atomicOr(err, 1u);
}

// step 1: one warp per x-row; label = first cell of the run (-1 on dead cells)
__global__ void k_cc_rows(int nx, int ny, int nz, const double *__restrict__ dinv, const double *__restrict__ bx,
                          int *__restrict__ label)
{
    const unsigned lane = threadIdx.x & 31u;
    const size_t row = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= (size_t)ny * nz) return;  // uniform across the warp
    const size_t base = row * (size_t)nx;
    int carry = -1;
    for (int i0 = 0; i0 < nx; i0 += 32) {
        const int i = i0 + (int)lane;
        const bool in = i < nx;
        const size_t c = base + (size_t)i;
        const bool live = in && pos_bits(dinv[c]);
        const bool join = live && i > 0 && pos_bits(bx[c]);
        const unsigned starts = __ballot_sync(0xffffffffu, live && !join);
        const unsigned m = starts & (0xffffffffu >> (31u - lane));
        const int start = m ? (int)(base + (size_t)i0 + (31 - __clz((int)m))) : carry;
        if (in) label[c] = live ? start : -1;
        carry = __shfl_sync(0xffffffffu, start, 31);
    }
}

// step 2: join the runs across open y- and z-faces
__global__ void k_cc_merge(int nx, int ny, int nz, const double *__restrict__ bx, const double *__restrict__ by,
                           const double *__restrict__ bz, int *label, unsigned *err)
{
    const unsigned n = (unsigned)nx * ny * nz;
    const unsigned sxy = (unsigned)nx * ny;
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_of(idx, nx, ny, i, j, k);
        // the run continues from the left (its own low x-face open)
        const bool left = i > 0 && pos_bits(bx[idx]);
        if (j > 0 && pos_bits(by[idx])) {
            // implied when the cell to the left is in this run, its y-face is open and its
            // neighbour is in the neighbour's run
            const bool implied = left && pos_bits(by[idx - 1]) && pos_bits(bx[idx - nx]);
            if (!implied) cc_union(label, (int)idx, (int)(idx - nx), err);
        }
        if (k > 0 && pos_bits(bz[idx])) {
            const bool implied = left && pos_bits(bz[idx - 1]) && pos_bits(bx[idx - sxy]);
            if (!implied) cc_union(label, (int)idx, (int)(idx - sxy), err);
        }
    }
}

// step 3: every live cell takes its root; count[0] += number of roots
__global__ void k_cc_flatten(unsigned n, int *label, unsigned *count, unsigned *err)
{
    unsigned roots = 0;
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int l = label[idx];
        if (l < 0) continue;
        unsigned budget = kCcBudget;
        const int r = cc_find(label, l, budget);
        if (!budget) atomicOr(err, 1u);
        label[idx] = r;
        roots += (r == (int)idx);
    }
    roots = __reduce_add_sync(0xffffffffu, roots);
    if ((threadIdx.x & 31u) == 0 && roots) atomicAdd(count, roots);
}

// the roots (one per component) in any order
__global__ void k_cc_roots(unsigned n, const int *__restrict__ label, int *__restrict__ roots, unsigned *slot,
                           unsigned cap)
{
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x)
        if (label[idx] == (int)idx) {
            const unsigned q = atomicAdd(slot, 1u);
            if (q < cap) roots[q] = (int)idx;
        }
}

// root -> component number (its rank among the sorted roots)
__global__ void k_cc_compact(unsigned n, int *__restrict__ label, const int *__restrict__ roots, int ncomp)
{
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int r = label[idx];
        if (r < 0) continue;
        int lo = 0, hi = ncomp - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (roots[mid] < r) lo = mid + 1;
            else hi = mid;
        }
        label[idx] = lo;
    }
}

// per-component sums of v (v null: of 1, the cell counts) over the live cells: each thread sums
// kCcChunk consecutive cells and adds to the component total once per change of component (a
// domain's cells mostly share one)
constexpr unsigned kCcChunk = 64;
__global__ void k_comp_sums(unsigned n, const double *__restrict__ v, const int *__restrict__ comp,
                            double *__restrict__ sums)
{
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned c0 = t * kCcChunk; c0 < n; c0 += stride * kCcChunk) {
        int cur = -1;
        double acc = 0.0;
        const unsigned c1 = min(n, c0 + kCcChunk);
        for (unsigned c = c0; c < c1; c++) {
            const int id = comp[c];
            if (id < 0) continue;
            if (id != cur) {
                if (cur >= 0) atomicAdd(sums + cur, acc);
                cur = id;
                acc = 0.0;
            }
            acc += v ? v[c] : 1.0;
        }
        if (cur >= 0) atomicAdd(sums + cur, acc);
    }
}

// The same sums in a fixed order (bitwise reproducible), eight components per pass: per-block
// sums of the components g0 .. g0+7 into part[q * gridDim.x + block], then summed over the blocks
__global__ void k_comp_sums8(unsigned n, const double *__restrict__ v, const int *__restrict__ comp, int g0,
                             double *__restrict__ part)
{
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int q = comp[idx] - g0;
        if ((unsigned)q < 8u) {
            const double x = v ? v[idx] : 1.0;
#pragma unroll
            for (int r = 0; r < 8; r++)
                if (q == r) acc[r] += x;
        }
    }
#pragma unroll
    for (int r = 0; r < 8; r++) {
        const double t = block_sum<kRedThreads>(acc[r]);
        if (threadIdx.x == 0) part[r * gridDim.x + blockIdx.x] = t;
    }
}
__global__ void k_comp_finish8(const double *__restrict__ part, int nblocks, int g0, int ncomp,
                               double *__restrict__ sums)
{
    for (int r = 0; r < 8; r++) {
        double a = 0.0;
        for (int i = threadIdx.x; i < nblocks; i += blockDim.x) a += part[r * nblocks + i];
        a = block_sum<kRedThreads>(a);
        if (threadIdx.x == 0 && g0 + r < ncomp) sums[g0 + r] = a;
    }
}

// out = v - its component's mean on live cells, 0 elsewhere; partial sums of out^2 and of v
__global__ void k_comp_center(unsigned n, const double *__restrict__ v, const int *__restrict__ comp,
                              const double *__restrict__ sums, const double *__restrict__ cnt,
                              double *__restrict__ out, double *__restrict__ partials)
{
    double a = 0.0, b = 0.0;
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int id = comp[idx];
        double o = 0.0;
        if (id >= 0) {
            o = v[idx] - sums[id] / cnt[id];
            b += v[idx];
        }
        out[idx] = o;
        a += o * o;
    }
    a = block_sum<kRedThreads>(a);
    b = block_sum<kRedThreads>(b);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

// f as a Scale2 (ok when f = 2^e)
inline Scale2 scale2(double f)
{
    int ex;
    const bool ok = std::frexp(f, &ex) == 0.5;
    return Scale2{f, ex - 1, ok ? 1 : 0};
}
// 1/h as a Scale2 for div_h: ok when h is a power of two (h = 2^(ex-1), 1/h = 2^(1-ex) exactly)
inline Scale2 inv_scale2(double h)
{
    int ex;
    const bool ok = std::frexp(h, &ex) == 0.5;
    return Scale2{1.0 / h, 1 - ex, ok ? 1 : 0};
}

inline dim3 row_grid(int threads_x, int ny, int nz)
{
    return dim3((unsigned)((threads_x + kRowThreads - 1) / kRowThreads), (unsigned)ny, (unsigned)nz);
}

// Blocks of kRowThreads threads over rows of threads_x threads each: x the next power of two >=
// threads_x (at most kRowThreads), the rest of the block over consecutive rows, so that a coarse
// level's short rows (32 or 64 threads) do not leave most of each block idle.  Kernels launched so
// take their row from blockIdx.y * blockDim.y + threadIdx.y and skip rows past the last.
inline dim3 row_block2(int threads_x)
{
    int bx = 1;
    while (bx < threads_x && bx < kRowThreads) bx *= 2;
    return dim3((unsigned)bx, (unsigned)(kRowThreads / bx));
}
inline dim3 row_grid2(int threads_x, int ny, int nz)
{
    const dim3 b = row_block2(threads_x);
    return dim3((unsigned)((threads_x + b.x - 1) / b.x), (unsigned)((ny + b.y - 1) / b.y), (unsigned)nz);
}

inline unsigned red_grid(size_t n)
{
    size_t b = (n + kRedThreads - 1) / kRedThreads;
    return (unsigned)(b < (size_t)kRedBlocks ? (b ? b : 1) : kRedBlocks);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_face_coeffs(Dims d, const double *phi, const uint8_t *solid, double rho_a, double drho,
                               double *bx, double *by, double *bz, cudaStream_t s)
{
    note_launch();
    k_face_coeffs<<<run_grid(d.nx, d.ny, d.nz), kRowThreads, 0, s>>>(d.nx, d.ny, d.nz, phi, solid, rho_a, drho, bx, by,
                                                                      bz);
    return cudaGetLastError();
}

cudaError_t launch_jacobi(size_t n, double scale, const double *dinv, const double *r, double *z, cudaStream_t s)
{
    note_launch();
    k_jacobi<<<red_grid(n), kRedThreads, 0, s>>>((unsigned)n, scale, dinv, r, z);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diag_inv(Dims d, const T *bx, const T *by, const T *bz, T *dinv, cudaStream_t s,
                            const LevelArrays<T> *op, T scale, uint8_t *open, double *changed)
{
    note_launch();
    k_diag_inv<T><<<run_grid(d.nx, d.ny, d.nz), kRowThreads, 0, s>>>(d.nx, d.ny, d.nz, bx, by, bz, dinv,
                                                                      op ? *op : LevelArrays<T>{},
                                                                      scale2((double)scale), open, changed);
    return cudaGetLastError();
}
template cudaError_t launch_diag_inv<double>(Dims, const double *, const double *, const double *, double *,
                                             cudaStream_t, const LevelArrays<double> *, double, uint8_t *, double *);

cudaError_t launch_level_f32(Dims d, const LevelArrays<double> &L, LevelArrays<float> &out, cudaStream_t s,
                             LevelArrays<float> *sf, Split sp)
{
    note_launch();
    const bool split = sf && sf->bx && sp.half;
    k_level_f32<<<run_grid(d.nx, d.ny, d.nz), kRowThreads, 0, s>>>(d.nx, d.ny, d.nz, L.bx, L.by, L.bz, out,
                                                                     split ? *sf : LevelArrays<float>{},
                                                                     split ? sp.half : 0);
    return cudaGetLastError();
}

cudaError_t launch_restrict_coeffs(Dims f, const double *bx, const double *by, const double *bz, double *cbx,
                                   double *cby, double *cbz, cudaStream_t s)
{
    note_launch();
    k_restrict_coeffs<<<row_grid(f.nx / 2, f.ny / 2, f.nz / 2), kRowThreads, 0, s>>>(f.nx, f.ny, f.nz, bx, by, bz, cbx,
                                                                                      cby, cbz);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_smooth(Dims d, T h2, const LevelArrays<T> &L, const T *b, T *p, int colour, cudaStream_t s,
                          int z0, int z1, bool zero)
{
    if (z1 < 0) z1 = d.nz;
    if (z1 <= z0) return cudaSuccess;
    note_launch();
    const dim3 g = row_grid2((d.nx + 1) / 2, d.ny, z1 - z0), blk = row_block2((d.nx + 1) / 2);
    if (zero)
        k_smooth<T, true><<<g, blk, 0, s>>>(d.nx, d.ny, d.nz, h2, L, b, p, colour, z0);
    else
        k_smooth<T, false><<<g, blk, 0, s>>>(d.nx, d.ny, d.nz, h2, L, b, p, colour, z0);
    return cudaGetLastError();
}
template cudaError_t launch_smooth<double>(Dims, double, const LevelArrays<double> &, const double *, double *, int,
                                           cudaStream_t, int, int, bool);
template cudaError_t launch_smooth<float>(Dims, float, const LevelArrays<float> &, const float *, float *, int,
                                          cudaStream_t, int, int, bool);

cudaError_t launch_smooth_split(Dims d, float h2, const LevelArrays<float> &L, const float *b, float *p, int colour,
                                cudaStream_t s, const float *urow, const float4 *arow, int rev, bool zero,
                                const LevelArrays<float> *S)
{
    note_launch();
    if (d.nx % 8 == 0) {  // four cells per thread, blocks of 32 threads x 4 rows
        if (!S || !S->bx || !S->by || !S->bz) return cudaErrorInvalidValue;
        const int G = d.nx / 8;
        const dim3 grid((G + 31) / 32, (d.ny + 3) / 4, d.nz), block(32, 4);
        if (arow) {
            if (zero)
                k_smooth_split4<true, true><<<grid, block, 0, s>>>(d.nx, d.ny, d.nz, h2, *S, b, p, colour, urow, arow, rev);
            else
                k_smooth_split4<true, false><<<grid, block, 0, s>>>(d.nx, d.ny, d.nz, h2, *S, b, p, colour, urow, arow,
                                                                    rev);
        } else {
            if (zero)
                k_smooth_split4<false, true><<<grid, block, 0, s>>>(d.nx, d.ny, d.nz, h2, *S, b, p, colour, urow,
                                                                    nullptr, rev);
            else
                k_smooth_split4<false, false><<<grid, block, 0, s>>>(d.nx, d.ny, d.nz, h2, *S, b, p, colour, urow,
                                                                     nullptr, rev);
        }
    } else {
        k_smooth_split<<<row_grid(d.nx / 2, d.ny, d.nz), kRowThreads, 0, s>>>(d.nx, d.ny, d.nz, h2, L, b, p, colour,
                                                                              urow, rev, zero ? 1 : 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_uniform_rows(Dims d, const float *bx, const float *by, const float *bz, float *urow,
                                cudaStream_t s, float4 *arow, unsigned *count)
{
    const int rows = d.ny * d.nz, warps = 8;
    note_launch();
    k_uniform_rows<<<(rows + warps - 1) / warps, 32 * warps, 0, s>>>(d.nx, d.ny, d.nz, bx, by, bz, urow, arow,
                                                                      count);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_resid_restrict(Dims f, T ih2, const LevelArrays<T> &L, const T *b, const T *p, T *bc,
                                  cudaStream_t s, Split sp, const float *urow, int rev)
{
    note_launch();
    const dim3 g = row_grid2(f.nx / 2, f.ny / 2, f.nz / 2), blk = row_block2(f.nx / 2);
    if constexpr (std::is_same<T, float>::value) {
        if (sp.half)
            k_resid_restrict_pairs<true><<<g, blk, 0, s>>>(f.nx, f.ny, f.nz, ih2, L, b, p, bc, sp.half, urow, rev);
        else
            k_resid_restrict_pairs<false><<<g, blk, 0, s>>>(f.nx, f.ny, f.nz, ih2, L, b, p, bc, 0, urow, rev);
    } else {
        if (urow) return cudaErrorInvalidValue;  // uniform rows describe FP32 coefficients
        if (sp.half) return cudaErrorInvalidValue;  // FP64 fields are never split
        k_resid_restrict<T><<<g, blk, 0, s>>>(f.nx, f.ny, f.nz, ih2, L, b, p, bc);
    }
    return cudaGetLastError();
}
template cudaError_t launch_resid_restrict<double>(Dims, double, const LevelArrays<double> &, const double *,
                                                   const double *, double *, cudaStream_t, Split, const float *, int);
template cudaError_t launch_resid_restrict<float>(Dims, float, const LevelArrays<float> &, const float *,
                                                  const float *, float *, cudaStream_t, Split, const float *, int);

template <typename T>
cudaError_t launch_prolong(Dims f, const T *ec, const T *dinv, T *p, cudaStream_t s, Split sp, const float *urow)
{
    note_launch();
    const dim3 g = row_grid2(f.nx / 2, f.ny / 2, f.nz / 2), blk = row_block2(f.nx / 2);
    if constexpr (std::is_same<T, float>::value) {
        if (sp.half) {
            k_prolong<T, true><<<g, blk, 0, s>>>(f.nx, f.ny, f.nz, ec, dinv, p, sp.half, urow);
            return cudaGetLastError();
        }
    } else if (sp.half) {
        return cudaErrorInvalidValue;  // FP64 fields are never split
    }
    k_prolong<T, false><<<g, blk, 0, s>>>(f.nx, f.ny, f.nz, ec, dinv, p, 0, sizeof(T) == 4 ? urow : nullptr);
    return cudaGetLastError();
}
template cudaError_t launch_prolong<double>(Dims, const double *, const double *, double *, cudaStream_t, Split,
                                            const float *);
template cudaError_t launch_prolong<float>(Dims, const float *, const float *, float *, cudaStream_t, Split,
                                           const float *);

// Tiles of 32 x 8 columns; z-chunks sized so that the grid has about 4 CTAs per SM.
template <typename T>
cudaError_t launch_rb_sweep(Dims d, T h2, const LevelArrays<T> &L, const T *b, const T *p_old, T *p_new, int first,
                            cudaStream_t s)
{
    constexpr int TX = 32, TY = 8;
    const int tx = (d.nx + TX - 1) / TX, ty = (d.ny + TY - 1) / TY;
    const int want = 4 * 152;
    int chunks = (want + tx * ty - 1) / (tx * ty);
    int zc = (d.nz + chunks - 1) / chunks;
    if (zc < 8) zc = 8;
    if (zc > d.nz) zc = d.nz;
    const dim3 grid((unsigned)tx, (unsigned)ty, (unsigned)((d.nz + zc - 1) / zc));
    note_launch();
    k_rb_sweep<T, TX, TY><<<grid, (TX + 4) * (TY + 4), 0, s>>>(d.nx, d.ny, d.nz, zc, h2, L, b, p_old, p_new, first);
    return cudaGetLastError();
}
template cudaError_t launch_rb_sweep<double>(Dims, double, const LevelArrays<double> &, const double *,
                                             const double *, double *, int, cudaStream_t);
template cudaError_t launch_rb_sweep<float>(Dims, float, const LevelArrays<float> &, const float *, const float *,
                                            float *, int, cudaStream_t);

template <typename T>
cudaError_t launch_coarse_solve(int n, const double *M, const T *b, T *e, cudaStream_t s)
{
    const int rows_per_cta = 8;  // one warp per row
    note_launch();
    k_coarse_solve<T><<<(n + rows_per_cta - 1) / rows_per_cta, 32 * rows_per_cta, (size_t)n * sizeof(double), s>>>(n, M, b,
                                                                                                                e);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_tail_down(const TailArgs<T> &a, cudaStream_t s)
{
    if (a.nlev < 2 || a.nlev > kTailMaxLevels) return cudaErrorInvalidValue;
    note_launch();
    k_tail_down<T><<<1, kTailDownThreads, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_tail_up(const TailArgs<T> &a, cudaStream_t s)
{
    if (a.nlev < 2 || a.nlev > kTailMaxLevels) return cudaErrorInvalidValue;
    note_launch();
    k_tail_up<T><<<1, kTailUpThreads, 0, s>>>(a);
    return cudaGetLastError();
}
template cudaError_t launch_tail_down<double>(const TailArgs<double> &, cudaStream_t);
template cudaError_t launch_tail_down<float>(const TailArgs<float> &, cudaStream_t);
template cudaError_t launch_tail_up<double>(const TailArgs<double> &, cudaStream_t);
template cudaError_t launch_tail_up<float>(const TailArgs<float> &, cudaStream_t);

template cudaError_t launch_coarse_solve<double>(int, const double *, const double *, double *, cudaStream_t);
template cudaError_t launch_coarse_solve<float>(int, const double *, const float *, float *, cudaStream_t);

cudaError_t launch_components(Dims d, const double *dinv, const double *bx, const double *by, const double *bz,
                              int *label, unsigned *ctr, cudaStream_t s)
{
    const unsigned n = (unsigned)d.n();
    cudaError_t e = cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const size_t rows = (size_t)d.ny * d.nz;
    note_launch();
    k_cc_rows<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(d.nx, d.ny, d.nz, dinv, bx, label);
    note_launch();
    k_cc_merge<<<red_grid(n), kRedThreads, 0, s>>>(d.nx, d.ny, d.nz, bx, by, bz, label, ctr + 1);
    note_launch();
    k_cc_flatten<<<red_grid(n), kRedThreads, 0, s>>>(n, label, ctr, ctr + 1);
    return cudaGetLastError();
}

cudaError_t launch_component_roots(size_t n, const int *label, int *roots, unsigned *slot, unsigned cap,
                                   cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(slot, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    note_launch();
    k_cc_roots<<<red_grid(n), kRedThreads, 0, s>>>((unsigned)n, label, roots, slot, cap);
    return cudaGetLastError();
}

cudaError_t launch_component_compact(size_t n, int *label, const int *sorted_roots, int ncomp, double *cnt,
                                     double *part, cudaStream_t s)
{
    note_launch();
    k_cc_compact<<<red_grid(n), kRedThreads, 0, s>>>((unsigned)n, label, sorted_roots, ncomp);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_comp_sums(n, nullptr, label, ncomp, cnt, part, s);
}

cudaError_t launch_comp_sums(size_t n, const double *v, const int *comp, int ncomp, double *sums, double *part,
                             cudaStream_t s)
{
    if (ncomp <= kCompOrdered) {  // fixed order, eight components per pass
        const unsigned g = red_grid(n);
        for (int g0 = 0; g0 < ncomp; g0 += 8) {
            note_launch();
            k_comp_sums8<<<g, kRedThreads, 0, s>>>((unsigned)n, v, comp, g0, part);
            note_launch();
            k_comp_finish8<<<1, kRedThreads, 0, s>>>(part, (int)g, g0, ncomp, sums);
        }
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(sums, 0, (size_t)ncomp * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const unsigned threads = (unsigned)((n + kCcChunk - 1) / kCcChunk);
    note_launch();
    k_comp_sums<<<red_grid(threads), kRedThreads, 0, s>>>((unsigned)n, v, comp, sums);
    return cudaGetLastError();
}

cudaError_t launch_comp_center(size_t n, const double *v, const int *comp, int ncomp, double *sums,
                               const double *cnt, double *out, double *partials, double *dscal, int slot_sq,
                               int slot_sum, cudaStream_t s, double *part)
{
    cudaError_t e = launch_comp_sums(n, v, comp, ncomp, sums, part, s);
    if (e != cudaSuccess) return e;
    const unsigned g = red_grid(n);
    note_launch();
    k_comp_center<<<g, kRedThreads, 0, s>>>((unsigned)n, v, comp, sums, cnt, out, partials);
    note_launch();
    k_finish2<<<1, kRedThreads, 0, s>>>(partials, (int)g, dscal, slot_sq, slot_sum);
    return cudaGetLastError();
}

cudaError_t launch_count_live(Dims d, const double *dinv, double *partials, double *dscal, cudaStream_t s)
{
    const unsigned g = red_grid(d.n());
    note_launch();
    k_count_live<<<g, kRedThreads, 0, s>>>((unsigned)d.n(), dinv, partials, dscal);
    return cudaGetLastError();
}

cudaError_t launch_rhs_prepare(Dims d, const double *rhs, const double *dinv, double *b0, double *partials,
                               double *dscal, cudaStream_t s)
{
    const unsigned g = red_grid(d.n());
    note_launch();
    k_sum_live<<<g, kRedThreads, 0, s>>>((unsigned)d.n(), rhs, dinv, partials, dscal);
    note_launch();
    k_rhs_center<<<g, kRedThreads, 0, s>>>((unsigned)d.n(), rhs, dinv, b0, dscal, partials);
    return cudaGetLastError();
}

cudaError_t launch_resid_norm(Dims d, double ih2, const LevelArrays<double> &L, const double *b, const double *p,
                              double *partials, double *dscal, cudaStream_t s)
{
    const unsigned g = red_grid(d.n());
    note_launch();
    k_resid_norm<<<g, kRedThreads, 0, s>>>(d.nx, d.ny, d.nz, ih2, L, b, p, partials, dscal);
    return cudaGetLastError();
}

cudaError_t launch_sub_mean_p(Dims d, const double *dinv, double *p, const double *dscal, cudaStream_t s)
{
    note_launch();
    k_sub_mean_p<<<red_grid(d.n()), kRedThreads, 0, s>>>((unsigned)d.n(), dinv, p, dscal);
    return cudaGetLastError();
}

cudaError_t launch_resid_cast(Dims d, double ih2, const LevelArrays<double> &L, const double *b, const double *p,
                              float *r32, double *partials, double *dscal, int scale_in, int scale_out,
                              cudaStream_t s, Split sp)
{
    const unsigned g = red_grid(d.n());
    if (scale_in < 0) {  // first pass: scale from ||b0||
        scale_in = S_SCALE0;
        note_launch();
        k_scale_from_nb2<<<1, 1, 0, s>>>(dscal, scale_in);
    }
    note_launch();
    k_resid_cast<<<g, kRedThreads, 0, s>>>(d.nx, d.ny, d.nz, ih2, L, b, p, r32, dscal, scale_in, scale_out, partials,
                                           sp.half);
    return cudaGetLastError();
}

cudaError_t launch_to_f32_layout(size_t n, const double *src, float *dst, cudaStream_t s, Split sp)
{
    note_launch();
    k_to_f32_layout<<<red_grid(n), kRedThreads, 0, s>>>((unsigned)n, src, dst, sp);
    return cudaGetLastError();
}

cudaError_t launch_from_f32_layout(size_t n, const float *src, double *dst, cudaStream_t s, Split sp)
{
    note_launch();
    k_from_f32_layout<<<red_grid(n), kRedThreads, 0, s>>>((unsigned)n, src, dst, sp);
    return cudaGetLastError();
}

cudaError_t launch_accumulate(Dims d, const double *dinv, const float *e32, double *p, const double *dscal,
                              int scale_slot, cudaStream_t s, Split sp)
{
    note_launch();
    (void)dinv;
    k_accumulate<<<red_grid(d.n()), kRedThreads, 0, s>>>((unsigned)d.n(), e32, p, dscal, scale_slot, sp);
    return cudaGetLastError();
}

cudaError_t launch_divergence(Dims d, double scale, const double *bx, const double *by, const double *bz,
                              const double *ux, const double *uy, const double *uz, double *rhs, cudaStream_t s)
{
    note_launch();
    k_divergence<<<row_grid(d.nx, d.ny, d.nz), kRowThreads, 0, s>>>(d.nx, d.ny, d.nz, scale2(scale), bx, by, bz, ux, uy, uz,
                                                                     rhs);
    return cudaGetLastError();
}

cudaError_t launch_correct(Dims d, double dt, double h, const double *bx, const double *by, const double *bz,
                           const double *p, const double *ux0, const double *uy0, const double *uz0, double *ux,
                           double *uy, double *uz, cudaStream_t s, const LevelArrays<double> *val)
{
    note_launch();
    k_correct<<<row_grid(d.nx, d.ny, d.nz), kRowThreads, 0, s>>>(d.nx, d.ny, d.nz, dt, h, inv_scale2(h), bx, by, bz, p,
                                                                  ux0, uy0, uz0, ux, uy, uz,
                                                                  val ? *val : LevelArrays<double>{});
    return cudaGetLastError();
}

cudaError_t launch_face_areas(Dims d, const double *psi, double *ax, double *ay, double *az, cudaStream_t s)
{
    note_launch();
    k_face_areas<<<row_grid(d.nx, d.ny, d.nz), kRowThreads, 0, s>>>(d.nx, d.ny, d.nz, psi, ax, ay, az);
    return cudaGetLastError();
}

cudaError_t launch_stretched_metrics(Dims d, const double *hx, const double *hy, const double *hz,
                                    const LevelArrays<double> &beta, const LevelArrays<double> &frac,
                                    const LevelArrays<double> &bout, const LevelArrays<double> &aout, cudaStream_t s)
{
    note_launch();
    k_stretched_metrics<<<row_grid(d.nx, d.ny, d.nz), kRowThreads, 0, s>>>(d.nx, d.ny, d.nz, hx, hy, hz, beta, frac,
                                                                           bout, aout);
    return cudaGetLastError();
}

cudaError_t launch_rk_combine(size_t n, const LevelArrays<double> &a, const LevelArrays<double> &b,
                              const LevelArrays<double> &r, double dt, const LevelArrays<double> &out, cudaStream_t s)
{
    note_launch();
    k_rk_combine<<<red_grid(n), kRedThreads, 0, s>>>(n, a, b, r, dt, out);
    return cudaGetLastError();
}

cudaError_t launch_momentum_rhs(Dims d, double h, const double *phi, double mu_air, double mu_water, double inv_re,
                                double g, int convect, const LevelArrays<double> &beta, const LevelArrays<double> &u,
                                const LevelArrays<double> &r, double *work, cudaStream_t s)
{
    MomArgs m;
    m.nx = d.nx;
    m.ny = d.ny;
    m.nz = d.nz;
    m.convect = convect ? 1 : 0;
    m.ih = 1.0 / h;
    m.mu_air = mu_air;
    m.dmu = mu_water - mu_air;
    m.inv_re = inv_re;
    m.g = g;
    m.phi = phi;
    m.beta = beta;
    m.u = u;
    m.r = r;
    m.w = work;
    const dim3 g2 = row_grid2(d.nx, d.ny, d.nz), blk = row_block2(d.nx);
    note_launch();
    k_mom_parts<<<g2, blk, 0, s>>>(m);
    note_launch();
    k_mom_combine<<<g2, blk, 0, s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_half(size_t n, const LevelArrays<double> &a, const LevelArrays<double> &b,
                        const LevelArrays<double> &out, cudaStream_t s)
{
    note_launch();
    k_half<<<red_grid(n), kRedThreads, 0, s>>>(n, a, b, out);
    return cudaGetLastError();
}

cudaError_t launch_vof_upwind(Dims d, double s_dt_h, const LevelArrays<double> &mask, const LevelArrays<double> &u,
                              const double *phi, double *phi_out, cudaStream_t s)
{
    note_launch();
    k_vof_upwind<<<row_grid(d.nx, d.ny, d.nz), kRowThreads, 0, s>>>(d.nx, d.ny, d.nz, s_dt_h, mask, u, phi, phi_out);
    return cudaGetLastError();
}

cudaError_t launch_area_coeffs(size_t n, const LevelArrays<double> &area, const LevelArrays<double> &beta,
                               const LevelArrays<double> &out, cudaStream_t s)
{
    note_launch();
    k_area_coeffs<<<red_grid(n), kRedThreads, 0, s>>>(n, area, beta, out);
    return cudaGetLastError();
}

cudaError_t launch_divergence_area(Dims d, double scale, const LevelArrays<double> &mask,
                                   const LevelArrays<double> &area, const LevelArrays<double> &u,
                                   const LevelArrays<double> &v, double *rhs, cudaStream_t s)
{
    note_launch();
    k_divergence_area<<<row_grid(d.nx, d.ny, d.nz), kRowThreads, 0, s>>>(d.nx, d.ny, d.nz, scale, mask, area, u, v,
                                                                         rhs);
    return cudaGetLastError();
}

// blocks of the kernels that share face products along rows (k_phi_grad, k_divergence_mul): W x R
// threads, a row rounded up to whole warps (at most kPhiW cells) by as many rows as fit
inline void row_share_grid(Dims d, dim3 &grid, dim3 &block)
{
    const int W = std::min((d.nx + 31) / 32 * 32, kPhiW), R = std::max(1, std::min(kPhiThreads / W, d.ny));
    grid = dim3((unsigned)((d.nx + W - 1) / W), (unsigned)((d.ny + R - 1) / R), (unsigned)((d.nz + kPhiRun - 1) / kPhiRun));
    block = dim3((unsigned)W, (unsigned)R);
}

cudaError_t launch_divergence_mul(Dims d, double scale, const LevelArrays<double> &L, const LevelArrays<double> &B,
                                  const double *wx, const double *wy, const double *wz, double *rhs, cudaStream_t s)
{
    note_launch();
    dim3 grid, block;
    row_share_grid(d, grid, block);
    k_divergence_mul<<<grid, block, 0, s>>>(d.nx, d.ny, d.nz, scale2(scale), L, B, wx, wy, wz, rhs);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_faces(Dims d, double h, double dt, const double *bx, const double *by, const double *bz,
                                 const double *p, const double *q, const double *wx, const double *wy,
                                 const double *wz, double *gux, double *guy, double *guz, double *gbx, double *gby,
                                 double *gbz, cudaStream_t s, const LevelArrays<double> *area)
{
    note_launch();
    k_adjoint_faces<<<row_grid(d.nx, d.ny, d.nz), kRowThreads, 0, s>>>(d.nx, d.ny, d.nz, h, inv_scale2(h), dt, bx, by,
                                                                        bz, p, q, wx, wy, wz, gux, guy, guz, gbx, gby,
                                                                        gbz, area ? *area : LevelArrays<double>{});
    return cudaGetLastError();
}

cudaError_t launch_phi_grad(Dims d, double neg_half_drho, const double *bx, const double *by, const double *bz,
                            const double *gbx, const double *gby, const double *gbz, double *gphi, cudaStream_t s)
{
    note_launch();
    dim3 grid, block;
    row_share_grid(d, grid, block);
    k_phi_grad<<<grid, block, 0, s>>>(d.nx, d.ny, d.nz, neg_half_drho, bx, by, bz, gbx, gby, gbz, gphi);
    return cudaGetLastError();
}


cudaError_t launch_pcg_resid(Dims d, double ih2, const LevelArrays<double> &L, const double *b, const double *p,
                             double *r, float *r32, double *partials, double *dscal, int scale_slot, cudaStream_t s,
                             Split sp, unsigned *pnz)
{
    const unsigned g = red_grid(d.n());
    if (pnz) {  // is p zero everywhere?
        cudaError_t e = cudaMemsetAsync(pnz, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        note_launch();
        k_nonzero<<<g, kRedThreads, 0, s>>>((unsigned)d.n(), p, pnz);
    }
    note_launch();
    k_pcg_resid<<<g, kRedThreads, 0, s>>>(d.nx, d.ny, d.nz, ih2, L, b, p, r, r32, dscal, scale_slot, partials, sp.half,
                                          make_fastdiv((unsigned)d.nx), make_fastdiv((unsigned)d.ny), pnz);
    return cudaGetLastError();
}

template <typename Z>
cudaError_t launch_pcg_dots(size_t n, const double *r, const Z *z, const Z *zo, double *partials, double *dscal,
                            int sz_slot, int so_slot, cudaStream_t s)
{
    const unsigned g = red_grid(n);
    note_launch();
    k_pcg_dots<Z><<<g, kRedThreads, 0, s>>>((unsigned)n, r, z, zo, dscal, sz_slot, so_slot, partials);
    return cudaGetLastError();
}
cudaError_t launch_pcg_dots32(size_t n, const float *r32, const float *z, const float *zo, double *partials,
                              double *dscal, int sr_slot, int sz_slot, int so_slot, cudaStream_t s)
{
    const unsigned g = red_grid(n);
    note_launch();
    k_pcg_dots32<<<g, kRedThreads, 0, s>>>((unsigned)n, r32, z, zo, dscal, sr_slot, sz_slot, so_slot, partials);
    return cudaGetLastError();
}
template cudaError_t launch_pcg_dots<double>(size_t, const double *, const double *, const double *, double *,
                                             double *, int, int, cudaStream_t);
template cudaError_t launch_pcg_dots<float>(size_t, const double *, const float *, const float *, double *, double *,
                                            int, int, cudaStream_t);

template <typename Z>
cudaError_t launch_pcg_dir(size_t n, const Z *z, double *d, double *dscal, int sz_slot, int so_slot, int first,
                           cudaStream_t s, Split sp, double *partials)
{
    if (sp.half && sizeof(Z) != 4) return cudaErrorInvalidValue;  // FP64 fields are never split
    if (so_slot >= 0 && sz_slot < 0) return cudaErrorInvalidValue;
    note_launch();
    k_pcg_dir<Z><<<red_grid(n), kRedThreads, 0, s>>>((unsigned)n, z, d, dscal, sz_slot, so_slot, first, sp, partials);
    return cudaGetLastError();
}
template cudaError_t launch_pcg_dir<double>(size_t, const double *, double *, double *, int, int, int, cudaStream_t,
                                            Split, double *);
template cudaError_t launch_pcg_dir<float>(size_t, const float *, double *, double *, int, int, int, cudaStream_t,
                                           Split, double *);

cudaError_t launch_pcg_apply(Dims d, const LevelArrays<double> &op, const double *dv, double *q, double *partials,
                             double *dscal, cudaStream_t s)
{
    const unsigned g = red_grid(d.n());
    note_launch();
    k_pcg_apply<<<g, kRedThreads, 0, s>>>(d.nx, d.ny, d.nz, op, op.dinv, dv, q, partials, dscal);
    return cudaGetLastError();
}

cudaError_t launch_pcg_update(size_t n, const double *dv, const double *q, double *p, double *r, float *r32,
                              double *partials, double *dscal, int scale_slot, int sd_slot, cudaStream_t s, Split sp)
{
    const unsigned g = red_grid(n);
    if (sd_slot >= 0 && sd_slot == scale_slot) return cudaErrorInvalidValue;  // read and written by the kernel
    note_launch();
    k_pcg_update<<<g, kRedThreads, 0, s>>>((unsigned)n, dv, q, p, r, r32, dscal, scale_slot, sd_slot, partials, sp);
    return cudaGetLastError();
}

int check_read(unsigned long long *first, unsigned long long *count)
{
#ifdef MGP_CHECK
    cudaError_t e = cudaMemcpyFromSymbol(first, g_check_first, sizeof *first);
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(count, g_check_count, sizeof *count);
    const unsigned long long zero = 0;
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_check_first, &zero, sizeof zero);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_check_count, &zero, sizeof zero);
    return e == cudaSuccess ? 1 : -1;
#else
    *first = 0;
    *count = 0;
    return 0;
#endif
}

}  // namespace mg
