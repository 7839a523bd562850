// mg_noalloc.cu -- residual check that allocates no memory.
//
// Some callers cannot call cudaMalloc: applications whose device memory is all
// owned by a pool or arena they must not bypass, time-critical loops where an
// allocation (which may synchronise the device) is not allowed, and embedding
// hosts that expose no allocator to plug-ins.  For them this file provides
// mg_residual_norm_noalloc, a variant of the solver's residual-norm reduction
// whose only scratch memory is a file-scope __device__ array: two slots of
// partial sums per z-plane, at most MG_NOALLOC_MAX_PLANES planes.  Every GPU that
// loads the library holds that array (128 KB) until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "mg_internal.cuh"

namespace {

constexpr int kPlaneThreads = 256;
constexpr int kMaxDevices = 64;

// Scratch: [0, 2P) pass-1 partials (sum of rhs, live count) per plane,
// [2P, 4P) pass-2 partials (||b0||^2, ||b0 - A p||^2) per plane, then 2 totals
// (mean, live count).  Every slot a call reads is written earlier in that call.
constexpr int kSlots = 4 * MG_NOALLOC_MAX_PLANES + 2;
static __device__ __align__(256) double g_noalloc_scratch[kSlots];

// Host-side cache of the array's device address, one per device (the symbol's
// name is only a host stand-in; kernels must be given the real address).  The
// address belongs to the device's context: after cudaDeviceReset on a device the
// cached entry is stale, and the library must not be called again on that device
// in this process.
double *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum(double v)
{
    __shared__ double sh[kPlaneThreads / 32];
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) r = warp_sum(l < kPlaneThreads / 32 ? sh[l] : 0.0);
    __syncthreads();
    return r;
}

// a cell is live iff at least one of its six faces is open
__device__ __forceinline__ bool live_at(int i, int j, int k, size_t c, int nx, int ny, int nz, size_t sxy,
                                        const double *bx, const double *by, const double *bz)
{
    double s = bx[c];
    s += (i < nx - 1) ? bx[c + 1] : 0.0;
    s += by[c];
    s += (j < ny - 1) ? by[c + nx] : 0.0;
    s += bz[c];
    s += (k < nz - 1) ? bz[c + sxy] : 0.0;
    return s > 0.0;
}

// pass 1: one block per z-plane: sum of rhs over live cells and number of live cells
__global__ void k_plane_pass1(int nx, int ny, int nz, const double *__restrict__ bx, const double *__restrict__ by,
                              const double *__restrict__ bz, const double *__restrict__ rhs, double *scratch)
{
    const int k = blockIdx.x;
    const size_t sxy = (size_t)nx * ny;
    double s = 0.0, cnt = 0.0;
    for (int t = threadIdx.x; t < nx * ny; t += blockDim.x) {
        const int j = t / nx, i = t - j * nx;
        const size_t c = (size_t)k * sxy + t;
        if (live_at(i, j, k, c, nx, ny, nz, sxy, bx, by, bz)) {
            s += rhs[c];
            cnt += 1.0;
        }
    }
    s = block_sum(s);
    cnt = block_sum(cnt);
    if (threadIdx.x == 0) {
        scratch[2 * k] = s;
        scratch[2 * k + 1] = cnt;
    }
}

// one block: plane partials of pass 1 summed by a strided loop and a block reduction (a fixed
// order, so the result is deterministic) -> (mean of rhs, live count)
__global__ void k_plane_totals(int nz, const double *scratch_in, double *totals)
{
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        a += scratch_in[2 * k];
        b += scratch_in[2 * k + 1];
    }
    a = block_sum(a);
    b = block_sum(b);
    if (threadIdx.x == 0) {
        totals[0] = b > 0.0 ? a / b : 0.0;
        totals[1] = b;
    }
}

// pass 2: b0 = rhs - mean on live cells (0 elsewhere); ||b0||^2 and ||b0 - A p||^2 per plane.
// r = b0 - h^-2 sum_f beta_f (p_nb - p_c), products accumulated with fma in the order
// x-, x+, y-, y+, z-, z+ (the solver's residual).
__global__ void k_plane_pass2(int nx, int ny, int nz, double ih2, const double *__restrict__ bx,
                              const double *__restrict__ by, const double *__restrict__ bz,
                              const double *__restrict__ rhs, const double *__restrict__ p, const double *totals,
                              double *scratch_out)
{
    const int k = blockIdx.x;
    const size_t sxy = (size_t)nx * ny;
    const double mean = totals[0];
    double bb = 0.0, rr = 0.0;
    for (int t = threadIdx.x; t < nx * ny; t += blockDim.x) {
        const int j = t / nx, i = t - j * nx;
        const size_t c = (size_t)k * sxy + t;
        const double b0 = live_at(i, j, k, c, nx, ny, nz, sxy, bx, by, bz) ? rhs[c] - mean : 0.0;
        const double pc = p[c];
        double s = 0.0;
        if (i > 0) s = fma(bx[c], p[c - 1] - pc, s);
        if (i < nx - 1) s = fma(bx[c + 1], p[c + 1] - pc, s);
        if (j > 0) s = fma(by[c], p[c - nx] - pc, s);
        if (j < ny - 1) s = fma(by[c + nx], p[c + nx] - pc, s);
        if (k > 0) s = fma(bz[c], p[c - sxy] - pc, s);
        if (k < nz - 1) s = fma(bz[c + sxy], p[c + sxy] - pc, s);
        const double r = fma(-s, ih2, b0);
        bb += b0 * b0;
        rr += r * r;
    }
    bb = block_sum(bb);
    rr = block_sum(rr);
    if (threadIdx.x == 0) {
        scratch_out[2 * k] = bb;
        scratch_out[2 * k + 1] = rr;
    }
}

__global__ void k_noalloc_finish(int nz, const double *scratch_out, const double *totals, double *out)
{
    double bb = 0.0, rr = 0.0;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        bb += scratch_out[2 * k];
        rr += scratch_out[2 * k + 1];
    }
    bb = block_sum(bb);
    rr = block_sum(rr);
    if (threadIdx.x == 0) {
        out[0] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        out[1] = sqrt(bb);
        out[2] = totals[0];
        out[3] = totals[1];
    }
}

int noalloc_fail(int code, const char *msg)
{
    mg::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int mg_residual_norm_noalloc(const mg_grid *g, const double *const beta[3], const double *rhs,
                                        const double *p, double *out, void *stream)
{
    mg::set_last_error("");
    if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1 || !(g->h > 0.0) || !std::isfinite(g->h) ||
        (double)g->nx * g->ny * g->nz >= 2147483647.0)
        return noalloc_fail(MG_ERR_ARG, "mg_residual_norm_noalloc: bad grid");
    if (g->nz > MG_NOALLOC_MAX_PLANES) {
        char buf[160];
        snprintf(buf, sizeof buf,
                 "mg_residual_norm_noalloc: nz = %d exceeds the static scratch limit of %d z-planes", g->nz,
                 MG_NOALLOC_MAX_PLANES);
        return noalloc_fail(MG_ERR_ARG, buf);
    }
    if (!beta || !beta[0] || !beta[1] || !beta[2] || !rhs || !p || !out)
        return noalloc_fail(MG_ERR_ARG, "mg_residual_norm_noalloc: null pointer");
    for (const void *q : {(const void *)beta[0], (const void *)beta[1], (const void *)beta[2], (const void *)rhs,
                          (const void *)p, (const void *)out})
        if (reinterpret_cast<uintptr_t>(q) % 16 != 0)
            return noalloc_fail(MG_ERR_ARG, "mg_residual_norm_noalloc: arrays must be 16-byte aligned");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return noalloc_fail(MG_ERR_CUDA, "mg_residual_norm_noalloc: no current CUDA device");
    }
    double *scratch = nullptr;
    {
        // one-time set-up per device (with that device current): the array's address
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return noalloc_fail(MG_ERR_CUDA, "mg_residual_norm_noalloc: cudaGetSymbolAddress failed");
            }
            g_scratch_addr[dev] = (double *)ptr;
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    double *pass1 = scratch;
    double *pass2 = scratch + 2 * MG_NOALLOC_MAX_PLANES;
    double *totals = scratch + 4 * MG_NOALLOC_MAX_PLANES;
    k_plane_pass1<<<nz, kPlaneThreads, 0, s>>>(nx, ny, nz, beta[0], beta[1], beta[2], rhs, pass1);
    k_plane_totals<<<1, kPlaneThreads, 0, s>>>(nz, pass1, totals);
    k_plane_pass2<<<nz, kPlaneThreads, 0, s>>>(nx, ny, nz, 1.0 / (g->h * g->h), beta[0], beta[1], beta[2], rhs, p,
                                               totals, pass2);
    k_noalloc_finish<<<1, kPlaneThreads, 0, s>>>(nz, pass2, totals, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(MG_ERR_CUDA, cudaGetErrorString(e));
    return MG_OK;
}
