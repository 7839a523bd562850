// mg_sweep_tma.cu -- fused red-black sweep (FP32) with TMA-staged planes.
//
// One launch performs one full red-black Gauss-Seidel sweep of a grid level (the
// smoother of the multigrid cycle), first colour then second, reading the iterate
// from p_old and writing p_new.  Each CTA owns a TX x TY tile of columns and a
// chunk of z-planes and marches up the chunk with a two-plane wavefront: at step s
// it updates the first colour on plane s, then the second colour on plane s-1.
// The first colour on a one-cell ring around the tile (and on one plane below and
// above the chunk) is recomputed from p_old exactly as the neighbouring CTA does,
// so CTAs never depend on each other.  Per cell the arithmetic is that of the
// per-colour smoother (fused multiply-adds in the order x-, x+, y-, y+, z-, z+),
// so the result is bit-identical to two colour passes.
//
// Data movement: one elected thread streams whole plane tiles of the five inputs
// (p, bx, by, bz, b) from HBM into a ring of shared-memory stages with TMA
// (cp.async.bulk.tensor.3d, completion counted on one mbarrier per stage), several
// planes ahead of the compute.  The tile is (TX + 8) x (TY + 4): a halo of 4
// columns in x keeps every copy's start on a 16-byte boundary, 2 rows in y; cells
// outside the grid arrive as zeros.  Every mbarrier wait is bounded: on timeout the
// CTA records an error in dscal[S_ERR] and returns (the host reports it).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <tuple>

#include "mg_internal.cuh"

namespace mg {
namespace {

#ifndef MG_TMA_TX
#define MG_TMA_TX 32
#endif
#ifndef MG_TMA_TY
#define MG_TMA_TY 8
#endif
#ifndef MG_TMA_STAGES
#define MG_TMA_STAGES 6
#endif
#ifndef MG_TMA_CTAS_PER_SM
#define MG_TMA_CTAS_PER_SM 3
#endif
constexpr int TX = MG_TMA_TX, TY = MG_TMA_TY;  // interior tile
constexpr int BW = TX + 8;           // TMA box width (x halo 4 each side)
constexpr int BH = TY + 4;           // TMA box height (y halo 2 each side)
constexpr int CW = TX + 2, CH = TY + 2;  // compute region: interior + ring 1
constexpr int NA = 5;                // arrays per plane: p, bx, by, bz, b (1/diag is formed on the fly)
constexpr int STAGES = MG_TMA_STAGES;  // resident planes s-1, s, s+1, the rest in flight
constexpr int TILE = BW * BH;        // floats per array tile (a multiple of 32 floats = 128 B)
static_assert((TILE * sizeof(float)) % 128 == 0, "tiles must stay 128-byte aligned");
constexpr int THREADS = CW * CH;
constexpr size_t SMEM_BYTES = (size_t)STAGES * NA * TILE * sizeof(float) + STAGES * sizeof(unsigned long long) + 128;
constexpr long kWaitLimit = 1L << 24;

enum { A_P = 0, A_BX = 1, A_BY = 2, A_BZ = 3, A_B = 4 };

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bounded wait for the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    const unsigned a = smem_u32(bar);
    for (long it = 0; it < kWaitLimit; it++) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

struct Maps {
    CUtensorMap m[NA];
};

// 1 / (sum of the six face coefficients), summed in the order of the per-colour smoother
__device__ __forceinline__ float inv_diag32(float bxl, float bxh, float byl, float byh, float bzl, float bzh)
{
    const float sum = ((((bxl + bxh) + byl) + byh) + bzl) + bzh;
    return sum > 0.f ? 1.f / sum : 0.f;
}

__global__ void __launch_bounds__(THREADS) k_rb_sweep_tma(const __grid_constant__ Maps maps, int nx, int ny, int nz,
                                                          int zc, float h2, float *__restrict__ p_new, int first,
                                                          double *__restrict__ dscal)
{
    extern __shared__ unsigned char smem_raw[];
    float *tiles = (float *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    unsigned long long *bars = (unsigned long long *)(tiles + (size_t)STAGES * NA * TILE);

    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, nz);
    const int zfirst = z0 - 2;  // first plane staged
    const int zlast = z1 + 1;   // last plane needed
    const int lx = threadIdx.x % CW, ly = threadIdx.x / CW;
    const int i = x0 - 1 + lx, j = y0 - 1 + ly;  // ring 1 + interior
    const int sx = lx + 3, sy = ly + 1;          // position in the staged tile
    const bool dom = (i >= 0 && i < nx && j >= 0 && j < ny);
    const bool inner = dom && lx >= 1 && lx <= TX && ly >= 1 && ly <= TY;
    const bool xlo = i > 0, xhi = i < nx - 1, ylo = j > 0, yhi = j < ny - 1;
    const int second = first ^ 1;
    const size_t sxy = (size_t)nx * ny;
    const size_t col = dom ? (size_t)j * nx + i : 0;
    const unsigned stage_bytes = NA * TILE * sizeof(float);

    auto tile = [&](int z, int a) -> float * {
        const int st = (z - zfirst) % STAGES;
        return tiles + ((size_t)st * NA + a) * TILE;
    };
    auto at = [&](const float *t, int y, int x) -> float { return t[y * BW + x]; };
    // thread 0: stage plane z (TMA for planes inside the grid, a bare arrive otherwise); planes are
    // issued in order, each at most STAGES ahead of the oldest one not yet waited for, so every
    // stage has at most one copy outstanding
    int last_issued = zfirst - 1;
    auto issue = [&](int z) {
        last_issued = z;
        unsigned long long *bar = &bars[(z - zfirst) % STAGES];
        if (z >= 0 && z < nz && z <= zlast) {
            mbar_expect_tx(bar, stage_bytes);
            for (int a = 0; a < NA; a++) tma_load_3d(tile(z, a), &maps.m[a], x0 - 4, y0 - 2, z, bar);
        } else {
            mbar_arrive(bar);
        }
    };
    // all threads: wait until plane z is staged; the decision to give up is CTA-uniform.
    // next_wait: the oldest plane whose copy has not been waited for
    int next_wait = zfirst;
    auto wait_plane = [&](int z) -> bool {
        const unsigned parity = (unsigned)(((z - zfirst) / STAGES) & 1);
        bool ok = mbar_wait(&bars[(z - zfirst) % STAGES], parity);
        ok = !__syncthreads_or(!ok);
        if (ok) next_wait = z + 1;
        return ok;
    };

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; st++) mbar_init(&bars[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int z = zfirst; z < zfirst + STAGES; z++) issue(z);

    float q_m2 = 0.f, q_m1 = 0.f, q_0 = 0.f, q_p1 = 0.f;
    // the iterate at planes z0-2 and z0-1 (z0-1 is the first plane updated)
    bool ok = wait_plane(zfirst) && wait_plane(zfirst + 1);
    if (ok) {
        if (zfirst >= 0) q_m1 = at(tile(zfirst, A_P), sy, sx);
        if (zfirst + 1 >= 0) q_0 = at(tile(zfirst + 1, A_P), sy, sx);
    }
    for (int s = z0 - 1; ok && s <= z1; s++) {
        if (!wait_plane(s + 1)) {
            ok = false;
            break;
        }
        float *tp = tile(s, A_P);
        q_p1 = (s + 1 < nz) ? at(tile(s + 1, A_P), sy, sx) : 0.f;
        // first colour on plane s (ring 1 and interior); its x-y neighbours are of the
        // other colour, so writing the new value at once races with no reader
        if (dom && s >= 0 && s < nz && ((i + j + s) & 1) == first) {
            const float *tbx = tile(s, A_BX), *tby = tile(s, A_BY);
            float acc = 0.f;
            const float bxl = at(tbx, sy, sx), bxh = xhi ? at(tbx, sy, sx + 1) : 0.f;
            const float byl = at(tby, sy, sx), byh = yhi ? at(tby, sy + 1, sx) : 0.f;
            const float bzl = at(tile(s, A_BZ), sy, sx), bzh = (s < nz - 1) ? at(tile(s + 1, A_BZ), sy, sx) : 0.f;
            if (xlo) acc = fmaf(bxl, at(tp, sy, sx - 1), acc);
            if (xhi) acc = fmaf(bxh, at(tp, sy, sx + 1), acc);
            if (ylo) acc = fmaf(byl, at(tp, sy - 1, sx), acc);
            if (yhi) acc = fmaf(byh, at(tp, sy + 1, sx), acc);
            if (s > 0) acc = fmaf(bzl, q_m1, acc);
            if (s < nz - 1) acc = fmaf(bzh, q_p1, acc);
            q_0 = inv_diag32(bxl, bxh, byl, byh, bzl, bzh) * fmaf(-h2, at(tile(s, A_B), sy, sx), acc);
            tp[sy * BW + sx] = q_0;
        }
        __syncthreads();
        // second colour on plane s-1; plane s-1 is then final for the interior
        const int z = s - 1;
        if (inner && z >= z0 && z < z1) {
            if (((i + j + z) & 1) == second) {
                const float *tq = tile(z, A_P), *tbx = tile(z, A_BX), *tby = tile(z, A_BY);
                float acc = 0.f;
                const float bxl = at(tbx, sy, sx), bxh = xhi ? at(tbx, sy, sx + 1) : 0.f;
                const float byl = at(tby, sy, sx), byh = yhi ? at(tby, sy + 1, sx) : 0.f;
                const float bzl = at(tile(z, A_BZ), sy, sx), bzh = (z < nz - 1) ? at(tile(s, A_BZ), sy, sx) : 0.f;
                if (xlo) acc = fmaf(bxl, at(tq, sy, sx - 1), acc);
                if (xhi) acc = fmaf(bxh, at(tq, sy, sx + 1), acc);
                if (ylo) acc = fmaf(byl, at(tq, sy - 1, sx), acc);
                if (yhi) acc = fmaf(byh, at(tq, sy + 1, sx), acc);
                if (z > 0) acc = fmaf(bzl, q_m2, acc);
                if (z < nz - 1) acc = fmaf(bzh, q_0, acc);
                q_m1 = inv_diag32(bxl, bxh, byl, byh, bzl, bzh) * fmaf(-h2, at(tile(z, A_B), sy, sx), acc);
            }
            p_new[(size_t)z * sxy + col] = q_m1;
        }
        // plane s-1's stage is free: order this CTA's shared-memory accesses before the
        // asynchronous copy that refills it with plane s-1+STAGES
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0 && s - 1 + STAGES <= zlast) issue(s - 1 + STAGES);
        q_m2 = q_m1;
        q_m1 = q_0;
        q_0 = q_p1;
    }
    // every copy issued is for a plane <= zlast, and every such plane was waited on,
    // so on success no copy is in flight here
    if (!ok && threadIdx.x == 0) {
        dscal[S_ERR] = 1.0;
        // drain: wait once more (bounded) for each plane issued and not yet waited for, on the
        // phase its copy completes, so that no copy is left writing into this CTA's shared memory
        // unless it is still not delivered after that second bounded wait
        for (int z = next_wait; z <= last_issued; z++)
            mbar_wait(&bars[(z - zfirst) % STAGES], (unsigned)(((z - zfirst) / STAGES) & 1));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_map_mutex;
// A map encodes only an address, the dimensions and the strides, so a cached map stays valid
// for any buffer later allocated at the same address with the same dimensions.
std::map<std::tuple<const void *, int, int, int>, CUtensorMap> g_maps;

cudaError_t get_encode()
{
    if (g_encode) return cudaSuccess;
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return cudaSuccess;
}

cudaError_t map_of(const float *base, int nx, int ny, int nz, CUtensorMap *out)
{
    std::lock_guard<std::mutex> lock(g_map_mutex);
    const auto key = std::make_tuple((const void *)base, nx, ny, nz);
    auto it = g_maps.find(key);
    if (it != g_maps.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    CUtensorMap m;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float), (cuuint64_t)nx * ny * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)BW, (cuuint32_t)BH, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = g_encode(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)base, dims, strides, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    g_maps[key] = m;
    *out = m;
    return cudaSuccess;
}

}  // namespace

bool tma_sweep_supported(Dims d)
{
    // TMA strides must be multiples of 16 bytes (nx % 4 == 0 for FP32) and a level needs a full tile
    return d.nx % 4 == 0 && d.nx >= TX && d.ny >= TY && d.nz >= 8;
}

cudaError_t launch_rb_sweep_tma_zc(Dims d, float h2, const LevelArrays<float> &L, const float *b, const float *p_old,
                                   float *p_new, int first, double *dscal, cudaStream_t s, int zc_force)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_rb_sweep_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    Maps maps;
    const float *src[NA] = {p_old, L.bx, L.by, L.bz, b};
    for (int a = 0; a < NA; a++) {
        cudaError_t e = map_of(src[a], d.nx, d.ny, d.nz, &maps.m[a]);
        if (e != cudaSuccess) return e;
    }
    const int tx = (d.nx + TX - 1) / TX, ty = (d.ny + TY - 1) / TY;
    // z-chunk: balance whole waves of resident CTAs (3 per SM on 152 SMs) against the two
    // extra planes each chunk recomputes
    const int wave = MG_TMA_CTAS_PER_SM * 152;
    int zc = d.nz;
    double best = 1e300;
    for (int cand : {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 1024}) {
        if (cand > d.nz && cand != 8) continue;
        const int c = cand > d.nz ? d.nz : cand;
        const long ctas = (long)tx * ty * ((d.nz + c - 1) / c);
        const double t = (double)((ctas + wave - 1) / wave) * (c + 3);
        if (t < best) {
            best = t;
            zc = c;
        }
    }
    if (zc_force > 0) zc = zc_force < d.nz ? zc_force : d.nz;
    const dim3 grid((unsigned)tx, (unsigned)ty, (unsigned)((d.nz + zc - 1) / zc));
    note_kernel_launch();
    k_rb_sweep_tma<<<grid, THREADS, SMEM_BYTES, s>>>(maps, d.nx, d.ny, d.nz, zc, h2, p_new, first, dscal);
    return cudaGetLastError();
}

cudaError_t launch_rb_sweep_tma(Dims d, float h2, const LevelArrays<float> &L, const float *b, const float *p_old,
                                float *p_new, int first, double *dscal, cudaStream_t s)
{
    return launch_rb_sweep_tma_zc(d, h2, L, b, p_old, p_new, first, dscal, s, 0);
}

}  // namespace mg
