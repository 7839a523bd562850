// mg_api.cu -- C ABI of the GB300 variable-density pressure projection (host side).
//
// Owns the multigrid hierarchy (one mg_ctx per set of face coefficients), drives
// the V-cycles on the caller's stream, and computes the dense minimum-norm inverse
// of the coarsest grid's operator on the host in FP64 (one Cholesky
// factorisation per connected component of a rank-one-shifted operator).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <string>
#include <type_traits>
#include <vector>

#include "mg_internal.cuh"

using mg::Dims;
using mg::LevelArrays;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail(e_ == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                          \
    } while (0)

#define CKS(expr)              \
    do {                       \
        int s_ = (expr);       \
        if (s_ != MG_OK) return s_; \
    } while (0)

}  // namespace

namespace mg {
void set_last_error(const char *msg) { g_err = msg; }
}  // namespace mg

struct mg_ctx {
    mg_grid g{};
    mg_opts o{};
    cudaStream_t s = nullptr;
    int nlev = 0;
    std::vector<Dims> dims;
    std::vector<double> hs;
    std::vector<LevelArrays<double>> L64;
    std::vector<LevelArrays<float>> L32;
    std::vector<double *> palt64;  // second iterate buffer per level for fused sweeps (null if unused)
    std::vector<float *> palt32;
    // conjugate-gradient vectors (krylov = 1): FP64 r, d, q; z, z_old (FP64 cycles) or a
    // second FP32 cycle output (mixed cycles)
    double *kr = nullptr, *kd = nullptr, *kq = nullptr, *kz = nullptr, *kzo = nullptr;
    // CG operator on the finest grid: h^-2 beta in bx/by/bz and h^-2 sum(beta) in dinv
    LevelArrays<double> kop;
    float *ke_alt = nullptr;
    // layout of the finest FP32 iterate / right-hand side (L32[0].p, L32[0].b, ke_alt): colour-split
    // for the per-colour smoother in mixed precision, natural otherwise
    mg::Split split0;
    // fractional face areas (mg_set_face_areas): the open fractions, and 1/rho on the faces as given
    // to mg_setup / mg_update (the operator then uses area * 1/rho); the body velocity on the faces
    // (mg_set_body_velocity)
    bool has_area = false, has_vb = false;
    LevelArrays<double> karea, kbeta, kvb;
    // the time step's scratch (mg_rk2_step): face coefficients of the two stages, u~, u*, phi*
    LevelArrays<double> rk_b1, rk_b2, rk_ut, rk_us, rk_r;
    double *rk_phis = nullptr;
    double *rk_work = nullptr;  // the momentum terms' per-cell fluxes and stresses
    float *urow0 = nullptr;  // uniform-row values of the finest FP32 level (with split0)
    // banded-row records of the finest FP32 level (with split0 and nx % 8 == 0), the two row
    // counts of the last hierarchy build, and whether its sweeps use the records (more banded
    // rows than uniform ones: a stretched grid)
    float4 *arow0 = nullptr;
    unsigned *rowcnt = nullptr;
    // the finest FP32 face arrays in the colour-split layout (with split0 and nx % 8 == 0), read
    // by the colour passes on rows without a record
    LevelArrays<float> sf0;
    bool banded = false;
    // connected regions of the live fine cells: their number; for more than one, each live cell's
    // region number (cc_label, the union-find labels otherwise), the cells per region (device
    // cc_cnt, host hcnt) and the per-region sums of the current solve (cc_sum, host hsum)
    int ncomp = 1, ncomp_raw = 0;
    int *cc_label = nullptr, *cc_roots = nullptr;
    uint8_t *open_bits = nullptr;  // open low faces of each fine cell at the last labelling
    unsigned *cc_ctr = nullptr;
    unsigned *pnz = nullptr;  // the zero test of a solve's initial guess
    double *cc_sum = nullptr, *cc_cnt = nullptr, *cc_part = nullptr;
    std::vector<double> hcnt, hsum;
    bool incompat = false;      // the current solve's rhs failed the compatibility test
    double incompat_mean = 0.0, incompat_rms = 0.0;
    double *b0 = nullptr;       // compatible fine rhs of the current solve
    double *rhs_tmp = nullptr;  // projection / adjoint right-hand side
    double *qbuf = nullptr;     // adjoint solution when the caller passes none
    double *M = nullptr;        // coarsest dense inverse (device, ncoarse^2)
    int ncoarse = 0;
    double *partials = nullptr; // reduction partials
    double *dscal = nullptr;    // device scalars (mg::Scal)
    double *hscal = nullptr;    // pinned host mirror of dscal
    // pinned staging of the coarsest grid's inverse: its three face arrays (3 ncoarse), the
    // inverse (ncoarse^2), then the two row counters of the finest uniform / banded rows
    double *hcoarse = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t ev_h = nullptr;  // the coarsest faces and the scalars reached the host
    // the coarse-grid correction of one V-cycle (everything below the finest level) as a
    // CUDA graph per precision, captured on first use on a private stream
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t coarse_graph[2] = {nullptr, nullptr};  // [0] FP64, [1] FP32
    unsigned long long coarse_graph_kernels[2] = {0, 0};   // kernel nodes per graph (launch counter)
    bool capturing = false;
    float ms_setup = 0.f;
    double nlive = 0.0;
    std::vector<void *> allocs;
    // profiling (opts.profile): event pairs recorded around finest-grid kernels
    std::vector<cudaEvent_t> pev;
    std::vector<int> pgroup;
    size_t pused = 0;

    template <typename T>
    int alloc(T **p, size_t n)
    {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, n * sizeof(T) + 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(MG_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
        }
        allocs.push_back(q);
        *p = (T *)q;
        return MG_OK;
    }
    ~mg_ctx()
    {
        for (void *q : allocs) cudaFree(q);
        if (hscal) cudaFreeHost(hscal);
        if (hcoarse) cudaFreeHost(hcoarse);
        if (ev_h) cudaEventDestroy(ev_h);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        for (cudaEvent_t e : pev) cudaEventDestroy(e);
        for (cudaGraphExec_t g : coarse_graph)
            if (g) cudaGraphExecDestroy(g);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

namespace {

// every device array starts on a 16-byte boundary (the kernels move aligned pairs); null passes
bool aligned16(std::initializer_list<const void *> ptrs)
{
    for (const void *q : ptrs)
        if (reinterpret_cast<uintptr_t>(q) % 16 != 0) return false;
    return true;
}

// most disconnected fluid regions a context handles (per-region sums and counts: 1 MB)
constexpr int kMaxRegions = 1 << 16;

bool forces_ok(const mg_forces *f)
{
    return f && std::isfinite(f->g) && std::isfinite(f->inv_re) && f->inv_re >= 0.0 && std::isfinite(f->mu_air) &&
           f->mu_air >= 0.0 && std::isfinite(f->mu_water) && f->mu_water >= 0.0;
}

bool grid_ok(const mg_grid *g)
{
    return g && g->nx >= 1 && g->ny >= 1 && g->nz >= 1 && g->h > 0.0 && std::isfinite(g->h) &&
           (double)g->nx * g->ny * g->nz < 2147483647.0;
}

// ---------------------------------------------------------------------------
// Coarsest-grid dense inverse (host, FP64).  A is assembled face by face; for
// each connected component of >= 2 cells the Moore-Penrose inverse is formed
// from one Cholesky factorisation of the shifted matrix -A + (a/m) 1 1^T (see
// below); isolated cells get zero rows and columns.
// ---------------------------------------------------------------------------
// dot product with four partial sums (lets the compiler keep several FMA chains in flight)
inline double dot4(const double *a, const double *b, int n)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int q = 0;
    for (; q + 4 <= n; q += 4) {
        s0 += a[q] * b[q];
        s1 += a[q + 1] * b[q + 1];
        s2 += a[q + 2] * b[q + 2];
        s3 += a[q + 3] * b[q + 3];
    }
    for (; q < n; q++) s0 += a[q] * b[q];
    return (s0 + s1) + (s2 + s3);
}

int coarse_inverse(int nx, int ny, int nz, double h, const double *bx, const double *by, const double *bz, double *M)
{
    const int n = nx * ny * nz;
    const double ih2 = 1.0 / (h * h);
    std::vector<double> A((size_t)n * n, 0.0);
    auto couple = [&](int a, int c, double beta) {
        if (beta <= 0.0) return;
        const double v = beta * ih2;
        A[(size_t)a * n + a] -= v;
        A[(size_t)c * n + c] -= v;
        A[(size_t)a * n + c] += v;
        A[(size_t)c * n + a] += v;
    };
    auto id = [&](int i, int j, int k) { return (k * ny + j) * nx + i; };
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const int c = id(i, j, k);
                if (i > 0) couple(id(i - 1, j, k), c, bx[c]);
                if (j > 0) couple(id(i, j - 1, k), c, by[c]);
                if (k > 0) couple(id(i, j, k - 1), c, bz[c]);
            }
    // components (union of cells joined by a nonzero off-diagonal)
    std::vector<int> comp(n, -1);
    std::vector<std::vector<int>> members;
    for (int s0 = 0; s0 < n; s0++) {
        if (comp[s0] >= 0) continue;
        const int cid = (int)members.size();
        members.emplace_back();
        std::vector<int> stack{s0};
        comp[s0] = cid;
        while (!stack.empty()) {
            const int a = stack.back();
            stack.pop_back();
            members[cid].push_back(a);
            for (int b = 0; b < n; b++)
                if (b != a && A[(size_t)a * n + b] != 0.0 && comp[b] < 0) {
                    comp[b] = cid;
                    stack.push_back(b);
                }
        }
    }
    std::fill(M, M + (size_t)n * n, 0.0);
    for (auto &mem : members) {
        const int m = (int)mem.size();
        if (m < 2) continue;
        // L = -A on the component (positive semi-definite, null vector 1).  With
        // J = 1 1^T and a = trace(L)/m (inside L's spectrum), L + (a/m) J is
        // positive definite and its inverse is L^+ + J/(a m): no cancellation.
        std::vector<double> S((size_t)m * m);
        double tr = 0.0;
        for (int q = 0; q < m; q++) tr += -A[(size_t)mem[q] * n + mem[q]];
        const double a = tr / m, shift = a / m;
        for (int x = 0; x < m; x++)
            for (int y = 0; y < m; y++) S[(size_t)x * m + y] = -A[(size_t)mem[x] * n + mem[y]] + shift;
        // Cholesky S = C C^T (C lower, in place), left-looking by 32-column panels: the panel's
        // diagonal block serially, then its rows below in parallel (one parallel region per panel)
        const int PB = 32;
        int bad = 0;
        for (int j0 = 0; j0 < m && !bad; j0 += PB) {
            const int j1 = std::min(j0 + PB, m);
            for (int j = j0; j < j1 && !bad; j++) {
                double *rj = &S[(size_t)j * m];
                const double dd = rj[j] - dot4(rj, rj, j);
                if (!(dd > 0.0)) {
                    bad = 1;
                    break;
                }
                rj[j] = std::sqrt(dd);
                for (int i = j + 1; i < j1; i++) {
                    double *ri = &S[(size_t)i * m];
                    ri[j] = (ri[j] - dot4(ri, rj, j)) / rj[j];
                }
            }
            if (bad) break;
#pragma omp parallel for schedule(static) if (m - j1 > 64)
            for (int i = j1; i < m; i++) {
                double *ri = &S[(size_t)i * m];
                for (int j = j0; j < j1; j++) {
                    const double *rj = &S[(size_t)j * m];
                    ri[j] = (ri[j] - dot4(ri, rj, j)) / rj[j];
                }
            }
        }
        if (bad) return fail(MG_ERR_ARG, "coarsest-grid operator is not semi-definite");
        // W = C^-1 (lower), stored by columns as rows of WT (upper): column j solves C w = e_j
        std::vector<double> WT((size_t)m * m, 0.0);
#pragma omp parallel for schedule(dynamic, 4) if (m > 128)
        for (int j = 0; j < m; j++) {
            double *w = &WT[(size_t)j * m];
            for (int i = j; i < m; i++) {
                const double *ci = &S[(size_t)i * m];
                w[i] = ((i == j ? 1.0 : 0.0) - dot4(ci + j, w + j, i - j)) / ci[i];
            }
        }
        // X = S^-1 = W^T W: X[x][y] = sum_{q >= max(x,y)} WT[x][q] WT[y][q]
        std::vector<double> X((size_t)m * m);
#pragma omp parallel for schedule(dynamic, 4) if (m > 128)
        for (int x = 0; x < m; x++) {
            const double *wx = &WT[(size_t)x * m];
            for (int y = 0; y <= x; y++) {
                const double v = dot4(wx + x, &WT[(size_t)y * m] + x, m - x);
                X[(size_t)x * m + y] = v;
                X[(size_t)y * m + x] = v;
            }
        }
        // A^+ = -L^+ = -(X - J/(a m))
        const double jc = 1.0 / (a * m);
        for (int x = 0; x < m; x++)
            for (int y2 = 0; y2 < m; y2++) M[(size_t)mem[x] * n + mem[y2]] = -(X[(size_t)x * m + y2] - jc);
    }
    return MG_OK;
}

template <typename T>
int level_alloc(mg_ctx *c, LevelArrays<T> &L, size_t n, bool with_bp)
{
    CKS(c->alloc(&L.bx, n));
    CKS(c->alloc(&L.by, n));
    CKS(c->alloc(&L.bz, n));
    CKS(c->alloc(&L.dinv, n));
    if (with_bp) {
        CKS(c->alloc(&L.b, n));
        CKS(c->alloc(&L.p, n));
    }
    return MG_OK;
}

// Profiling: an event pair around one finest-grid kernel launch (no-op unless enabled).
struct ProfScope {
    mg_ctx *c;
    int slot = -1;
    ProfScope(mg_ctx *c_, int group, bool on) : c(c_)
    {
        if (!on || !c->o.profile || c->capturing || c->pused + 2 > c->pev.size()) return;
        slot = (int)c->pused;
        c->pused += 2;
        c->pgroup[slot / 2] = group;
        cudaEventRecord(c->pev[slot], c->s);
    }
    ~ProfScope()
    {
        if (slot >= 0) cudaEventRecord(c->pev[slot + 1], c->s);
    }
};

// ---------------------------------------------------------------------------
// V-cycle on level l (p updated in place): pre-smooth nu1 x (red, black),
// residual + restriction, coarse correction (recursion or exact solve),
// prolongation, post-smooth nu2 x (black, red).
// ---------------------------------------------------------------------------
template <typename T>
T *palt_of(mg_ctx *c, int l);
template <>
double *palt_of<double>(mg_ctx *c, int l) { return c->palt64.empty() ? nullptr : c->palt64[l]; }
template <>
float *palt_of<float>(mg_ctx *c, int l) { return c->palt32.empty() ? nullptr : c->palt32[l]; }

// fused sweeps pay off on levels with at least one full 32 x 8 tile and 8 planes
bool fused_level(const Dims &d) { return d.nx >= 32 && d.ny >= 8 && d.nz >= 8; }

template <typename T>
bool use_fused(const mg_ctx *c, int l)
{
    if (!fused_level(c->dims[l]) || l == c->nlev - 1) return false;
    if (c->o.smoother == 2) return true;
    if (c->o.smoother == 3) return sizeof(T) == 4;
    return false;  // auto and 1: one pass per colour (the measured fastest on GB300)
}

// FP32 levels in auto mode sweep with the TMA-staged kernel where its layout allows
template <typename T>
bool tma_level(const mg_ctx *c, int l)
{
    return sizeof(T) == 4 && c->o.smoother == 3 && mg::tma_sweep_supported(c->dims[l]);
}
inline cudaError_t launch_sweep_tma(Dims d, float h2, const LevelArrays<float> &L, const float *b, const float *pold,
                                    float *pnew, int first, double *dscal, cudaStream_t s)
{
    return mg::launch_rb_sweep_tma(d, h2, L, b, pold, pnew, first, dscal, s);
}
inline cudaError_t launch_sweep_tma(Dims, double, const LevelArrays<double> &, const double *, const double *,
                                    double *, int, double *, cudaStream_t)
{
    return cudaErrorNotSupported;  // FP64 levels never take this path
}

template <typename T>
int coarse_correction_graph(mg_ctx *c, const std::vector<LevelArrays<T>> &L);

// First level of the coarse tail in precision T: the largest level below the finest, above the
// coarsest, whose six fields (p, b, three face arrays, dinv) fit in an SM's L1; -1 if none.
constexpr size_t kTailBytes = 200 * 1024;
template <typename T>
int tail_start(const mg_ctx *c)
{
    if (!c->o.coarse_tail) return -1;
    for (int l = 1; l + 1 < c->nlev; l++)
        if (c->dims[l].n() * 6 * sizeof(T) <= kTailBytes && c->nlev - l <= mg::kTailMaxLevels) return l;
    return -1;
}

// zero: p is taken as zero on entry (a cycle from a zero guess): the coarsest solve overwrites it,
// the coarse tail zeroes it in its kernel, and the per-colour passes start with a pass that reads
// no iterate, so no separate clearing pass is needed (the fused sweeps and nu1 = 0 clear it first)
template <typename T>
int vcycle(mg_ctx *c, const std::vector<LevelArrays<T>> &L, int l, const T *b, T *p, bool zero = false)
{
    cudaStream_t s = c->s;
    const Dims d = c->dims[l];
    if (l == c->nlev - 1) {
        CK(mg::launch_coarse_solve<T>(c->ncoarse, c->M, b, p, s));
        return MG_OK;
    }
    if (l == tail_start<T>(c)) {  // this level and all below: one CTA, two launches
        mg::TailArgs<T> a{};
        a.nlev = c->nlev - l;
        a.nu1 = c->o.nu1;
        a.nu2 = c->o.nu2;
        a.zero0 = zero ? 1 : 0;
        for (int q = 0; q < a.nlev; q++) {
            const int lv = l + q;
            const Dims dl = c->dims[lv];
            a.lev[q] = mg::TailLevel<T>{dl.nx, dl.ny, dl.nz, (T)(c->hs[lv] * c->hs[lv]),
                                        (T)(1.0 / (c->hs[lv] * c->hs[lv])), L[lv],
                                        mg::make_fastdiv((unsigned)(dl.nx + 1) / 2), mg::make_fastdiv((unsigned)dl.ny),
                                        mg::make_fastdiv((unsigned)std::max(dl.nx / 2, 1)),
                                        mg::make_fastdiv((unsigned)std::max(dl.ny / 2, 1))};
        }
        a.lev[0].L.b = const_cast<T *>(b);
        a.lev[0].L.p = p;
        const LevelArrays<T> &Lc = L[c->nlev - 1];
        CK(mg::launch_tail_down<T>(a, s));
        CK(mg::launch_coarse_solve<T>(c->ncoarse, c->M, Lc.b, Lc.p, s));
        CK(mg::launch_tail_up<T>(a, s));
        return MG_OK;
    }
    const T h2 = (T)(c->hs[l] * c->hs[l]);
    const T ih2 = (T)(1.0 / (c->hs[l] * c->hs[l]));
    const bool fine = (l == 0);
    const bool fused = use_fused<T>(c, l) && palt_of<T>(c, l) != nullptr;
    const mg::Split sp = (sizeof(T) == 4 && l == 0) ? c->split0 : mg::Split{};
    const float *urow = (sizeof(T) == 4 && l == 0) ? c->urow0 : nullptr;
    const float4 *arow = (sizeof(T) == 4 && l == 0 && c->banded) ? c->arow0 : nullptr;
    T *cur = p, *alt = palt_of<T>(c, l);
    // plane order of the finest colour passes (pass_order = 1): each group of passes alternates
    // descending, ascending, ... so that every pass starts on the planes its predecessor (or the
    // prolongation, ascending) touched last, which are still in L2; the restriction that follows
    // the last (ascending) pre-smoothing pass runs descending
    const bool alternate = c->o.pass_order == 1 && sp.half;
    int npass = 0;
    // the first pass reads no iterate when p starts at zero; otherwise clear p first
    bool zpass = zero && !fused && c->o.nu1 >= 1;
    if (zero && !zpass) CK(cudaMemsetAsync(p, 0, d.n() * sizeof(T), s));
    // one red-black sweep, `first` colour first
    auto sweep = [&](int first) -> int {
        ProfScope ps(c, MG_PROF_SMOOTH, fine);
        if (fused) {
            if (tma_level<T>(c, l))
                CK(launch_sweep_tma(d, h2, L[l], b, cur, alt, first, c->dscal, s));
            else
                CK(mg::launch_rb_sweep<T>(d, h2, L[l], b, cur, alt, first, s));
            std::swap(cur, alt);
        } else if (sp.half) {
            if constexpr (std::is_same<T, float>::value) {
                const int r0 = alternate ? (npass + 1) & 1 : 0;
                CK(mg::launch_smooth_split(d, h2, L[l], b, cur, first, s, urow, arow, r0, zpass, &c->sf0));
                CK(mg::launch_smooth_split(d, h2, L[l], b, cur, first ^ 1, s, urow, arow, r0 ^ (alternate ? 1 : 0),
                                           false, &c->sf0));
                npass += 2;
            }
        } else {
            CK(mg::launch_smooth<T>(d, h2, L[l], b, cur, first, s, 0, -1, zpass));
            CK(mg::launch_smooth<T>(d, h2, L[l], b, cur, first ^ 1, s));
        }
        zpass = false;
        return MG_OK;
    };
    for (int it = 0; it < c->o.nu1; it++) CKS(sweep(0));
    const LevelArrays<T> &C = L[l + 1];
    {
        ProfScope ps(c, MG_PROF_RESTRICT, fine);
        // descending after an ascending last pass (an even number of passes, the last ascending)
        const int rrev = alternate && npass > 0 && (npass & 1) == 0 ? 1 : 0;
        CK(mg::launch_resid_restrict<T>(d, ih2, L[l], b, cur, C.b, s, sp, urow, rrev));
    }
    npass = 0;
    {
        ProfScope ps(c, MG_PROF_COARSE, fine);
        if (fine && c->o.coarse_graph && !c->capturing)
            CKS(coarse_correction_graph<T>(c, L));
        else
            CKS(vcycle<T>(c, L, l + 1, C.b, C.p, true));
    }
    {
        ProfScope ps(c, MG_PROF_PROLONG, fine);
        CK(mg::launch_prolong<T>(d, C.p, L[l].dinv, cur, s, sp, urow));
    }
    for (int it = 0; it < c->o.nu2; it++) CKS(sweep(1));
    if (cur != p) CK(cudaMemcpyAsync(p, cur, d.n() * sizeof(T), cudaMemcpyDeviceToDevice, s));
    return MG_OK;
}

// The coarse-grid correction of a V-cycle on the finest level: zero the level-1
// correction, V-cycle levels 1..coarsest.  Its buffers are the context's own, so one
// captured graph per precision serves every call; it is launched on the caller's stream.
template <typename T>
int coarse_correction_graph(mg_ctx *c, const std::vector<LevelArrays<T>> &L)
{
    const int slot = sizeof(T) == 4 ? 1 : 0;
    if (!c->coarse_graph[slot]) {
        if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        cudaStream_t user = c->s;
        c->s = c->cap_stream;
        c->capturing = true;
        cudaGraph_t g = nullptr;
        int st = MG_OK;
        const unsigned long long k0 = mg::launch_count();
        cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = [&]() -> int {
                CKS(vcycle<T>(c, L, 1, L[1].b, L[1].p, true));
                return MG_OK;
            }();
            e = cudaStreamEndCapture(c->cap_stream, &g);
        }
        c->s = user;
        c->capturing = false;
        c->coarse_graph_kernels[slot] = mg::launch_count() - k0;
        if (st != MG_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return fail(MG_ERR_CUDA, "coarse-grid graph capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->coarse_graph[slot], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->coarse_graph[slot] = nullptr;
            return fail(MG_ERR_CUDA, "coarse-grid graph instantiation failed: %s", cudaGetErrorString(e));
        }
    }
    CK(cudaGraphLaunch(c->coarse_graph[slot], c->s));
    for (unsigned long long k = 0; k < c->coarse_graph_kernels[slot]; k++) mg::note_kernel_launch();
    return MG_OK;
}

// read the device scalars into the pinned mirror (one stream sync); report a kernel whose
// bounded wait expired
int check_scalars(mg_ctx *c);
int read_scalars(mg_ctx *c)
{
    CK(cudaMemcpyAsync(c->hscal, c->dscal, mg::S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    return check_scalars(c);
}

// the scalars just read: report a kernel whose bounded wait expired (and clear its flag)
int check_scalars(mg_ctx *c)
{
    if (c->hscal[mg::S_ERR] != 0.0) {
        CK(cudaMemsetAsync(c->dscal + mg::S_ERR, 0, sizeof(double), c->s));
        return fail(MG_ERR_CUDA, "a pipelined smoothing kernel's bounded wait expired (data not delivered)");
    }
    return MG_OK;
}

void stats_begin(mg_stats *st)
{
    if (!st) return;
    st->cycles = 0;
    st->rel_resid = 0.0;
    st->rhs_norm = 0.0;
    st->rhs_mean_removed = 0.0;
    for (double &v : st->resid_hist) v = 0.0;
}

// The compatible right-hand side b0 of a solve (Eq. neumann with Eq. pois: one constant per
// connected fluid region spans A's null space, so b is solvable only with zero sum on each): the
// rhs minus its mean on each region, 0 on dead cells; dscal gets S_SUM_B (the sum over the live
// cells) and S_NB2 (||b0||^2).  The region sums go to the host with the next read_scalars.
int prepare_rhs(mg_ctx *c, const double *rhs)
{
    const Dims d = c->dims[0];
    if (c->ncomp > 1) {
        CK(mg::launch_comp_center(d.n(), rhs, c->cc_label, c->ncomp, c->cc_sum, c->cc_cnt, c->b0, c->partials,
                                  c->dscal, mg::S_NB2, mg::S_SUM_B, c->s, c->cc_part));
        c->hsum.resize(c->ncomp);
        CK(cudaMemcpyAsync(c->hsum.data(), c->cc_sum, c->ncomp * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    } else {
        CK(mg::launch_rhs_prepare(d, rhs, c->L64[0].dinv, c->b0, c->partials, c->dscal, c->s));
    }
    return MG_OK;
}

// After the first read_scalars of a solve: the rhs is incompatible when the mean it had on some
// region exceeds kIncompatible times its RMS over the live cells (both before the removal):
// sum b^2 = ||b0||^2 + sum over regions of (cells x mean^2).
constexpr double kIncompatible = 1e-8;
void check_compatible(mg_ctx *c)
{
    c->incompat = false;
    const double n = c->nlive, nb2 = c->hscal[mg::S_NB2];
    if (!(n > 0.0) || !std::isfinite(nb2)) return;
    double worst = 0.0, sq = nb2;
    if (c->ncomp > 1) {
        for (int m = 0; m < c->ncomp; m++) {
            const double mean = c->hsum[m] / c->hcnt[m];
            sq += c->hcnt[m] * mean * mean;
            worst = std::max(worst, std::fabs(mean));
        }
    } else {
        const double mean = c->hscal[mg::S_SUM_B] / n;
        sq += n * mean * mean;
        worst = std::fabs(mean);
    }
    const double rms = std::sqrt(sq / n);
    c->incompat = worst > kIncompatible * rms;
    c->incompat_mean = worst;
    c->incompat_rms = rms;
}

// a solve that converged on an incompatible rhs reports it (p is the solution for the rhs with
// its region means removed)
int final_status(mg_ctx *c, int status)
{
    if (status == MG_OK && c->incompat)
        return fail(MG_ERR_INCOMPATIBLE,
                    "right-hand side incompatible with the Neumann problem: mean %.3e on a fluid region against an "
                    "RMS of %.3e; the mean of each region was removed and the solve converged",
                    c->incompat_mean, c->incompat_rms);
    return status;
}

// p -= its mean over each fluid region (live cells), dead cells 0; with one region the mean is
// dscal[S_SUM_P] / nlive from the last residual pass
int remove_p_mean(mg_ctx *c, double *p)
{
    const Dims d = c->dims[0];
    if (c->ncomp > 1)
        CK(mg::launch_comp_center(d.n(), p, c->cc_label, c->ncomp, c->cc_sum, c->cc_cnt, p, c->partials, c->dscal,
                                  -1, -1, c->s, c->cc_part));
    else
        CK(mg::launch_sub_mean_p(d, c->L64[0].dinv, p, c->dscal, c->s));
    return MG_OK;
}

int solve_impl(mg_ctx *c, const double *rhs, double *p, double tol, mg_stats *st)
{
    cudaStream_t s = c->s;
    const Dims d = c->dims[0];
    const double ih2 = 1.0 / (c->hs[0] * c->hs[0]);
    const bool mixed = c->o.prec == MG_MIXED;
    stats_begin(st);
    if (st) st->ms_setup = c->ms_setup;
    CK(cudaEventRecord(c->ev0, s));
    CKS(prepare_rhs(c, rhs));
    int scale_slot = mg::S_SCALE0, next_slot = mg::S_SCALE1;
    if (mixed) {
        ProfScope ps(c, MG_PROF_RESID64, true);
        CK(mg::launch_resid_cast(d, ih2, c->L64[0], c->b0, p, c->L32[0].b, c->partials, c->dscal, -1, next_slot, s,
                                 c->split0));
    } else {
        ProfScope ps(c, MG_PROF_RESID64, true);
        CK(mg::launch_resid_norm(d, ih2, c->L64[0], c->b0, p, c->partials, c->dscal, s));
    }
    CKS(read_scalars(c));
    check_compatible(c);
    const double nb2 = c->hscal[mg::S_NB2];
    if (st) {
        st->rhs_norm = std::sqrt(nb2);
        st->rhs_mean_removed = c->nlive > 0 ? c->hscal[mg::S_SUM_B] / c->nlive : 0.0;
    }
    if (!std::isfinite(nb2)) return fail(MG_ERR_NAN, "right-hand side is not finite");
    if (nb2 == 0.0 || c->nlive == 0.0) {
        CK(cudaMemsetAsync(p, 0, d.n() * sizeof(double), s));
        CK(cudaEventRecord(c->ev1, s));
        CK(cudaEventSynchronize(c->ev1));
        if (st) cudaEventElapsedTime(&st->ms_solve, c->ev0, c->ev1);
        return final_status(c, MG_OK);
    }
    double rel = std::sqrt(c->hscal[mg::S_RR] / nb2);
    int cyc = 0, status = MG_OK;
    int nhist = 0;
    while (!(rel <= tol)) {
        if (!std::isfinite(rel)) {
            status = fail(MG_ERR_NAN, "residual norm is not finite after %d cycles", cyc);
            break;
        }
        if (cyc >= c->o.max_cycles) {
            status = fail(MG_ERR_NOT_CONVERGED, "not converged: relative residual %.3e after %d cycles (tol %.1e)",
                          rel, cyc, tol);
            break;
        }
        cyc++;
        if (mixed) {
            for (int ic = 0; ic < c->o.inner_cycles; ic++)
                CKS(vcycle<float>(c, c->L32, 0, c->L32[0].b, c->L32[0].p, ic == 0));
            CK(mg::launch_accumulate(d, c->L64[0].dinv, c->L32[0].p, p, c->dscal, scale_slot, s, c->split0));
            std::swap(scale_slot, next_slot);
            ProfScope ps(c, MG_PROF_RESID64, true);
            CK(mg::launch_resid_cast(d, ih2, c->L64[0], c->b0, p, c->L32[0].b, c->partials, c->dscal, scale_slot,
                                     next_slot, s, c->split0));
        } else {
            CKS(vcycle<double>(c, c->L64, 0, c->b0, p));
            if (cyc % c->o.check_every != 0 && cyc < c->o.max_cycles) continue;
            ProfScope ps(c, MG_PROF_RESID64, true);
            CK(mg::launch_resid_norm(d, ih2, c->L64[0], c->b0, p, c->partials, c->dscal, s));
        }
        CKS(read_scalars(c));
        rel = std::sqrt(c->hscal[mg::S_RR] / nb2);
        if (st && nhist < 256) st->resid_hist[nhist++] = rel;
    }
    // zero mean over each region's live cells (the cycle commutes with constant shifts, so once
    // suffices)
    CKS(remove_p_mean(c, p));
    CK(cudaEventRecord(c->ev1, s));
    CK(cudaEventSynchronize(c->ev1));
    if (st) {
        st->cycles = cyc;
        st->rel_resid = rel;
        cudaEventElapsedTime(&st->ms_solve, c->ev0, c->ev1);
    }
    return final_status(c, status);
}

int compute_hierarchy(mg_ctx *c, const double *const face_coeffs[3])
{
    cudaStream_t s = c->s;
    const Dims dc = c->dims.back();
    const size_t n0 = c->dims[0].n();
    CK(cudaMemsetAsync(c->dscal, 0, mg::S_COUNT * sizeof(double), s));
    if (c->has_area) {  // keep 1/rho; the operator's coefficient is area * 1/rho
        double *kb[3] = {c->kbeta.bx, c->kbeta.by, c->kbeta.bz};
        for (int a = 0; a < 3; a++)
            if (face_coeffs[a] != kb[a])
                CK(cudaMemcpyAsync(kb[a], face_coeffs[a], n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(mg::launch_area_coeffs(n0, c->karea, c->kbeta, c->L64[0], s));
    } else {
        CK(cudaMemcpyAsync(c->L64[0].bx, face_coeffs[0], n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(c->L64[0].by, face_coeffs[1], n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(c->L64[0].bz, face_coeffs[2], n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    for (int l = 0; l < c->nlev; l++) {
        if (l > 0)
            CK(mg::launch_restrict_coeffs(c->dims[l - 1], c->L64[l - 1].bx, c->L64[l - 1].by, c->L64[l - 1].bz,
                                          c->L64[l].bx, c->L64[l].by, c->L64[l].bz, s));
        // the finest level's CG operator (scaled coefficients and diagonal) comes out of the same pass
        const bool op = l == 0 && c->kop.dinv;
        CK(mg::launch_diag_inv<double>(c->dims[l], c->L64[l].bx, c->L64[l].by, c->L64[l].bz, c->L64[l].dinv, s,
                                       op ? &c->kop : nullptr, 1.0 / (c->hs[0] * c->hs[0]),
                                       l == 0 ? c->open_bits : nullptr, c->dscal + mg::S_TOPO));
    }
    CK(mg::launch_count_live(c->dims[0], c->L64[0].dinv, c->partials, c->dscal, s));
    // the coarsest operator and the scalars to the pinned host mirrors; the host waits for them
    // alone (event), while the FP32 copies queued next still run: the host's inverse of the
    // coarsest operator overlaps them
    const int nc = c->ncoarse;
    double *hcb = c->hcoarse, *hM = c->hcoarse + 3 * (size_t)nc;
    unsigned *hrow = reinterpret_cast<unsigned *>(hM + (size_t)nc * nc);
    const double *src[3] = {c->L64.back().bx, c->L64.back().by, c->L64.back().bz};
    for (int a = 0; a < 3; a++)
        CK(cudaMemcpyAsync(hcb + (size_t)a * nc, src[a], nc * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->hscal, c->dscal, mg::S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(c->ev_h, s));
    if (c->o.prec == MG_MIXED) {
        // narrowed faces and 1/sum of them (the value the FP32 smoothers form on the fly); the
        // finest level's faces also in the colour-split layout
        for (int l = 0; l < c->nlev; l++)
            CK(mg::launch_level_f32(c->dims[l], c->L64[l], c->L32[l], s, l == 0 ? &c->sf0 : nullptr, c->split0));
        if (c->rowcnt) CK(cudaMemsetAsync(c->rowcnt, 0, 2 * sizeof(unsigned), s));
        if (c->urow0)
            CK(mg::launch_uniform_rows(c->dims[0], c->L32[0].bx, c->L32[0].by, c->L32[0].bz, c->urow0, s, c->arow0,
                                       c->rowcnt));
        if (c->rowcnt) CK(cudaMemcpyAsync(hrow, c->rowcnt, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaEventSynchronize(c->ev_h));
    CKS(check_scalars(c));
    c->nlive = c->hscal[mg::S_NLIVE];
    // connected regions of the live fine cells, labelled again where the open faces changed
    // (first build included: the stored bits start as 0xff)
    unsigned cc[2] = {(unsigned)c->ncomp, 0};
    if (c->hscal[mg::S_TOPO] != 0.0) {
        CK(mg::launch_components(c->dims[0], c->L64[0].dinv, c->L64[0].bx, c->L64[0].by, c->L64[0].bz, c->cc_label,
                                 c->cc_ctr, s));
        CK(cudaMemcpyAsync(cc, c->cc_ctr, sizeof cc, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } else {
        cc[0] = (unsigned)(c->ncomp_raw);
    }
    if (cc[1]) return fail(MG_ERR_CUDA, "fluid-region labelling: a bounded union-find loop gave up");
    if (cc[0] > (unsigned)kMaxRegions)
        return fail(MG_ERR_ARG, "the fluid forms %u disconnected regions (at most %d supported)", cc[0], kMaxRegions);
    c->ncomp = (int)std::max(cc[0], 1u);
    const bool relabel = c->hscal[mg::S_TOPO] != 0.0;
    c->ncomp_raw = (int)cc[0];
    std::vector<int> roots;
    if (cc[0] > 1 && relabel) {  // number the regions by their smallest cell index; cells per region
        CK(mg::launch_component_roots(n0, c->cc_label, c->cc_roots, c->cc_ctr, (unsigned)kMaxRegions, s));
        roots.resize(cc[0]);
        CK(cudaMemcpyAsync(roots.data(), c->cc_roots, cc[0] * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::sort(roots.begin(), roots.end());
        CK(cudaMemcpyAsync(c->cc_roots, roots.data(), cc[0] * sizeof(int), cudaMemcpyHostToDevice, s));
        CK(mg::launch_component_compact(n0, c->cc_label, c->cc_roots, c->ncomp, c->cc_cnt, c->cc_part, s));
        c->hcnt.resize(c->ncomp);
        CK(cudaMemcpyAsync(c->hcnt.data(), c->cc_cnt, c->ncomp * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    CKS(coarse_inverse(dc.nx, dc.ny, dc.nz, c->hs.back(), hcb, hcb + nc, hcb + 2 * (size_t)nc, hM));
    CK(cudaMemcpyAsync(c->M, hM, (size_t)nc * nc * sizeof(double), cudaMemcpyHostToDevice, s));
    // the pinned staging must outlive the copy; the row counters have arrived
    CK(cudaStreamSynchronize(s));
    if (c->o.prec == MG_MIXED && c->rowcnt) c->banded = hrow[1] > hrow[0];
    return MG_OK;
}

// ---------------------------------------------------------------------------
// Multigrid-preconditioned conjugate gradients, flexible (Polak-Ribiere) form:
//   r = b - A p; z = M r; d = z
//   repeat: q = A d; alpha = <r,z>/<d,q>; p += alpha d; r -= alpha q
//           z' = M r; beta = (<r,z'> - <r,z>) / <r_old,z>; d = z' + beta d
// M = inner_cycles V-cycles from a zero guess, FP64 or FP32 (on r scaled by the
// RMS of the previous residual).  Convergence is decided on the recursive r and
// confirmed with the true residual (restart from p if it is above the target).
// The target is kCgTolFactor * tol: the relative solution error of a CG iterate is
// 4 to 23 times its relative residual on the 128^3, 256^3 and 512x256x128 workloads,
// so the CG stops where the residual is 0.4 tol and the error below 10 tol.
// ---------------------------------------------------------------------------
constexpr double kCgTolFactor = 0.4;

int pcg_impl(mg_ctx *c, const double *rhs, double *p, double tol_user, mg_stats *st)
{
    const double tol = tol_user * kCgTolFactor;
    cudaStream_t s = c->s;
    const Dims d = c->dims[0];
    const size_t n = d.n();
    const double ih2 = 1.0 / (c->hs[0] * c->hs[0]);
    const bool mixed = c->o.prec == MG_MIXED;
    stats_begin(st);
    if (st) st->ms_setup = c->ms_setup;
    CK(cudaEventRecord(c->ev0, s));
    CKS(prepare_rhs(c, rhs));
    bool first_check = true;
    float *e_cur = mixed ? c->L32[0].p : nullptr, *e_old = mixed ? c->ke_alt : nullptr;
    int sc_cur = mg::S_SCALE0, sc_old = mg::S_SCALE1;
    double *z = c->kz, *zo = c->kzo;
    int it = 0, status = MG_OK, nhist = 0;
    double rel = 0.0, nb2 = 0.0;
    bool done = false, zeroed = false;
    // precondition: z = M r (FP64) or e_cur = M (r / scale) (mixed); M = V-cycles, or the inverse
    // diagonal of A (Jacobi: -h^2 dinv)
    auto precondition = [&]() -> int {
        if (c->o.precond == 1) {
            CK(mg::launch_jacobi(n, -c->hs[0] * c->hs[0], c->L64[0].dinv, c->kr, z, s));
        } else if (mixed) {
            for (int v = 0; v < c->o.inner_cycles; v++) CKS(vcycle<float>(c, c->L32, 0, c->L32[0].b, e_cur, v == 0));
        } else {
            for (int v = 0; v < c->o.inner_cycles; v++) CKS(vcycle<double>(c, c->L64, 0, c->kr, z, v == 0));
        }
        return MG_OK;
    };
    while (!done) {
        // (re)start: true residual
        {
            ProfScope ps(c, MG_PROF_RESID64, true);
            // the first residual of a solve tests p for zero (a zero guess needs no stencil)
            CK(mg::launch_pcg_resid(d, ih2, c->L64[0], c->b0, p, c->kr, mixed ? c->L32[0].b : nullptr, c->partials,
                                    c->dscal, sc_cur, s, c->split0, first_check ? c->pnz : nullptr));
        }
        CKS(read_scalars(c));
        if (first_check) check_compatible(c);
        first_check = false;
        nb2 = c->hscal[mg::S_NB2];
        if (st) {
            st->rhs_norm = std::sqrt(nb2);
            st->rhs_mean_removed = c->nlive > 0 ? c->hscal[mg::S_SUM_B] / c->nlive : 0.0;
        }
        if (!std::isfinite(nb2)) return fail(MG_ERR_NAN, "right-hand side is not finite");
        if (nb2 == 0.0 || c->nlive == 0.0) {
            CK(cudaMemsetAsync(p, 0, n * sizeof(double), s));
            rel = 0.0;
            zeroed = true;
            break;
        }
        rel = std::sqrt(c->hscal[mg::S_RR] / nb2);
        if (rel <= tol) break;
        if (!std::isfinite(rel)) {
            status = fail(MG_ERR_NAN, "residual norm is not finite after %d iterations", it);
            break;
        }
        if (it >= c->o.max_cycles) {
            status = fail(MG_ERR_NOT_CONVERGED,
                          "not converged: relative residual %.3e after %d iterations (tol %.1e, CG target %.1e)", rel,
                          it, tol_user, tol);
            break;
        }
        CKS(precondition());
        if (mixed) {
            CK(mg::launch_pcg_dots32(n, c->L32[0].b, e_cur, nullptr, c->partials, c->dscal, sc_cur, sc_cur, -1, s));
            CK(mg::launch_pcg_dir<float>(n, e_cur, c->kd, c->dscal, sc_cur, -1, 1, s, c->split0, c->partials));
        } else {
            CK(mg::launch_pcg_dots<double>(n, c->kr, z, nullptr, c->partials, c->dscal, -1, -1, s));
            CK(mg::launch_pcg_dir<double>(n, z, c->kd, c->dscal, -1, -1, 1, s, {}, c->partials));
        }
        for (;;) {
            it++;
            {
                ProfScope ps(c, MG_PROF_APPLY, true);
                CK(mg::launch_pcg_apply(d, c->kop, c->kd, c->kq, c->partials, c->dscal, s));
            }
            std::swap(e_cur, e_old);
            std::swap(sc_cur, sc_old);
            std::swap(z, zo);
            {
                ProfScope ps(c, MG_PROF_RESID64, true);
                CK(mg::launch_pcg_update(n, c->kd, c->kq, p, c->kr, mixed ? c->L32[0].b : nullptr, c->partials, c->dscal,
                                         sc_cur, mixed ? sc_old : -1, s, c->split0));
            }
            CKS(read_scalars(c));
            rel = std::sqrt(c->hscal[mg::S_RR] / nb2);
            if (st && nhist < 256) st->resid_hist[nhist++] = rel;
            if (rel <= tol || !std::isfinite(rel) || it >= c->o.max_cycles) break;
            CKS(precondition());
            ProfScope ps(c, MG_PROF_KRYLOV, true);
            if (mixed) {
                CK(mg::launch_pcg_dots32(n, c->L32[0].b, e_cur, e_old, c->partials, c->dscal, sc_cur, sc_cur, sc_old,
                                         s));
                CK(mg::launch_pcg_dir<float>(n, e_cur, c->kd, c->dscal, sc_cur, sc_old, 0, s, c->split0, c->partials));
            } else {
                CK(mg::launch_pcg_dots<double>(n, c->kr, z, zo, c->partials, c->dscal, -1, -1, s));
                CK(mg::launch_pcg_dir<double>(n, z, c->kd, c->dscal, -1, -1, 0, s, {}, c->partials));
            }
        }
        if (!std::isfinite(rel)) {
            status = fail(MG_ERR_NAN, "residual norm is not finite after %d iterations", it);
            break;
        }
        // the loop top re-checks with the true residual (and restarts if needed)
    }
    (void)done;
    if (!zeroed && (status == MG_OK || status == MG_ERR_NOT_CONVERGED)) CKS(remove_p_mean(c, p));
    CK(cudaEventRecord(c->ev1, s));
    CK(cudaEventSynchronize(c->ev1));
    if (st) {
        st->cycles = it;
        st->rel_resid = rel;
        cudaEventElapsedTime(&st->ms_solve, c->ev0, c->ev1);
    }
    return final_status(c, status);
}

int ensure(mg_ctx *c, double **p, size_t n)
{
    if (*p) return MG_OK;
    return c->alloc(p, n);
}

}  // namespace

extern "C" {

void mg_default_opts(mg_opts *o)
{
    if (!o) return;
    o->nu1 = 2;
    o->nu2 = 2;
    o->max_cycles = 100;
    o->check_every = 1;
    o->coarse_max_cells = 512;
    o->prec = MG_FP64;
    o->inner_cycles = 1;
    o->profile = 0;
    o->smoother = 0;
    o->krylov = 0;
    o->coarse_graph = 1;
    o->coarse_tail = 1;
    o->precond = 0;
    o->pass_order = 1;
}

const char *mg_last_error(void) { return g_err.c_str(); }

int mg_face_coeffs(const mg_grid *g, const double *phi, const uint8_t *solid_mask, double rho_air, double rho_water,
                   double *const beta_out[3], void *stream)
{
    g_err.clear();
    if (!grid_ok(g)) return fail(MG_ERR_ARG, "mg_face_coeffs: bad grid");
    if (!phi || !beta_out || !beta_out[0] || !beta_out[1] || !beta_out[2])
        return fail(MG_ERR_ARG, "mg_face_coeffs: null pointer");
    if (!(rho_air > 0.0) || !(rho_water > 0.0)) return fail(MG_ERR_ARG, "mg_face_coeffs: densities must be > 0");
    if (!aligned16({phi, solid_mask, beta_out[0], beta_out[1], beta_out[2]}))
        return fail(MG_ERR_ARG, "mg_face_coeffs: arrays must be 16-byte aligned");
    const Dims d{g->nx, g->ny, g->nz};
    CK(mg::launch_face_coeffs(d, phi, solid_mask, rho_air, rho_water - rho_air, beta_out[0], beta_out[1], beta_out[2],
                              (cudaStream_t)stream));
    return MG_OK;
}

int mg_setup(mg_ctx **out, const mg_grid *g, const double *const face_coeffs[3], const mg_bc *bc,
             const uint8_t *solid_mask, const mg_opts *opt, void *stream)
{
    g_err.clear();
    (void)solid_mask;
    const auto t0 = std::chrono::steady_clock::now();
    if (!out) return fail(MG_ERR_ARG, "mg_setup: out is null");
    *out = nullptr;
    if (!grid_ok(g)) return fail(MG_ERR_ARG, "mg_setup: bad grid");
    if (!face_coeffs || !face_coeffs[0] || !face_coeffs[1] || !face_coeffs[2])
        return fail(MG_ERR_ARG, "mg_setup: null face coefficient pointer");
    if (!aligned16({face_coeffs[0], face_coeffs[1], face_coeffs[2], solid_mask}))
        return fail(MG_ERR_ARG, "mg_setup: arrays must be 16-byte aligned");
    if (bc)
        for (int w = 0; w < 6; w++)
            if (bc->wall[w] != MG_BC_NEUMANN) return fail(MG_ERR_ARG, "mg_setup: only Neumann walls are supported");
    mg_opts o;
    mg_default_opts(&o);
    if (opt) o = *opt;
    if (o.nu1 < 0 || o.nu2 < 0 || o.nu1 + o.nu2 < 1 || o.max_cycles < 0 || o.check_every < 1 ||
        o.coarse_max_cells < 1 || o.coarse_max_cells > 2048 || (o.prec != MG_FP64 && o.prec != MG_MIXED) ||
        o.inner_cycles < 1 || o.profile < 0 || o.smoother < 0 || o.smoother > 3 || o.krylov < 0 || o.krylov > 1 || o.coarse_graph < 0 || o.coarse_graph > 1 ||
        o.coarse_tail < 0 || o.coarse_tail > 1 || o.precond < 0 || o.precond > 1 || o.pass_order < 0 ||
        o.pass_order > 1 ||
        (o.precond == 1 && (o.krylov != 1 || o.prec != MG_FP64)))
        return fail(MG_ERR_ARG, "mg_setup: invalid options");

    mg_ctx *c = new mg_ctx();
    c->g = *g;
    c->o = o;
    c->s = (cudaStream_t)stream;
    auto bail = [&](int code) {
        delete c;
        return code;
    };
    // levels: halve while every axis is even and >= 8
    Dims d{g->nx, g->ny, g->nz};
    double h = g->h;
    for (;;) {
        c->dims.push_back(d);
        c->hs.push_back(h);
        if (!(d.nx % 2 == 0 && d.ny % 2 == 0 && d.nz % 2 == 0 && d.nx >= 8 && d.ny >= 8 && d.nz >= 8)) break;
        d = Dims{d.nx / 2, d.ny / 2, d.nz / 2};
        h *= 2.0;
    }
    c->nlev = (int)c->dims.size();
    // the finest FP32 fields are colour-split when its sweeps are colour passes; a hierarchy of
    // two or more levels has even dims on the finest
    if (c->o.prec == MG_MIXED && c->o.smoother <= 1 && c->nlev >= 2)
        c->split0 = mg::Split{c->dims[0].n() / 2, c->dims[0].nx, c->dims[0].ny, mg::make_fastdiv(c->dims[0].nx),
                              mg::make_fastdiv(c->dims[0].ny)};
    const Dims dc = c->dims.back();
    if ((long long)dc.n() > o.coarse_max_cells)
        return bail(fail(MG_ERR_ARG, "mg_setup: coarsest grid %dx%dx%d has %zu cells > coarse_max_cells=%d", dc.nx,
                         dc.ny, dc.nz, dc.n(), o.coarse_max_cells));
    c->ncoarse = (int)dc.n();
    int st = MG_OK;
    c->L64.resize(c->nlev);
    for (int l = 0; l < c->nlev && st == MG_OK; l++) st = level_alloc<double>(c, c->L64[l], c->dims[l].n(), l > 0);
    if (st == MG_OK) st = c->alloc(&c->b0, c->dims[0].n());
    if (st == MG_OK) st = c->alloc(&c->partials, mg::kRedPartials);
    if (st == MG_OK && cudaMemsetAsync(c->partials, 0, mg::kRedPartials * sizeof(double), c->s) != cudaSuccess)
        st = fail(MG_ERR_CUDA, "mg_setup: memset failed");
    if (st == MG_OK) st = c->alloc(&c->dscal, mg::S_COUNT);
    if (st == MG_OK) st = c->alloc(&c->M, (size_t)c->ncoarse * c->ncoarse);
    if (st == MG_OK) st = c->alloc(&c->cc_label, c->dims[0].n());
    if (st == MG_OK) st = c->alloc(&c->open_bits, c->dims[0].n());
    if (st == MG_OK && cudaMemsetAsync(c->open_bits, 0xff, c->dims[0].n(), c->s) != cudaSuccess)
        st = fail(MG_ERR_CUDA, "mg_setup: memset failed");
    if (st == MG_OK) st = c->alloc(&c->cc_ctr, 4);
    if (st == MG_OK) st = c->alloc(&c->pnz, 1);
    if (st == MG_OK) st = c->alloc(&c->cc_roots, kMaxRegions);
    if (st == MG_OK) st = c->alloc(&c->cc_sum, kMaxRegions);
    if (st == MG_OK) st = c->alloc(&c->cc_cnt, kMaxRegions);
    if (st == MG_OK) st = c->alloc(&c->cc_part, 8 * mg::kRedBlocks);
    if (st != MG_OK) return bail(st);
    if (cudaMallocHost(&c->hscal, mg::S_COUNT * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->hcoarse, (3 * (size_t)c->ncoarse + (size_t)c->ncoarse * c->ncoarse + 1) * sizeof(double)) !=
            cudaSuccess ||
        cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_h, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(MG_ERR_CUDA, "mg_setup: pinned buffer / event creation failed"));
    }
    if (c->o.prec == MG_MIXED) {
        c->L32.resize(c->nlev);
        for (int l = 0; l < c->nlev && st == MG_OK; l++) st = level_alloc<float>(c, c->L32[l], c->dims[l].n(), true);
        if (st == MG_OK && c->split0.half) st = c->alloc(&c->urow0, (size_t)c->dims[0].ny * c->dims[0].nz);
        if (st == MG_OK && c->split0.half && c->dims[0].nx % 8 == 0) {
            st = c->alloc(&c->arow0, (size_t)c->dims[0].ny * c->dims[0].nz);
            if (st == MG_OK) st = c->alloc(&c->rowcnt, 2);
            if (st == MG_OK) st = c->alloc(&c->sf0.bx, c->dims[0].n());
            if (st == MG_OK) st = c->alloc(&c->sf0.by, c->dims[0].n());
            if (st == MG_OK) st = c->alloc(&c->sf0.bz, c->dims[0].n());
        }
        if (st != MG_OK) return bail(st);
    }
    if (c->o.krylov) {
        const size_t n0 = c->dims[0].n();
        st = c->alloc(&c->kr, n0);
        if (st == MG_OK) st = level_alloc<double>(c, c->kop, n0, false);
        if (st == MG_OK) st = c->alloc(&c->kd, n0);
        if (st == MG_OK) st = c->alloc(&c->kq, n0);
        if (st == MG_OK && c->o.prec == MG_MIXED) st = c->alloc(&c->ke_alt, n0);
        if (st == MG_OK && c->o.prec != MG_MIXED) st = c->alloc(&c->kz, n0);
        if (st == MG_OK && c->o.prec != MG_MIXED) st = c->alloc(&c->kzo, n0);
        if (st != MG_OK) return bail(st);
    }
    // second iterate buffers for the fused sweeps
    for (int l = 0; l + 1 < c->nlev && st == MG_OK; l++) {
        const bool f64 = c->o.smoother == 2 && fused_level(c->dims[l]);
        const bool f32 = c->o.prec == MG_MIXED && c->o.smoother >= 2 && fused_level(c->dims[l]);
        if (f64) {
            c->palt64.resize(c->nlev, nullptr);
            st = c->alloc(&c->palt64[l], c->dims[l].n());
        }
        if (f32 && st == MG_OK) {
            c->palt32.resize(c->nlev, nullptr);
            st = c->alloc(&c->palt32[l], c->dims[l].n());
        }
    }
    if (st != MG_OK) return bail(st);
    if (c->o.profile) {
        c->pev.resize(2 * 32768);
        c->pgroup.resize(32768);
        for (auto &e : c->pev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return bail(fail(MG_ERR_CUDA, "mg_setup: event creation failed"));
            }
    }
    st = compute_hierarchy(c, face_coeffs);
    if (st != MG_OK) return bail(st);
    c->ms_setup = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = c;
    return MG_OK;
}

int mg_update(mg_ctx *c, const double *const face_coeffs[3])
{
    g_err.clear();
    if (!c || !face_coeffs || !face_coeffs[0] || !face_coeffs[1] || !face_coeffs[2])
        return fail(MG_ERR_ARG, "mg_update: null argument");
    if (!aligned16({face_coeffs[0], face_coeffs[1], face_coeffs[2]}))
        return fail(MG_ERR_ARG, "mg_update: arrays must be 16-byte aligned");
    const auto t0 = std::chrono::steady_clock::now();
    {
        ProfScope ps(c, MG_PROF_UPDATE, true);
        CKS(compute_hierarchy(c, face_coeffs));
    }
    c->ms_setup = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return MG_OK;
}

int mg_solve(mg_ctx *c, const double *rhs, double *p, double tol, mg_stats *stats)
{
    g_err.clear();
    if (!c || !rhs || !p) return fail(MG_ERR_ARG, "mg_solve: null argument");
    if (rhs == p) return fail(MG_ERR_ARG, "mg_solve: rhs and p must not alias");
    if (!aligned16({rhs, p})) return fail(MG_ERR_ARG, "mg_solve: arrays must be 16-byte aligned");
    if (!(tol > 0.0)) return fail(MG_ERR_ARG, "mg_solve: tol must be > 0");
    return c->o.krylov ? pcg_impl(c, rhs, p, tol, stats) : solve_impl(c, rhs, p, tol, stats);
}

int mg_vcycle(mg_ctx *c, const double *rhs, double *p)
{
    g_err.clear();
    if (!c || !rhs || !p) return fail(MG_ERR_ARG, "mg_vcycle: null argument");
    if (!aligned16({rhs, p})) return fail(MG_ERR_ARG, "mg_vcycle: arrays must be 16-byte aligned");
    if (c->o.prec != MG_MIXED) return vcycle<double>(c, c->L64, 0, rhs, p);
    // the cycle of a mixed context: FP32 copies of rhs and p in the finest FP32 level's layout,
    // one FP32 V-cycle on them, p widened back
    const size_t n = c->dims[0].n();
    CK(mg::launch_to_f32_layout(n, rhs, c->L32[0].b, c->s, c->split0));
    CK(mg::launch_to_f32_layout(n, p, c->L32[0].p, c->s, c->split0));
    CKS(vcycle<float>(c, c->L32, 0, c->L32[0].b, c->L32[0].p));
    CK(mg::launch_from_f32_layout(n, c->L32[0].p, p, c->s, c->split0));
    return MG_OK;
}

int mg_divergence(mg_ctx *c, const double *const u[3], double dt, double *rhs)
{
    g_err.clear();
    if (!c || !u || !u[0] || !u[1] || !u[2] || !rhs) return fail(MG_ERR_ARG, "mg_divergence: null argument");
    if (!(dt > 0.0)) return fail(MG_ERR_ARG, "mg_divergence: dt must be > 0");
    if (!aligned16({u[0], u[1], u[2], rhs})) return fail(MG_ERR_ARG, "mg_divergence: arrays must be 16-byte aligned");
    const LevelArrays<double> &L = c->L64[0];
    if (c->has_area || c->has_vb) {
        LevelArrays<double> uu{};
        uu.bx = const_cast<double *>(u[0]);
        uu.by = const_cast<double *>(u[1]);
        uu.bz = const_cast<double *>(u[2]);
        CK(mg::launch_divergence_area(c->dims[0], 1.0 / (dt * c->g.h), L, c->has_area ? c->karea : LevelArrays<double>{},
                                      uu, c->has_vb ? c->kvb : LevelArrays<double>{}, rhs, c->s));
    } else {
        CK(mg::launch_divergence(c->dims[0], 1.0 / (dt * c->g.h), L.bx, L.by, L.bz, u[0], u[1], u[2], rhs, c->s));
    }
    return MG_OK;
}

int mg_correct(mg_ctx *c, const double *const u_star[3], const double *p, double dt, double *const u[3])
{
    g_err.clear();
    if (!c || !u_star || !u || !p) return fail(MG_ERR_ARG, "mg_correct: null argument");
    for (int a = 0; a < 3; a++)
        if (!u_star[a] || !u[a]) return fail(MG_ERR_ARG, "mg_correct: null face array");
    if (!aligned16({u_star[0], u_star[1], u_star[2], u[0], u[1], u[2], p}))
        return fail(MG_ERR_ARG, "mg_correct: arrays must be 16-byte aligned");
    const LevelArrays<double> &L = c->L64[0];
    CK(mg::launch_correct(c->dims[0], dt, c->g.h, L.bx, L.by, L.bz, p, u_star[0], u_star[1], u_star[2], u[0], u[1],
                          u[2], c->s, c->has_area ? &c->kbeta : nullptr));
    return MG_OK;
}

int mg_face_areas(const mg_grid *g, const double *psi_nodes, double *const area_out[3], void *stream)
{
    g_err.clear();
    if (!grid_ok(g)) return fail(MG_ERR_ARG, "mg_face_areas: bad grid");
    if (!psi_nodes || !area_out || !area_out[0] || !area_out[1] || !area_out[2])
        return fail(MG_ERR_ARG, "mg_face_areas: null pointer");
    if (!aligned16({psi_nodes, area_out[0], area_out[1], area_out[2]}))
        return fail(MG_ERR_ARG, "mg_face_areas: arrays must be 16-byte aligned");
    CK(mg::launch_face_areas(Dims{g->nx, g->ny, g->nz}, psi_nodes, area_out[0], area_out[1], area_out[2],
                             (cudaStream_t)stream));
    return MG_OK;
}

int mg_stretched_metrics(const mg_grid *g, const double *hx, const double *hy, const double *hz,
                         const double *const beta[3], const double *const frac[3], double *const beta_out[3],
                         double *const area_out[3], void *stream)
{
    g_err.clear();
    if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1 || (double)g->nx * g->ny * g->nz >= 2147483647.0)
        return fail(MG_ERR_ARG, "mg_stretched_metrics: bad grid");
    if (!hx || !hy || !hz || !beta || !beta_out || !area_out) return fail(MG_ERR_ARG, "mg_stretched_metrics: null pointer");
    for (int a = 0; a < 3; a++)
        if (!beta[a] || !beta_out[a] || !area_out[a] || (frac && !frac[a]))
            return fail(MG_ERR_ARG, "mg_stretched_metrics: null face array");
    if (!aligned16({hx, hy, hz, beta[0], beta[1], beta[2], beta_out[0], beta_out[1], beta_out[2], area_out[0],
                    area_out[1], area_out[2]}) ||
        (frac && !aligned16({frac[0], frac[1], frac[2]})))
        return fail(MG_ERR_ARG, "mg_stretched_metrics: arrays must be 16-byte aligned");
    auto view = [](const double *const x[3]) {
        LevelArrays<double> v{};
        if (x) {
            v.bx = const_cast<double *>(x[0]);
            v.by = const_cast<double *>(x[1]);
            v.bz = const_cast<double *>(x[2]);
        }
        return v;
    };
    CK(mg::launch_stretched_metrics(Dims{g->nx, g->ny, g->nz}, hx, hy, hz, view(beta), view(frac),
                                    view(beta_out), view(area_out), (cudaStream_t)stream));
    return MG_OK;
}

int mg_momentum_rhs(const mg_grid *g, const double *phi, const double *const beta[3], const double *const u[3],
                    const mg_forces *f, double *const R[3], double *work, void *stream)
{
    g_err.clear();
    if (!grid_ok(g)) return fail(MG_ERR_ARG, "mg_momentum_rhs: bad grid");
    if (!phi || !beta || !u || !f || !R || !work) return fail(MG_ERR_ARG, "mg_momentum_rhs: null argument");
    for (int a = 0; a < 3; a++)
        if (!beta[a] || !u[a] || !R[a]) return fail(MG_ERR_ARG, "mg_momentum_rhs: null face array");
    if (!forces_ok(f)) return fail(MG_ERR_ARG, "mg_momentum_rhs: forces not finite or viscosities not >= 0");
    if (!aligned16({phi, beta[0], beta[1], beta[2], u[0], u[1], u[2], R[0], R[1], R[2], work}))
        return fail(MG_ERR_ARG, "mg_momentum_rhs: arrays must be 16-byte aligned");
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            if ((const double *)R[a] == u[b] || (const double *)R[a] == beta[b] || (const double *)R[a] == phi)
                return fail(MG_ERR_ARG, "mg_momentum_rhs: R must not alias its inputs");
    LevelArrays<double> B, U, RR;
    B.bx = const_cast<double *>(beta[0]);
    B.by = const_cast<double *>(beta[1]);
    B.bz = const_cast<double *>(beta[2]);
    U.bx = const_cast<double *>(u[0]);
    U.by = const_cast<double *>(u[1]);
    U.bz = const_cast<double *>(u[2]);
    RR.bx = R[0];
    RR.by = R[1];
    RR.bz = R[2];
    CK(mg::launch_momentum_rhs(Dims{g->nx, g->ny, g->nz}, g->h, phi, f->mu_air, f->mu_water, f->inv_re, f->g,
                               f->convection, B, U, RR, work, (cudaStream_t)stream));
    return MG_OK;
}

int mg_rk2_step(mg_ctx *c, const double *phi, const uint8_t *solid_mask, double rho_air, double rho_water,
                const mg_forces *forces, double dt, double *const u[3], double *phi_out, double *p_out, double tol,
                mg_stats *stats)
{
    g_err.clear();
    if (!c || !phi || !u || !u[0] || !u[1] || !u[2] || !phi_out || !p_out || !forces)
        return fail(MG_ERR_ARG, "mg_rk2_step: null argument");
    if (!(dt > 0.0) || !(tol > 0.0) || !(rho_air > 0.0) || !(rho_water > 0.0) || !forces_ok(forces))
        return fail(MG_ERR_ARG, "mg_rk2_step: dt, tol and the densities must be > 0, the forces finite");
    if (!aligned16({phi, solid_mask, u[0], u[1], u[2], phi_out, p_out}))
        return fail(MG_ERR_ARG, "mg_rk2_step: arrays must be 16-byte aligned");
    if (phi_out == phi) return fail(MG_ERR_ARG, "mg_rk2_step: phi_out must not alias phi");
    const size_t n = c->dims[0].n();
    const Dims d = c->dims[0];
    cudaStream_t s = c->s;
    if (!c->rk_phis) {
        for (LevelArrays<double> *L : {&c->rk_b1, &c->rk_b2, &c->rk_ut, &c->rk_us, &c->rk_r}) {
            CKS(c->alloc(&L->bx, n));
            CKS(c->alloc(&L->by, n));
            CKS(c->alloc(&L->bz, n));
        }
        CKS(c->alloc(&c->rk_phis, n));
        CKS(c->alloc(&c->rk_work, mg::kMomWork * n));
    }
    LevelArrays<double> uk{};
    uk.bx = u[0];
    uk.by = u[1];
    uk.bz = u[2];
    const LevelArrays<double> none{};
    const double drho = rho_water - rho_air, s_dt_h = dt / c->g.h;
    std::string incompat;  // message of a projection that reported an incompatible rhs
    auto faces = [](const LevelArrays<double> &L) {
        return std::array<double *, 3>{L.bx, L.by, L.bz};
    };
    // stage 1: rho(phi^k); u~ = u^k + dt R; u* = u~ - dt B G P*  (Eq. poisson1, runge1)
    CK(mg::launch_face_coeffs(d, phi, solid_mask, rho_air, drho, c->rk_b1.bx, c->rk_b1.by, c->rk_b1.bz, s));
    {
        const auto b1 = faces(c->rk_b1);
        const double *cb1[3] = {b1[0], b1[1], b1[2]};
        CKS(compute_hierarchy(c, cb1));
    }
    // R(u^k, phi^k) with the first stage's 1/rho
    CK(mg::launch_momentum_rhs(d, c->g.h, phi, forces->mu_air, forces->mu_water, forces->inv_re, forces->g,
                               forces->convection, c->rk_b1, uk, c->rk_r, c->rk_work, s));
    CK(mg::launch_rk_combine(n, uk, none, c->rk_r, dt, c->rk_ut, s));
    CK(cudaMemsetAsync(p_out, 0, n * sizeof(double), s));
    {
        const double *ut[3] = {c->rk_ut.bx, c->rk_ut.by, c->rk_ut.bz};
        double *us[3] = {c->rk_us.bx, c->rk_us.by, c->rk_us.bz};
        const int st = mg_project(c, ut, us, p_out, dt, tol, stats);
        if (st == MG_ERR_INCOMPATIBLE) incompat = g_err;
        else if (st != MG_OK) return st;
    }
    // phi* = phi^k - VOF(u^k, phi^k, dt)
    CK(mg::launch_vof_upwind(d, s_dt_h, c->rk_b1, uk, phi, c->rk_phis, s));
    // stage 2: rho(phi*); u~~ = (u* + u^k) + dt R; u^{k+1} = (u~~ - dt B* G P) / 2  (Eq. poisson2, runge2)
    CK(mg::launch_face_coeffs(d, c->rk_phis, solid_mask, rho_air, drho, c->rk_b2.bx, c->rk_b2.by, c->rk_b2.bz, s));
    {
        const auto b2 = faces(c->rk_b2);
        const double *cb2[3] = {b2[0], b2[1], b2[2]};
        CKS(compute_hierarchy(c, cb2));
    }
    // R(u*, phi*) with the second stage's 1/rho
    CK(mg::launch_momentum_rhs(d, c->g.h, c->rk_phis, forces->mu_air, forces->mu_water, forces->inv_re, forces->g,
                               forces->convection, c->rk_b2, c->rk_us, c->rk_r, c->rk_work, s));
    CK(mg::launch_rk_combine(n, c->rk_us, uk, c->rk_r, dt, c->rk_ut, s));
    // (u* + u^k) / 2 for the second VOF, kept in u* (u^k is overwritten below)
    CK(mg::launch_half(n, c->rk_us, uk, c->rk_us, s));
    // phi^{k+1} = phi^k - VOF((u* + u^k)/2, phi^k, dt), with the first stage's face mask
    CK(mg::launch_vof_upwind(d, s_dt_h, c->rk_b1, c->rk_us, phi, phi_out, s));
    CK(cudaMemsetAsync(p_out, 0, n * sizeof(double), s));
    {
        const double *ut[3] = {c->rk_ut.bx, c->rk_ut.by, c->rk_ut.bz};
        const int st = mg_project(c, ut, u, p_out, dt, tol, stats);
        if (st == MG_ERR_INCOMPATIBLE) incompat = g_err;
        else if (st != MG_OK) return st;
    }
    CK(mg::launch_half(n, uk, none, uk, s));
    if (!incompat.empty()) return fail(MG_ERR_INCOMPATIBLE, "%s", incompat.c_str());
    return MG_OK;
}

int mg_set_face_areas(mg_ctx *c, const double *const area[3])
{
    g_err.clear();
    if (!c) return fail(MG_ERR_ARG, "mg_set_face_areas: null context");
    const size_t n0 = c->dims[0].n();
    if (!area) {
        if (!c->has_area) return MG_OK;
        c->has_area = false;
        const double *kb[3] = {c->kbeta.bx, c->kbeta.by, c->kbeta.bz};
        return compute_hierarchy(c, kb);
    }
    if (!area[0] || !area[1] || !area[2]) return fail(MG_ERR_ARG, "mg_set_face_areas: null face array");
    if (!aligned16({area[0], area[1], area[2]}))
        return fail(MG_ERR_ARG, "mg_set_face_areas: arrays must be 16-byte aligned");
    if (!c->karea.bx) {
        CKS(c->alloc(&c->karea.bx, n0));
        CKS(c->alloc(&c->karea.by, n0));
        CKS(c->alloc(&c->karea.bz, n0));
        CKS(c->alloc(&c->kbeta.bx, n0));
        CKS(c->alloc(&c->kbeta.by, n0));
        CKS(c->alloc(&c->kbeta.bz, n0));
    }
    cudaStream_t s = c->s;
    if (!c->has_area) {  // the coefficients given so far are 1/rho
        CK(cudaMemcpyAsync(c->kbeta.bx, c->L64[0].bx, n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(c->kbeta.by, c->L64[0].by, n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(c->kbeta.bz, c->L64[0].bz, n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaMemcpyAsync(c->karea.bx, area[0], n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->karea.by, area[1], n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->karea.bz, area[2], n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    c->has_area = true;
    const double *kb[3] = {c->kbeta.bx, c->kbeta.by, c->kbeta.bz};
    return compute_hierarchy(c, kb);
}

int mg_set_body_velocity(mg_ctx *c, const double *const v[3])
{
    g_err.clear();
    if (!c) return fail(MG_ERR_ARG, "mg_set_body_velocity: null context");
    if (!v) {
        c->has_vb = false;
        return MG_OK;
    }
    if (!v[0] || !v[1] || !v[2]) return fail(MG_ERR_ARG, "mg_set_body_velocity: null face array");
    if (!aligned16({v[0], v[1], v[2]})) return fail(MG_ERR_ARG, "mg_set_body_velocity: arrays must be 16-byte aligned");
    const size_t n0 = c->dims[0].n();
    if (!c->kvb.bx) {
        CKS(c->alloc(&c->kvb.bx, n0));
        CKS(c->alloc(&c->kvb.by, n0));
        CKS(c->alloc(&c->kvb.bz, n0));
    }
    CK(cudaMemcpyAsync(c->kvb.bx, v[0], n0 * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
    CK(cudaMemcpyAsync(c->kvb.by, v[1], n0 * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
    CK(cudaMemcpyAsync(c->kvb.bz, v[2], n0 * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
    c->has_vb = true;
    return MG_OK;
}

int mg_project(mg_ctx *c, const double *const u_star[3], double *const u[3], double *p, double dt, double tol,
               mg_stats *stats)
{
    g_err.clear();
    if (!c || !u_star || !u || !p) return fail(MG_ERR_ARG, "mg_project: null argument");
    for (int a = 0; a < 3; a++)
        if (!u_star[a] || !u[a]) return fail(MG_ERR_ARG, "mg_project: null face array");
    if (!(dt > 0.0) || !(tol > 0.0)) return fail(MG_ERR_ARG, "mg_project: dt and tol must be > 0");
    if (!aligned16({u_star[0], u_star[1], u_star[2], u[0], u[1], u[2], p}))
        return fail(MG_ERR_ARG, "mg_project: arrays must be 16-byte aligned");
    CKS(ensure(c, &c->rhs_tmp, c->dims[0].n()));
    CKS(mg_divergence(c, u_star, dt, c->rhs_tmp));
    const int st = c->o.krylov ? pcg_impl(c, c->rhs_tmp, p, tol, stats) : solve_impl(c, c->rhs_tmp, p, tol, stats);
    if (st != MG_OK && st != MG_ERR_NOT_CONVERGED && st != MG_ERR_INCOMPATIBLE) return st;
    const std::string keep = g_err;
    CKS(mg_correct(c, u_star, p, dt, u));
    g_err = keep;
    return st;
}

int mg_project_adjoint(mg_ctx *c, const double *const w[3], const double *p, double dt, double tol,
                       double *const grad_u[3], double *const grad_beta[3], double *q_out, mg_stats *stats)
{
    g_err.clear();
    if (!c || !w || !p || !grad_u) return fail(MG_ERR_ARG, "mg_project_adjoint: null argument");
    for (int a = 0; a < 3; a++) {
        if (!w[a] || !grad_u[a]) return fail(MG_ERR_ARG, "mg_project_adjoint: null face array");
        for (int b = 0; b < 3; b++)
            if ((const double *)grad_u[a] == w[b]) return fail(MG_ERR_ARG, "mg_project_adjoint: grad_u aliases w");
    }
    if (!(dt > 0.0) || !(tol > 0.0)) return fail(MG_ERR_ARG, "mg_project_adjoint: dt and tol must be > 0");
    if (!aligned16({w[0], w[1], w[2], grad_u[0], grad_u[1], grad_u[2], p, q_out}) ||
        (grad_beta && !aligned16({grad_beta[0], grad_beta[1], grad_beta[2]})))
        return fail(MG_ERR_ARG, "mg_project_adjoint: arrays must be 16-byte aligned");
    const size_t n = c->dims[0].n();
    CKS(ensure(c, &c->rhs_tmp, n));
    double *q = q_out;
    if (!q) {
        CKS(ensure(c, &c->qbuf, n));
        q = c->qbuf;
        CK(cudaMemsetAsync(q, 0, n * sizeof(double), c->s));
    }
    const LevelArrays<double> &L = c->L64[0];
    // c = D(beta w), the products beta * w rounded once; beta = 1/rho (with fractional areas the
    // operator's coefficient is area * 1/rho, and D sums the open faces without their areas)
    const LevelArrays<double> &B = c->has_area ? c->kbeta : L;
    CK(mg::launch_divergence_mul(c->dims[0], 1.0 / c->g.h, L, B, w[0], w[1], w[2], c->rhs_tmp, c->s));
    const int st = c->o.krylov ? pcg_impl(c, c->rhs_tmp, q, tol, stats) : solve_impl(c, c->rhs_tmp, q, tol, stats);
    if (st != MG_OK && st != MG_ERR_NOT_CONVERGED && st != MG_ERR_INCOMPATIBLE) return st;
    const std::string keep = g_err;
    double *gb[3] = {nullptr, nullptr, nullptr};
    if (grad_beta)
        for (int a = 0; a < 3; a++) gb[a] = grad_beta[a];
    CK(mg::launch_adjoint_faces(c->dims[0], c->g.h, dt, L.bx, L.by, L.bz, p, q, w[0], w[1], w[2], grad_u[0],
                                grad_u[1], grad_u[2], gb[0], gb[1], gb[2], c->s, c->has_area ? &c->karea : nullptr));
    g_err = keep;
    return st;
}

int mg_phi_grad(const mg_grid *g, const double *const beta[3], const double *const grad_beta[3], double rho_air,
                double rho_water, double *grad_phi, void *stream)
{
    g_err.clear();
    if (!grid_ok(g)) return fail(MG_ERR_ARG, "mg_phi_grad: bad grid");
    if (!beta || !grad_beta || !grad_phi) return fail(MG_ERR_ARG, "mg_phi_grad: null argument");
    for (int a = 0; a < 3; a++)
        if (!beta[a] || !grad_beta[a]) return fail(MG_ERR_ARG, "mg_phi_grad: null face array");
    if (!aligned16({beta[0], beta[1], beta[2], grad_beta[0], grad_beta[1], grad_beta[2], grad_phi}))
        return fail(MG_ERR_ARG, "mg_phi_grad: arrays must be 16-byte aligned");
    const Dims d{g->nx, g->ny, g->nz};
    CK(mg::launch_phi_grad(d, -0.5 * (rho_water - rho_air), beta[0], beta[1], beta[2], grad_beta[0], grad_beta[1],
                           grad_beta[2], grad_phi, (cudaStream_t)stream));
    return MG_OK;
}

int mg_num_levels(const mg_ctx *c) { return c ? c->nlev : 0; }

int mg_level_dims(const mg_ctx *c, int level, int dims[3])
{
    if (!c || !dims || level < 0 || level >= c->nlev) return fail(MG_ERR_ARG, "mg_level_dims: bad level");
    dims[0] = c->dims[level].nx;
    dims[1] = c->dims[level].ny;
    dims[2] = c->dims[level].nz;
    return MG_OK;
}

int mg_level_array(mg_ctx *c, int level, int which, double *out)
{
    g_err.clear();
    if (!c || !out || level < 0 || level >= c->nlev || which < 0 || which > 3)
        return fail(MG_ERR_ARG, "mg_level_array: bad argument");
    if (!aligned16({out})) return fail(MG_ERR_ARG, "mg_level_array: out must be 16-byte aligned");
    const LevelArrays<double> &L = c->L64[level];
    const double *src = which == 0 ? L.bx : which == 1 ? L.by : which == 2 ? L.bz : L.dinv;
    CK(cudaMemcpyAsync(out, src, c->dims[level].n() * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
    return MG_OK;
}

uint64_t mg_kernel_launches(void) { return (uint64_t)mg::launch_count(); }

int mg_check_read(int *enabled, uint64_t *first, uint64_t *count)
{
    g_err.clear();
    if (!enabled || !first || !count) return fail(MG_ERR_ARG, "mg_check_read: null argument");
    unsigned long long f = 0, n = 0;
    const int r = mg::check_read(&f, &n);
    if (r < 0) return fail(MG_ERR_CUDA, "mg_check_read: reading the check record failed");
    *enabled = r;
    *first = f;
    *count = n;
    return MG_OK;
}

int mg_profile_read(mg_ctx *c, int group, int *count, double *ms_total)
{
    g_err.clear();
    if (!c || group < 0 || group >= MG_PROF_GROUPS) return fail(MG_ERR_ARG, "mg_profile_read: bad argument");
    int n = 0;
    double tot = 0.0;
    for (size_t i = 0; i + 1 < c->pused; i += 2) {
        if (c->pgroup[i / 2] != group) continue;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->pev[i], c->pev[i + 1]));
        tot += ms;
        n++;
    }
    if (count) *count = n;
    if (ms_total) *ms_total = tot;
    return MG_OK;
}

void mg_profile_reset(mg_ctx *c)
{
    if (c) c->pused = 0;
}

void mg_destroy(mg_ctx *c)
{
    if (!c) return;
    if (c->s) cudaStreamSynchronize(c->s);
    else cudaDeviceSynchronize();
    delete c;
}

}  // extern "C"
