/*
 * mg_oracle.c -- plain FP64 CPU oracle of the variable-density pressure projection.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; it is loaded by the tests, by the smoke check and by the
 * CPU-baseline leg of the benchmark.  It shares no code with the CUDA path.
 *
 * It is written for a reader who checks it against the paper by eye: plain
 * loops over cells and faces, no blocking, no fusion, fixed summation order.
 * Rounding is specified, not left to the compiler (-ffp-contract=off): the
 * stencil sums of the smoother, the residual and the prolongation accumulate
 * their products with C99 fma() in the stated order; everything else is
 * separately rounded IEEE arithmetic.
 *
 * Grid: nx*ny*nz cells, isotropic spacing h, C order [k][j][i], x fastest.
 * Faces: bx[k][j][i] is the x-face between cells (i-1,j,k) and (i,j,k); i = 0 is
 * the low wall (always closed); the high wall face is not stored (closed).
 * Same for by (index j) and bz (index k).
 *
 * Discrete problem (paper, Eq. pois / Eq. poisson1 with the finite-volume form
 * Eq. integral2, the static body contributing no flux):
 *     (A p)_c = h^-2 * sum_{open faces f of c} beta_f (p_nb - p_c) = b_c
 * with beta_f = area_f / rho_f the face value of (1/rho)*area (Poisson solver
 * section) and rho = lam + (1 - lam) * phi (Eq. density, H(phi) = phi).
 *
 * Parity pins for every function are in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IX(i, j, k) (((size_t)(k) * (size_t)ny + (size_t)(j)) * (size_t)nx + (size_t)(i))

/* ------------------------------------------------------------------------- */
/* Face coefficients (Eq. density; Poisson solver section: the product of     */
/* one over the density and the cut-surface area, evaluated on fine faces).   */
/* The face density is the harmonic mean of 1/rho of the two cells,          */
/* i.e. beta = 2 / (rho_L + rho_R).  Faces that are walls or touch a solid    */
/* cell have zero area (binary cut cells).                                   */
/* ------------------------------------------------------------------------- */
static double face_beta(double phiL, double phiR, double lam)
{
    double rhoL = lam + (1.0 - lam) * phiL;
    double rhoR = lam + (1.0 - lam) * phiR;
    return 2.0 / (rhoL + rhoR);
}

void orc_face_coeffs(int nx, int ny, int nz, const double *phi, const uint8_t *solid, double lam,
                     double *bx, double *by, double *bz)
{
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = IX(i, j, k);
                int sc = solid ? solid[c] : 0;
                /* x face between (i-1,j,k) and (i,j,k) */
                if (i == 0 || sc || (solid && solid[IX(i - 1, j, k)]))
                    bx[c] = 0.0;
                else
                    bx[c] = face_beta(phi[IX(i - 1, j, k)], phi[c], lam);
                if (j == 0 || sc || (solid && solid[IX(i, j - 1, k)]))
                    by[c] = 0.0;
                else
                    by[c] = face_beta(phi[IX(i, j - 1, k)], phi[c], lam);
                if (k == 0 || sc || (solid && solid[IX(i, j, k - 1)]))
                    bz[c] = 0.0;
                else
                    bz[c] = face_beta(phi[IX(i, j, k - 1)], phi[c], lam);
            }
}

/* ------------------------------------------------------------------------- */
/* Operator A (Eq. integral2 divided by the cell volume): for each of the six */
/* faces in the order x-, x+, y-, y+, z-, z+ add beta_f (p_nb - p_c); scale   */
/* by h^-2.  A wall face has no neighbour and no term.                        */
/* ------------------------------------------------------------------------- */
void orc_apply_A(int nx, int ny, int nz, double h, const double *bx, const double *by,
                 const double *bz, const double *p, double *Ap)
{
    double ih2 = 1.0 / (h * h);
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = IX(i, j, k);
                double s = 0.0;
                if (i > 0) s += bx[c] * (p[IX(i - 1, j, k)] - p[c]);
                if (i < nx - 1) s += bx[IX(i + 1, j, k)] * (p[IX(i + 1, j, k)] - p[c]);
                if (j > 0) s += by[c] * (p[IX(i, j - 1, k)] - p[c]);
                if (j < ny - 1) s += by[IX(i, j + 1, k)] * (p[IX(i, j + 1, k)] - p[c]);
                if (k > 0) s += bz[c] * (p[IX(i, j, k - 1)] - p[c]);
                if (k < nz - 1) s += bz[IX(i, j, k + 1)] * (p[IX(i, j, k + 1)] - p[c]);
                Ap[c] = s * ih2;
            }
}

/* sum of the six face coefficients of each cell; dinv = 1/sum, 0 if sum = 0 */
void orc_diag_inv(int nx, int ny, int nz, const double *bx, const double *by, const double *bz,
                  double *dinv)
{
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = IX(i, j, k);
                double s = bx[c];
                s += (i < nx - 1) ? bx[IX(i + 1, j, k)] : 0.0;
                s += by[c];
                s += (j < ny - 1) ? by[IX(i, j + 1, k)] : 0.0;
                s += bz[c];
                s += (k < nz - 1) ? bz[IX(i, j, k + 1)] : 0.0;
                dinv[c] = (s > 0.0) ? 1.0 / s : 0.0;
            }
}

/* ------------------------------------------------------------------------- */
/* Connected fluid components: cells joined by faces with beta > 0.  A cell   */
/* with no open face is its own component (isolated).  Breadth-first search.  */
/* The Neumann problem (Eq. neumann on the hull, closed walls) determines p   */
/* up to one constant per component.                                          */
/* ------------------------------------------------------------------------- */
int orc_components(int nx, int ny, int nz, const double *bx, const double *by, const double *bz,
                   int *label)
{
    size_t n = (size_t)nx * ny * nz;
    for (size_t c = 0; c < n; c++) label[c] = -1;
    size_t *queue = (size_t *)malloc(n * sizeof(size_t));
    int ncomp = 0;
    for (size_t seed = 0; seed < n; seed++) {
        if (label[seed] >= 0) continue;
        size_t head = 0, tail = 0;
        queue[tail++] = seed;
        label[seed] = ncomp;
        while (head < tail) {
            size_t c = queue[head++];
            int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((size_t)nx * ny));
            size_t nb[6];
            double fb[6];
            int m = 0;
            if (i > 0) { nb[m] = IX(i - 1, j, k); fb[m++] = bx[c]; }
            if (i < nx - 1) { nb[m] = IX(i + 1, j, k); fb[m++] = bx[IX(i + 1, j, k)]; }
            if (j > 0) { nb[m] = IX(i, j - 1, k); fb[m++] = by[c]; }
            if (j < ny - 1) { nb[m] = IX(i, j + 1, k); fb[m++] = by[IX(i, j + 1, k)]; }
            if (k > 0) { nb[m] = IX(i, j, k - 1); fb[m++] = bz[c]; }
            if (k < nz - 1) { nb[m] = IX(i, j, k + 1); fb[m++] = bz[IX(i, j, k + 1)]; }
            for (int q = 0; q < m; q++)
                if (fb[q] > 0.0 && label[nb[q]] < 0) {
                    label[nb[q]] = ncomp;
                    queue[tail++] = nb[q];
                }
        }
        ncomp++;
    }
    free(queue);
    return ncomp;
}

/* subtract from v its mean over each component (isolated cells become 0) */
void orc_remove_mean(size_t n, const int *label, int ncomp, double *v)
{
    double *sum = (double *)calloc((size_t)ncomp, sizeof(double));
    double *cnt = (double *)calloc((size_t)ncomp, sizeof(double));
    for (size_t c = 0; c < n; c++) {
        sum[label[c]] += v[c];
        cnt[label[c]] += 1.0;
    }
    for (size_t c = 0; c < n; c++) v[c] -= sum[label[c]] / cnt[label[c]];
    free(sum);
    free(cnt);
}

/* ------------------------------------------------------------------------- */
/* Red-black Gauss-Seidel: one colour (colour = (i+j+k) mod 2).  Each cell    */
/* of that colour solves its own row of A p = b with its neighbours fixed:     */
/*   p_c = dinv_c * (sum_f beta_f p_nb - h^2 b_c)                            */
/* Sum order: x-, x+, y-, y+, z-, z+ (fma).  No two cells of one colour touch */
/* each other, so the update order inside a colour does not matter.           */
/* ------------------------------------------------------------------------- */
void orc_smooth_colour(int nx, int ny, int nz, double h, const double *bx, const double *by,
                       const double *bz, const double *dinv, const double *b, double *p, int colour)
{
    double h2 = h * h;
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                if (((i + j + k) & 1) != colour) continue;
                size_t c = IX(i, j, k);
                double s = 0.0;
                if (i > 0) s = fma(bx[c], p[IX(i - 1, j, k)], s);
                if (i < nx - 1) s = fma(bx[IX(i + 1, j, k)], p[IX(i + 1, j, k)], s);
                if (j > 0) s = fma(by[c], p[IX(i, j - 1, k)], s);
                if (j < ny - 1) s = fma(by[IX(i, j + 1, k)], p[IX(i, j + 1, k)], s);
                if (k > 0) s = fma(bz[c], p[IX(i, j, k - 1)], s);
                if (k < nz - 1) s = fma(bz[IX(i, j, k + 1)], p[IX(i, j, k + 1)], s);
                p[c] = dinv[c] * fma(-h2, b[c], s); /* dinv * (s - h^2 b) */
            }
}

/* ------------------------------------------------------------------------- */
/* Coefficient restriction (Poisson solver section: the face product          */
/* (1/rho)*area is moved from the fine to the coarse grid as one unit).  The  */
/* coarse face is covered by 2x2 coplanar fine faces; its coefficient is      */
/* their mean (the fine fluxes through the four faces add up to the coarse    */
/* flux, with the coarse gradient over twice the spacing).                    */
/* ------------------------------------------------------------------------- */
void orc_restrict_coeffs(int nx, int ny, int nz, const double *bx, const double *by, const double *bz,
                         double *cbx, double *cby, double *cbz)
{
    int NX = nx / 2, NY = ny / 2, NZ = nz / 2;
    #pragma omp parallel for schedule(static)
    for (int K = 0; K < NZ; K++)
        for (int J = 0; J < NY; J++)
            for (int I = 0; I < NX; I++) {
                size_t C = ((size_t)K * NY + J) * NX + I;
                cbx[C] = 0.25 * (bx[IX(2 * I, 2 * J, 2 * K)] + bx[IX(2 * I, 2 * J + 1, 2 * K)] +
                                 bx[IX(2 * I, 2 * J, 2 * K + 1)] + bx[IX(2 * I, 2 * J + 1, 2 * K + 1)]);
                cby[C] = 0.25 * (by[IX(2 * I, 2 * J, 2 * K)] + by[IX(2 * I + 1, 2 * J, 2 * K)] +
                                 by[IX(2 * I, 2 * J, 2 * K + 1)] + by[IX(2 * I + 1, 2 * J, 2 * K + 1)]);
                cbz[C] = 0.25 * (bz[IX(2 * I, 2 * J, 2 * K)] + bz[IX(2 * I + 1, 2 * J, 2 * K)] +
                                 bz[IX(2 * I, 2 * J + 1, 2 * K)] + bz[IX(2 * I + 1, 2 * J + 1, 2 * K)]);
            }
}

/* residual r = b - A p: the flux sum s = sum_f beta_f (p_nb - p_c) (fma, order  */
/* x-, x+, y-, y+, z-, z+), then r = b - h^-2 s (fma)                          */
void orc_residual(int nx, int ny, int nz, double h, const double *bx, const double *by,
                  const double *bz, const double *b, const double *p, double *r)
{
    double ih2 = 1.0 / (h * h);
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = IX(i, j, k);
                double s = 0.0;
                if (i > 0) s = fma(bx[c], p[IX(i - 1, j, k)] - p[c], s);
                if (i < nx - 1) s = fma(bx[IX(i + 1, j, k)], p[IX(i + 1, j, k)] - p[c], s);
                if (j > 0) s = fma(by[c], p[IX(i, j - 1, k)] - p[c], s);
                if (j < ny - 1) s = fma(by[IX(i, j + 1, k)], p[IX(i, j + 1, k)] - p[c], s);
                if (k > 0) s = fma(bz[c], p[IX(i, j, k - 1)] - p[c], s);
                if (k < nz - 1) s = fma(bz[IX(i, j, k + 1)], p[IX(i, j, k + 1)] - p[c], s);
                r[c] = fma(-s, ih2, b[c]);
            }
}

/* cell-centred full weighting: coarse value = mean of the 8 children */
void orc_restrict(int nx, int ny, int nz, const double *r, double *rc)
{
    int NX = nx / 2, NY = ny / 2, NZ = nz / 2;
    #pragma omp parallel for schedule(static)
    for (int K = 0; K < NZ; K++)
        for (int J = 0; J < NY; J++)
            for (int I = 0; I < NX; I++) {
                double s = 0.0;
                for (int dk = 0; dk < 2; dk++)
                    for (int dj = 0; dj < 2; dj++)
                        for (int di = 0; di < 2; di++) s += r[IX(2 * I + di, 2 * J + dj, 2 * K + dk)];
                rc[((size_t)K * NY + J) * NX + I] = 0.125 * s;
            }
}

/* Trilinear cell-centred prolongation added to p.  Along each axis the fine  */
/* centre lies a quarter coarse cell from its parent's centre: weight 3/4 on  */
/* the parent and 1/4 on the next coarse cell on the same side; that index    */
/* is clamped to the domain at walls.  Cells with dinv = 0 are not updated.   */
/* The 8 weighted values are accumulated with fma (K outer, then J, then I).  */
void orc_prolong_add(int nx, int ny, int nz, const double *ec, const double *dinv, double *p)
{
    int NX = nx / 2, NY = ny / 2, NZ = nz / 2;
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = IX(i, j, k);
                if (dinv[c] == 0.0) continue;
                int I0 = i / 2, J0 = j / 2, K0 = k / 2;
                int I1 = (i & 1) ? I0 + 1 : I0 - 1;
                int J1 = (j & 1) ? J0 + 1 : J0 - 1;
                int K1 = (k & 1) ? K0 + 1 : K0 - 1;
                if (I1 < 0) I1 = 0;
                if (I1 > NX - 1) I1 = NX - 1;
                if (J1 < 0) J1 = 0;
                if (J1 > NY - 1) J1 = NY - 1;
                if (K1 < 0) K1 = 0;
                if (K1 > NZ - 1) K1 = NZ - 1;
                int Is[2] = {I0, I1}, Js[2] = {J0, J1}, Ks[2] = {K0, K1};
                double w[2] = {0.75, 0.25};
                double s = 0.0;
                for (int a = 0; a < 2; a++)
                    for (int bb = 0; bb < 2; bb++)
                        for (int d = 0; d < 2; d++)
                            s = fma(w[a] * w[bb] * w[d], ec[((size_t)Ks[a] * NY + Js[bb]) * NX + Is[d]], s);
                p[c] += s;
            }
}

/* ------------------------------------------------------------------------- */
/* Dense symmetric pseudo-inverse by the cyclic Jacobi eigenvalue method       */
/* (symmetric Schur decomposition, Golub & Van Loan sec. 8.5).  Eigenvalues    */
/* below 1e-9 of the largest magnitude are treated as zero (the null space:    */
/* one constant per component).  Used for the exact coarsest-grid solve.       */
/* ------------------------------------------------------------------------- */
void orc_pinv_sym(int n, const double *A, double *X)
{
    double *a = (double *)malloc((size_t)n * n * sizeof(double));
    double *v = (double *)calloc((size_t)n * n, sizeof(double));
    memcpy(a, A, (size_t)n * n * sizeof(double));
    for (int i = 0; i < n; i++) v[(size_t)i * n + i] = 1.0;
    double off_prev = -1.0;
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int p = 0; p < n; p++)
            for (int q = 0; q < n; q++) {
                double x = a[(size_t)p * n + q];
                tot += x * x;
                if (p != q) off += x * x;
            }
        /* stop at a relative off-diagonal mass of 1e-30, or once a sweep no
           longer halves it (the rounding floor has been reached) */
        if (off <= 1e-30 * tot || off == 0.0) break;
        if (off_prev >= 0.0 && off > 0.25 * off_prev && off <= 1e-24 * tot) break;
        off_prev = off;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                double apq = a[(size_t)p * n + q];
                if (apq == 0.0) continue;
                double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                /* a <- J^T a J with the rotation in the (p,q) plane */
                for (int m = 0; m < n; m++) {
                    double amp = a[(size_t)m * n + p], amq = a[(size_t)m * n + q];
                    a[(size_t)m * n + p] = cs * amp - sn * amq;
                    a[(size_t)m * n + q] = sn * amp + cs * amq;
                }
                for (int m = 0; m < n; m++) {
                    double apm = a[(size_t)p * n + m], aqm = a[(size_t)q * n + m];
                    a[(size_t)p * n + m] = cs * apm - sn * aqm;
                    a[(size_t)q * n + m] = sn * apm + cs * aqm;
                }
                for (int m = 0; m < n; m++) {
                    double vmp = v[(size_t)m * n + p], vmq = v[(size_t)m * n + q];
                    v[(size_t)m * n + p] = cs * vmp - sn * vmq;
                    v[(size_t)m * n + q] = sn * vmp + cs * vmq;
                }
            }
    }
    double lmax = 0.0;
    for (int i = 0; i < n; i++) lmax = fmax(lmax, fabs(a[(size_t)i * n + i]));
    memset(X, 0, (size_t)n * n * sizeof(double));
    for (int m = 0; m < n; m++) {
        double lam = a[(size_t)m * n + m];
        if (fabs(lam) <= 1e-9 * lmax) continue;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) X[(size_t)i * n + j] += v[(size_t)i * n + m] * v[(size_t)j * n + m] / lam;
    }
    free(a);
    free(v);
}

/* dense matrix of A (row c holds (A e_nb)_c), for the coarsest grid and tests */
void orc_dense_A(int nx, int ny, int nz, double h, const double *bx, const double *by, const double *bz,
                 double *M)
{
    size_t n = (size_t)nx * ny * nz;
    double *e = (double *)calloc(n, sizeof(double));
    double *col = (double *)malloc(n * sizeof(double));
    for (size_t q = 0; q < n; q++) {
        e[q] = 1.0;
        orc_apply_A(nx, ny, nz, h, bx, by, bz, e, col);
        for (size_t c = 0; c < n; c++) M[c * n + q] = col[c];
        e[q] = 0.0;
    }
    free(e);
    free(col);
}

/* ------------------------------------------------------------------------- */
/* Geometric multigrid hierarchy.  Coarsen while every dimension is even and  */
/* at least 8 (level spacing doubles).  The coarsest grid is solved exactly   */
/* with the pseudo-inverse (minimum-norm solution).                           */
/* ------------------------------------------------------------------------- */
#define ORC_MAXLEV 24
typedef struct {
    int nx, ny, nz;
    double h;
    double *bx, *by, *bz, *dinv, *b, *p, *r;
} orc_level;

typedef struct {
    int nlev, nu1, nu2;
    orc_level lev[ORC_MAXLEV];
    double *pinv; /* coarsest-grid pseudo-inverse, n x n */
} orc_mg;

static double *dalloc(size_t n) { return (double *)calloc(n, sizeof(double)); }

orc_mg *orc_mg_create(int nx, int ny, int nz, double h, const double *bx, const double *by,
                      const double *bz, int nu1, int nu2, int max_coarse)
{
    orc_mg *m = (orc_mg *)calloc(1, sizeof(orc_mg));
    m->nu1 = nu1;
    m->nu2 = nu2;
    int l = 0;
    for (;;) {
        orc_level *L = &m->lev[l];
        L->nx = nx;
        L->ny = ny;
        L->nz = nz;
        L->h = h;
        size_t n = (size_t)nx * ny * nz;
        L->bx = dalloc(n);
        L->by = dalloc(n);
        L->bz = dalloc(n);
        L->dinv = dalloc(n);
        L->b = dalloc(n);
        L->p = dalloc(n);
        L->r = dalloc(n);
        if (l == 0) {
            memcpy(L->bx, bx, n * sizeof(double));
            memcpy(L->by, by, n * sizeof(double));
            memcpy(L->bz, bz, n * sizeof(double));
        } else {
            orc_level *F = &m->lev[l - 1];
            orc_restrict_coeffs(F->nx, F->ny, F->nz, F->bx, F->by, F->bz, L->bx, L->by, L->bz);
        }
        orc_diag_inv(nx, ny, nz, L->bx, L->by, L->bz, L->dinv);
        l++;
        if (!(nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0 && nx >= 8 && ny >= 8 && nz >= 8) || l == ORC_MAXLEV)
            break;
        nx /= 2;
        ny /= 2;
        nz /= 2;
        h *= 2.0;
    }
    m->nlev = l;
    orc_level *C = &m->lev[l - 1];
    size_t nc = (size_t)C->nx * C->ny * C->nz;
    if (max_coarse > 0 && nc > (size_t)max_coarse) {
        m->pinv = NULL;
        return m;
    }
    double *Ad = dalloc(nc * nc);
    m->pinv = dalloc(nc * nc);
    orc_dense_A(C->nx, C->ny, C->nz, C->h, C->bx, C->by, C->bz, Ad);
    orc_pinv_sym((int)nc, Ad, m->pinv);
    free(Ad);
    return m;
}

void orc_mg_free(orc_mg *m)
{
    if (!m) return;
    for (int l = 0; l < m->nlev; l++) {
        orc_level *L = &m->lev[l];
        free(L->bx); free(L->by); free(L->bz); free(L->dinv); free(L->b); free(L->p); free(L->r);
    }
    free(m->pinv);
    free(m);
}

int orc_mg_nlev(const orc_mg *m) { return m->nlev; }
int orc_mg_ok(const orc_mg *m) { return m->pinv != NULL; }
void orc_mg_level_dims(const orc_mg *m, int l, int *dims) { dims[0] = m->lev[l].nx; dims[1] = m->lev[l].ny; dims[2] = m->lev[l].nz; }
const double *orc_mg_level_array(const orc_mg *m, int l, int which)
{
    const orc_level *L = &m->lev[l];
    switch (which) {
    case 0: return L->bx;
    case 1: return L->by;
    case 2: return L->bz;
    case 3: return L->dinv;
    default: return NULL;
    }
}
const double *orc_mg_pinv(const orc_mg *m) { return m->pinv; }

/* one V(nu1, nu2) cycle on level l: b given, p updated in place */
static void vcycle(orc_mg *m, int l, const double *b, double *p)
{
    orc_level *L = &m->lev[l];
    size_t n = (size_t)L->nx * L->ny * L->nz;
    if (l == m->nlev - 1) {
        /* exact coarsest-grid solve: p = A^+ b (p's incoming value is discarded) */
        for (size_t i = 0; i < n; i++) {
            double s = 0.0;
            for (size_t j = 0; j < n; j++) s += m->pinv[i * n + j] * b[j];
            p[i] = s;
        }
        return;
    }
    for (int s = 0; s < m->nu1; s++) {
        orc_smooth_colour(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, L->dinv, b, p, 0);
        orc_smooth_colour(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, L->dinv, b, p, 1);
    }
    orc_level *C = &m->lev[l + 1];
    size_t nc = (size_t)C->nx * C->ny * C->nz;
    orc_residual(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, b, p, L->r);
    orc_restrict(L->nx, L->ny, L->nz, L->r, C->b);
    memset(C->p, 0, nc * sizeof(double));
    vcycle(m, l + 1, C->b, C->p);
    orc_prolong_add(L->nx, L->ny, L->nz, C->p, L->dinv, p);
    for (int s = 0; s < m->nu2; s++) {
        orc_smooth_colour(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, L->dinv, b, p, 1);
        orc_smooth_colour(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, L->dinv, b, p, 0);
    }
}

/* One V-cycle on the finest level, without mean removal. */
void orc_mg_vcycle(orc_mg *m, const double *b, double *p) { vcycle(m, 0, b, p); }

static double norm2(size_t n, const double *v)
{
    double s = 0.0;
    for (size_t i = 0; i < n; i++) s += v[i] * v[i];
    return sqrt(s);
}

/* Multigrid solve: b is made compatible (per-component mean removed), then   */
/* V-cycles until ||b - A p|| / ||b|| <= tol; p's per-component mean is        */
/* removed after every cycle.  Returns the number of cycles (negative if not   */
/* converged); hist[c] = relative residual after cycle c+1.                    */
int orc_mg_solve(orc_mg *m, const double *b_in, double *p, double tol, int max_cycles, double *hist)
{
    orc_level *L = &m->lev[0];
    size_t n = (size_t)L->nx * L->ny * L->nz;
    int *label = (int *)malloc(n * sizeof(int));
    int ncomp = orc_components(L->nx, L->ny, L->nz, L->bx, L->by, L->bz, label);
    double *b = dalloc(n);
    memcpy(b, b_in, n * sizeof(double));
    orc_remove_mean(n, label, ncomp, b);
    double nb = norm2(n, b);
    int cyc = 0, ok = 0;
    if (nb == 0.0) {
        memset(p, 0, n * sizeof(double));
        ok = 1;
    }
    for (cyc = 1; !ok && cyc <= max_cycles; cyc++) {
        vcycle(m, 0, b, p);
        orc_remove_mean(n, label, ncomp, p);
        orc_residual(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, b, p, L->r);
        double rel = norm2(n, L->r) / nb;
        if (hist) hist[cyc - 1] = rel;
        if (rel <= tol) { ok = 1; break; }
    }
    free(label);
    free(b);
    if (nb == 0.0) return 0;
    return ok ? cyc : -max_cycles;
}

/* ------------------------------------------------------------------------- */
/* Multigrid-preconditioned conjugate gradients (the paper's preconditioned-CG */
/* family with the multigrid cycle as the preconditioner, Poisson-solver       */
/* section).  PCG on the semi-definite A (the signs cancel in alpha and beta), */
/* in the flexible (Polak-Ribiere) form beta = <r', z' - z> / <r, z>, which    */
/* tolerates a preconditioner that is not exactly symmetric (the cycle's       */
/* restriction is not the transpose of its prolongation); the preconditioner   */
/* is nvc V-cycles from a zero guess.  The                                     */
/* recursively updated residual decides convergence; the true residual is then */
/* checked and the iteration restarted from the current p if it is above tol.  */
/* Returns iterations (negative if not converged); hist[i] = recursive         */
/* relative residual after iteration i+1.                                      */
/* ------------------------------------------------------------------------- */
static double dot(size_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (size_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

int orc_mg_pcg(orc_mg *m, const double *b_in, double *p, double tol, int max_it, int nvc, double *hist)
{
    orc_level *L = &m->lev[0];
    size_t n = (size_t)L->nx * L->ny * L->nz;
    int *label = (int *)malloc(n * sizeof(int));
    int ncomp = orc_components(L->nx, L->ny, L->nz, L->bx, L->by, L->bz, label);
    double *b = dalloc(n), *r = dalloc(n), *z = dalloc(n), *zo = dalloc(n), *d = dalloc(n), *q = dalloc(n);
    memcpy(b, b_in, n * sizeof(double));
    orc_remove_mean(n, label, ncomp, b);
    double nb = norm2(n, b);
    int it = 0, ok = (nb == 0.0);
    if (ok) memset(p, 0, n * sizeof(double));
    while (!ok && it < max_it) {
        /* (re)start from the current p with its true residual */
        orc_residual(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, b, p, r);
        if (norm2(n, r) / nb <= tol) { ok = 1; break; }
        memset(z, 0, n * sizeof(double));
        for (int v = 0; v < nvc; v++) vcycle(m, 0, r, z);
        memcpy(d, z, n * sizeof(double));
        double rz = dot(n, r, z);
        while (it < max_it) {
            it++;
            orc_apply_A(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, d, q);
            double alpha = rz / dot(n, d, q);
            for (size_t c = 0; c < n; c++) { p[c] += alpha * d[c]; r[c] -= alpha * q[c]; }
            double rel = norm2(n, r) / nb;
            if (hist) hist[it - 1] = rel;
            if (rel <= tol) break;
            memcpy(zo, z, n * sizeof(double));
            memset(z, 0, n * sizeof(double));
            for (int v = 0; v < nvc; v++) vcycle(m, 0, r, z);
            double rzn = dot(n, r, z);
            double beta = (rzn - dot(n, r, zo)) / rz;
            rz = rzn;
            for (size_t c = 0; c < n; c++) d[c] = z[c] + beta * d[c];
        }
    }
    if (!ok && it <= max_it) {
        orc_residual(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, b, p, r);
        ok = norm2(n, r) / nb <= tol;
    }
    orc_remove_mean(n, label, ncomp, p);
    free(label); free(b); free(r); free(z); free(zo); free(d); free(q);
    if (nb == 0.0) return 0;
    return ok ? it : -max_it;
}

/* ------------------------------------------------------------------------- */
/* Jacobi-preconditioned conjugate gradients on -A p = -b (the paper's old     */
/* solver family, Poisson solver section), an algorithm independent of the    */
/* multigrid one.  b is made compatible first; p's mean is removed at the end. */
/* Returns iterations (negative if not converged).                            */
/* ------------------------------------------------------------------------- */
int orc_cg_solve(int nx, int ny, int nz, double h, const double *bx, const double *by, const double *bz,
                 const double *b_in, double *p, double tol, int max_it)
{
    size_t n = (size_t)nx * ny * nz;
    int *label = (int *)malloc(n * sizeof(int));
    int ncomp = orc_components(nx, ny, nz, bx, by, bz, label);
    double *b = dalloc(n), *r = dalloc(n), *z = dalloc(n), *d = dalloc(n), *q = dalloc(n), *dinv = dalloc(n);
    memcpy(b, b_in, n * sizeof(double));
    orc_remove_mean(n, label, ncomp, b);
    orc_diag_inv(nx, ny, nz, bx, by, bz, dinv);
    double h2 = h * h;
    /* r = (-b) - (-A) p = A p - b */
    orc_apply_A(nx, ny, nz, h, bx, by, bz, p, r);
    for (size_t c = 0; c < n; c++) r[c] = r[c] - b[c];
    double nb = norm2(n, b);
    int it = 0, ok = (nb == 0.0);
    if (ok) memset(p, 0, n * sizeof(double));
    double rz = 0.0;
    for (size_t c = 0; c < n; c++) { z[c] = h2 * dinv[c] * r[c]; d[c] = z[c]; rz += r[c] * z[c]; }
    for (it = 1; !ok && it <= max_it; it++) {
        orc_apply_A(nx, ny, nz, h, bx, by, bz, d, q);
        for (size_t c = 0; c < n; c++) q[c] = -q[c];          /* q = (-A) d */
        double dq = 0.0;
        for (size_t c = 0; c < n; c++) dq += d[c] * q[c];
        double alpha = rz / dq;
        for (size_t c = 0; c < n; c++) { p[c] += alpha * d[c]; r[c] -= alpha * q[c]; }
        if (norm2(n, r) / nb <= tol) { ok = 1; break; }
        double rz2 = 0.0;
        for (size_t c = 0; c < n; c++) { z[c] = h2 * dinv[c] * r[c]; rz2 += r[c] * z[c]; }
        double beta = rz2 / rz;
        rz = rz2;
        for (size_t c = 0; c < n; c++) d[c] = z[c] + beta * d[c];
    }
    orc_remove_mean(n, label, ncomp, p);
    free(label); free(b); free(r); free(z); free(d); free(q); free(dinv);
    if (nb == 0.0) return 0;
    return ok ? it : -max_it;
}

/* ------------------------------------------------------------------------- */
/* Projection (Eq. poisson1, Eq. runge1 with the static-body form of          */
/* Eq. integral2): b = D u* / dt, where D sums the outward fluxes through the */
/* open faces of a cell (a closed face carries the body velocity, 0 here):    */
/*   (D u)_c = h^-1 sum_axis (open(f_hi) u_hi - open(f_lo) u_lo)             */
/* A face is open iff beta_f > 0.                                             */
/* ------------------------------------------------------------------------- */
void orc_divergence(int nx, int ny, int nz, double h, double dt, const double *bx, const double *by,
                    const double *bz, const double *ux, const double *uy, const double *uz, double *b)
{
    double s = 1.0 / (dt * h);
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = IX(i, j, k);
                double d = 0.0;
                if (i < nx - 1 && bx[IX(i + 1, j, k)] > 0.0) d += ux[IX(i + 1, j, k)];
                if (bx[c] > 0.0) d -= ux[c];
                if (j < ny - 1 && by[IX(i, j + 1, k)] > 0.0) d += uy[IX(i, j + 1, k)];
                if (by[c] > 0.0) d -= uy[c];
                if (k < nz - 1 && bz[IX(i, j, k + 1)] > 0.0) d += uz[IX(i, j, k + 1)];
                if (bz[c] > 0.0) d -= uz[c];
                b[c] = s * d;
            }
}

/* ------------------------------------------------------------------------- */
/* Fractional face areas (Body Boundary Conditions section, Eq. integral2).  */
/* The body is the region psi <= 0 of a signed distance psi given at the     */
/* grid's nodes ((nz+1) x (ny+1) x (nx+1), node (i,j,k) at (i h, j h, k h)).  */
/* The paper takes the area fractions from a cited reference; the reading    */
/* here: a face is split into four triangles about its centre, psi at the    */
/* centre is the mean of the four corners, psi is linear on each triangle,   */
/* and the face's open fraction is the mean of the triangles' fractions where */
/* psi > 0.  Each triangle's fraction has a closed form: with one corner     */
/* value f > 0 and the other two g1, g2 <= 0 it is f^2 / ((f-g1)(f-g2));     */
/* with two corners > 0 and one value g <= 0 it is 1 - g^2/((g-f1)(g-f2)).   */
/* ------------------------------------------------------------------------- */
static double tri_open(double a, double b, double c)
{
    int pa = a > 0.0, pb = b > 0.0, pc = c > 0.0;
    int np = pa + pb + pc;
    if (np == 0) return 0.0;
    if (np == 3) return 1.0;
    if (np == 1) {
        double f = pa ? a : (pb ? b : c);
        double g1 = pa ? b : a, g2 = pc ? b : c;   /* the two others */
        return (f * f) / ((f - g1) * (f - g2));
    }
    /* np == 2: one corner g <= 0 */
    double g = !pa ? a : (!pb ? b : c);
    double f1 = !pa ? b : a, f2 = !pc ? b : c;
    return 1.0 - (g * g) / ((g - f1) * (g - f2));
}

/* corners in cyclic order around the face: f00, f10, f11, f01 */
double orc_face_open(double f00, double f10, double f01, double f11)
{
    double fc = ((f00 + f10) + (f01 + f11)) * 0.25;
    double t0 = tri_open(f00, f10, fc), t1 = tri_open(f10, f11, fc);
    double t2 = tri_open(f11, f01, fc), t3 = tri_open(f01, f00, fc);
    return (((t0 + t1) + t2) + t3) * 0.25;
}

/* open fractions of the low faces; wall faces (i = 0, j = 0, k = 0) are 0 */
void orc_face_areas(int nx, int ny, int nz, const double *psi, double *ax, double *ay, double *az)
{
    const size_t NX = (size_t)nx + 1, NXY = NX * ((size_t)ny + 1);
#define PSI(i, j, k) psi[(size_t)(k) * NXY + (size_t)(j) * NX + (size_t)(i)]
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = IX(i, j, k);
                /* x face at x = i h: corners over (y, z) */
                ax[c] = i == 0 ? 0.0 : orc_face_open(PSI(i, j, k), PSI(i, j + 1, k), PSI(i, j, k + 1), PSI(i, j + 1, k + 1));
                /* y face at y = j h: corners over (x, z) */
                ay[c] = j == 0 ? 0.0 : orc_face_open(PSI(i, j, k), PSI(i + 1, j, k), PSI(i, j, k + 1), PSI(i + 1, j, k + 1));
                /* z face at z = k h: corners over (x, y) */
                az[c] = k == 0 ? 0.0 : orc_face_open(PSI(i, j, k), PSI(i + 1, j, k), PSI(i, j + 1, k), PSI(i + 1, j + 1, k));
            }
#undef PSI
}

/* Right-hand side of Eq. integral2 with fractional areas: b = D_a (u - v) / dt,
 *   (D_a u)_c = h^-1 sum over the faces of c with a > 0 of +-a_f u_f   (x+, x-, y+, y-, z+, z-)
 * with v the body velocity at the face centres (NULL: a static body).  For a velocity field of
 * zero divergence, the flux of v through the body surface in a cut cell equals minus its flux
 * through the open parts of the cell's faces (Gauss's theorem), so subtracting v on the open
 * faces adds the body term of Eq. integral2; in cells the body does not cut it adds the discrete
 * divergence of v, zero for the rigid motions (linear in x) it stands for. */
void orc_divergence_area(int nx, int ny, int nz, double h, double dt, const double *ax, const double *ay,
                         const double *az, const double *ux, const double *uy, const double *uz, const double *vx,
                         const double *vy, const double *vz, double *b)
{
    double s = 1.0 / (dt * h);
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = IX(i, j, k);
                double d = 0.0;
                size_t f;
#define FLUX(arr_a, arr_u, arr_v, idx) ((arr_a)[idx] * ((arr_u)[idx] - ((arr_v) ? (arr_v)[idx] : 0.0)))
                if (i < nx - 1 && ax[f = IX(i + 1, j, k)] > 0.0) d += FLUX(ax, ux, vx, f);
                if (ax[c] > 0.0) d -= FLUX(ax, ux, vx, c);
                if (j < ny - 1 && ay[f = IX(i, j + 1, k)] > 0.0) d += FLUX(ay, uy, vy, f);
                if (ay[c] > 0.0) d -= FLUX(ay, uy, vy, c);
                if (k < nz - 1 && az[f = IX(i, j, k + 1)] > 0.0) d += FLUX(az, uz, vz, f);
                if (az[c] > 0.0) d -= FLUX(az, uz, vz, c);
#undef FLUX
                b[c] = s * d;
            }
}

/* ------------------------------------------------------------------------- */
/* Stretched grids (grids stretched along the Cartesian axes, Numerical      */
/* efficiency / parallel-computing sections).  Cell widths hx[i], hy[j],      */
/* hz[k].  Multiplying Eq. integral2 by the cell volume puts it on the index  */
/* grid (unit spacing) with, for each low face,                               */
/*   beta_idx = beta / d   (d: distance between the two cell centres)         */
/*   area     = (the face's two widths) * open fraction (1 without a body)    */
/* so that the operator is area * beta_idx (the product moved to the coarse   */
/* grids), the divergence sum(+-area u)/dt is the cell volume times b, and    */
/* the correction u - dt beta_idx (p_R - p_L) is the physical one.  Wall      */
/* faces: area 0, beta_idx 0.                                                 */
/* ------------------------------------------------------------------------- */
void orc_stretched_metrics(int nx, int ny, int nz, const double *hx, const double *hy, const double *hz,
                           const double *bx, const double *by, const double *bz, const double *fx, const double *fy,
                           const double *fz, double *obx, double *oby, double *obz, double *ax, double *ay, double *az)
{
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = IX(i, j, k);
                if (i == 0) { obx[c] = 0.0; ax[c] = 0.0; }
                else {
                    double d = 0.5 * (hx[i - 1] + hx[i]);
                    obx[c] = bx[c] / d;
                    ax[c] = (hy[j] * hz[k]) * (fx ? fx[c] : 1.0);
                }
                if (j == 0) { oby[c] = 0.0; ay[c] = 0.0; }
                else {
                    double d = 0.5 * (hy[j - 1] + hy[j]);
                    oby[c] = by[c] / d;
                    ay[c] = (hx[i] * hz[k]) * (fy ? fy[c] : 1.0);
                }
                if (k == 0) { obz[c] = 0.0; az[c] = 0.0; }
                else {
                    double d = 0.5 * (hz[k - 1] + hz[k]);
                    obz[c] = bz[c] / d;
                    az[c] = (hx[i] * hy[j]) * (fz ? fz[c] : 1.0);
                }
            }
}

/* ------------------------------------------------------------------------- */
/* VOF operator of the time integration (Eq. vof with Q = 0, Numerical Time  */
/* Integration section): VOF(u, phi, dt) = dt * h^-1 * sum over the open     */
/* faces of the cell of +-u_f phi_up(f), phi_up the value of the cell the    */
/* face velocity comes from (first-order upwind, unsplit); closed faces and  */
/* walls carry no flux.  The paper cites its VOF scheme; this is the simplest */
/* conservative one.  Face order x+, x-, y+, y-, z+, z-.                      */
/* ------------------------------------------------------------------------- */
void orc_vof_upwind(int nx, int ny, int nz, double h, double dt, const double *bx, const double *by, const double *bz,
                    const double *ux, const double *uy, const double *uz, const double *phi, double *out)
{
    double s = dt / h;
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = IX(i, j, k), f;
                double d = 0.0;
#define UPW(u, lo, hi) ((u) > 0.0 ? (u) * phi[lo] : (u) * phi[hi])
                if (i < nx - 1 && bx[f = IX(i + 1, j, k)] > 0.0) d += UPW(ux[f], c, f);
                if (bx[c] > 0.0) d -= UPW(ux[c], IX(i - 1, j, k), c);
                if (j < ny - 1 && by[f = IX(i, j + 1, k)] > 0.0) d += UPW(uy[f], c, f);
                if (by[c] > 0.0) d -= UPW(uy[c], IX(i, j - 1, k), c);
                if (k < nz - 1 && bz[f = IX(i, j, k + 1)] > 0.0) d += UPW(uz[f], c, f);
                if (bz[c] > 0.0) d -= UPW(uz[c], IX(i, j, k - 1), c);
#undef UPW
                out[c] = s * d;
            }
}

/* u_f = u*_f - dt beta_f (p_R - p_L) / h on open faces; closed faces keep u*. */
void orc_correct(int nx, int ny, int nz, double h, double dt, const double *bx, const double *by,
                 const double *bz, const double *p, const double *ux0, const double *uy0,
                 const double *uz0, double *ux, double *uy, double *uz)
{
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = IX(i, j, k);
                ux[c] = ux0[c];
                uy[c] = uy0[c];
                uz[c] = uz0[c];
                if (bx[c] > 0.0) ux[c] = ux0[c] - dt * bx[c] * (p[c] - p[IX(i - 1, j, k)]) / h;
                if (by[c] > 0.0) uy[c] = uy0[c] - dt * by[c] * (p[c] - p[IX(i, j - 1, k)]) / h;
                if (bz[c] > 0.0) uz[c] = uz0[c] - dt * bz[c] * (p[c] - p[IX(i, j, k - 1)]) / h;
            }
}

/* ------------------------------------------------------------------------- */
/* Adjoint pieces (derived from the projection u = u* - B G A^+ D u*, with    */
/* B = diag(beta), G = -D^T on open faces, A = D B G):                        */
/*   grad_u* = w - G q,       A q = D (beta w)                                */
/*   grad_beta_f = dt (G p)_f ((G q)_f - w_f)          (open faces; 0 else)   */
/*   grad_phi_c  = -(1 - lam)/2 sum_{open f of c} beta_f^2 grad_beta_f         */
/* ------------------------------------------------------------------------- */
void orc_face_scale(size_t n, const double *bx, const double *by, const double *bz, const double *wx,
                    const double *wy, const double *wz, double *ox, double *oy, double *oz)
{
    for (size_t c = 0; c < n; c++) { ox[c] = bx[c] * wx[c]; oy[c] = by[c] * wy[c]; oz[c] = bz[c] * wz[c]; }
}

/* (G q) on open faces, 0 on closed faces */
void orc_gradient(int nx, int ny, int nz, double h, const double *bx, const double *by, const double *bz,
                  const double *q, double *gx, double *gy, double *gz)
{
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = IX(i, j, k);
                gx[c] = bx[c] > 0.0 ? (q[c] - q[IX(i - 1, j, k)]) / h : 0.0;
                gy[c] = by[c] > 0.0 ? (q[c] - q[IX(i, j - 1, k)]) / h : 0.0;
                gz[c] = bz[c] > 0.0 ? (q[c] - q[IX(i, j, k - 1)]) / h : 0.0;
            }
}

void orc_phi_grad(int nx, int ny, int nz, double lam, const double *bx, const double *by, const double *bz,
                  const double *gbx, const double *gby, const double *gbz, double *gphi)
{
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = IX(i, j, k);
                double s = 0.0;
                /* the six faces of c; d beta_f / d rho_c = -beta_f^2 / 2 */
                s += bx[c] * bx[c] * gbx[c];
                if (i < nx - 1) s += bx[IX(i + 1, j, k)] * bx[IX(i + 1, j, k)] * gbx[IX(i + 1, j, k)];
                s += by[c] * by[c] * gby[c];
                if (j < ny - 1) s += by[IX(i, j + 1, k)] * by[IX(i, j + 1, k)] * gby[IX(i, j + 1, k)];
                s += bz[c] * bz[c] * gbz[c];
                if (k < nz - 1) s += bz[IX(i, j, k + 1)] * bz[IX(i, j, k + 1)] * gbz[IX(i, j, k + 1)];
                gphi[c] = -0.5 * (1.0 - lam) * s;
            }
}

/* ------------------------------------------------------------------------- */
/* Momentum right-hand side R_i of Eq. navi without the pressure gradient and */
/* the sub-grid stress (Numerical Time Integration section: R_i holds the     */
/* convective, viscous and body-force terms):                                  */
/*   R_i = -d/dx_j (u_j u_i) + 1/(rho Re) d/dx_j (2 mu S_ij) - delta_i3 g      */
/* with S_ij = (du_i/dx_j + du_j/dx_i)/2, mu = mu_air + (mu_water - mu_air)   */
/* phi (Eq. density, H(phi) = phi) and 1/rho on a face = beta_f (the face     */
/* coefficient 2/(rho_L + rho_R)).  The paper does not give the discrete      */
/* operators; this is the second-order central, conservative MAC form:        */
/*   - u_i u_i at cell centres from the mean of the cell's two i-faces;       */
/*     u_j u_i (j != i) at the cell edges from the mean of the two j-faces    */
/*     and the mean of the two i-faces that meet there;                       */
/*   - 2 mu S_ii at cell centres (mu of the cell), 2 mu S_ij at the edges     */
/*     (mu = mean of the four cells around the edge, summed in cell-index     */
/*     order);                                                                */
/*   - each divergence the difference of the two values that bracket the     */
/*     face, over h.                                                          */
/* Walls are free-slip: normal velocity 0 (the stored wall face, or the high  */
/* wall, 0), tangential velocity mirrored into the ghost row, so no momentum  */
/* flux and no shear cross a wall.  Closed faces (walls, faces at a solid)    */
/* enter the stencils with their stored velocity and get R = 0.               */
/* Sums in the order written, separately rounded.                             */
/* ------------------------------------------------------------------------- */
static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* face velocity of axis a at face index (i,j,k) along its own axis in [0, n_a]
   (n_a: the high wall, 0); the other two indices mirrored into the domain */
static double fvel(const double *u, int a, int i, int j, int k, int nx, int ny, int nz)
{
    if ((a == 0 && i >= nx) || (a == 1 && j >= ny) || (a == 2 && k >= nz)) return 0.0;
    i = clampi(i, 0, nx - 1);
    j = clampi(j, 0, ny - 1);
    k = clampi(k, 0, nz - 1);
    return u[IX(i, j, k)];
}

static double cmu(const double *phi, double mua, double dmu, int i, int j, int k, int nx, int ny, int nz)
{
    i = clampi(i, 0, nx - 1);
    j = clampi(j, 0, ny - 1);
    k = clampi(k, 0, nz - 1);
    return mua + dmu * phi[IX(i, j, k)];
}

void orc_momentum_rhs(int nx, int ny, int nz, double h, const double *phi, double mu_air, double mu_water,
                      double inv_re, double g, int convect, const double *bx, const double *by, const double *bz,
                      const double *ux, const double *uy, const double *uz, double *rx, double *ry, double *rz)
{
    const double ih = 1.0 / h, dmu = mu_water - mu_air;
    const double *U[3] = {ux, uy, uz};
    const double *B[3] = {bx, by, bz};
    double *R[3] = {rx, ry, rz};
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const size_t c = IX(i, j, k);
                for (int a = 0; a < 3; a++) {
                    if (!(B[a][c] > 0.0)) {
                        R[a][c] = 0.0;
                        continue;
                    }
                    /* unit offsets of the face's own axis a and of the two others b, d */
                    int o[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
                    const int *ea = o[a];
                    double conv = 0.0, visc = 0.0;
                    /* normal part: cells (face - 1) and (face) along a */
                    {
                        const double um = fvel(U[a], a, i - ea[0], j - ea[1], k - ea[2], nx, ny, nz);
                        const double u0 = fvel(U[a], a, i, j, k, nx, ny, nz);
                        const double up = fvel(U[a], a, i + ea[0], j + ea[1], k + ea[2], nx, ny, nz);
                        const double cm = 0.5 * (um + u0), cp = 0.5 * (u0 + up);
                        conv = (cp * cp - cm * cm) * ih;
                        const double mum = cmu(phi, mu_air, dmu, i - ea[0], j - ea[1], k - ea[2], nx, ny, nz);
                        const double mup = cmu(phi, mu_air, dmu, i, j, k, nx, ny, nz);
                        const double tp = 2.0 * mup * ((up - u0) * ih);
                        const double tm = 2.0 * mum * ((u0 - um) * ih);
                        visc = tp - tm;
                    }
                    /* the two tangential directions b in the order x, y, z (skipping a) */
                    for (int b = 0; b < 3; b++) {
                        if (b == a) continue;
                        const int *eb = o[b];
                        /* edges at the low (index of the face) and high (+1 along b) side */
                        double fl[2], tl[2];
                        for (int side = 0; side < 2; side++) {
                            /* edge between faces of axis a at b-index (n-1, n), n = face's b-index + side */
                            const int si = i + side * eb[0], sj = j + side * eb[1], sk = k + side * eb[2];
                            /* u_a on the two a-faces meeting at the edge: b-index n-1 and n */
                            const double ua0 = fvel(U[a], a, si - eb[0], sj - eb[1], sk - eb[2], nx, ny, nz);
                            const double ua1 = fvel(U[a], a, si, sj, sk, nx, ny, nz);
                            /* u_b on the two b-faces meeting at the edge: a-index (face - 1) and face */
                            const double ub0 = fvel(U[b], b, si - ea[0], sj - ea[1], sk - ea[2], nx, ny, nz);
                            const double ub1 = fvel(U[b], b, si, sj, sk, nx, ny, nz);
                            const double vb = 0.5 * (ub0 + ub1), va = 0.5 * (ua0 + ua1);
                            fl[side] = vb * va;
                            /* mu at the edge: mean of the four cells (a-index face-1, face) x (b-index n-1, n) */
                            const double m00 = cmu(phi, mu_air, dmu, si - ea[0] - eb[0], sj - ea[1] - eb[1],
                                                   sk - ea[2] - eb[2], nx, ny, nz);
                            const double m10 = cmu(phi, mu_air, dmu, si - eb[0], sj - eb[1], sk - eb[2], nx, ny, nz);
                            const double m01 = cmu(phi, mu_air, dmu, si - ea[0], sj - ea[1], sk - ea[2], nx, ny, nz);
                            const double m11 = cmu(phi, mu_air, dmu, si, sj, sk, nx, ny, nz);
                            /* the four cells summed in the order of their cell index (the lower
                               of the two axes varies fastest), the same for all four faces that
                               share the edge */
                            const double me = a < b ? 0.25 * (((m00 + m10) + m01) + m11)
                                                    : 0.25 * (((m00 + m01) + m10) + m11);
                            tl[side] = me * ((ua1 - ua0) * ih + (ub1 - ub0) * ih);
                        }
                        conv = conv + (fl[1] - fl[0]) * ih;
                        visc = visc + (tl[1] - tl[0]);
                    }
                    double r = 0.0;
                    if (convect) r = -conv;
                    r = r + (inv_re * B[a][c]) * (visc * ih);
                    if (a == 2) r = r - g;
                    R[a][c] = r;
                }
            }
}
