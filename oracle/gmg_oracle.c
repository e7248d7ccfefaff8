/*
 * gmg_oracle.c -- plain, slow, single-threaded FP64 reference of the
 * geometric-multigrid pressure-Poisson solve.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker that the CUDA solver is
 * compared against; it shares no code, header, table or helper with the
 * solver, and nothing on the solver's product path may call it.  Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark load it.
 *
 * What it computes (paper: "Scaling WaterLily.jl with MPI and an improved
 * geometric multigrid solver"):
 *   - Sec. 3 (intro): GMG = smoother for high-frequency error plus coarse-grid
 *     correction (CGC) for low-frequency error, iterated as V-cycles;
 *   - Sec. 3.1: red-black Gauss-Seidel smoother, under-relaxed by a factor
 *     omega that adapts to residual growth or decay after each V-cycle so that
 *     the residual decays monotonically;
 *   - Sec. 3.2: isotropic coarsening (all axes halved together, depth limited
 *     by the smallest axis) versus anisotropic coarsening (each axis halved
 *     independently).
 * The paper does not write the operator, the transfer stencils, the coarse
 * operator, the sweep counts or the omega rule; the readings taken here are:
 *   C1 operator  (A p)_I = sum_d [ b_d(I+e_d)(p(I+e_d) - p_I) + b_d(I)(p(I-e_d) - p_I) ]
 *                in grid units; Neumann axes have zero boundary faces,
 *                periodic axes wrap.
 *   C2 sweep     red cells ((i+j+k) even) then black; each cell
 *                p <- (1-w) p + w (sum_f b_f p_nb - b) / sum_f b_f; cells with
 *                sum_f b_f = 0 are skipped.
 *   C3 schedule  aniso: axis d halves while n_d is even and n_d/2 >= n_min (on
 *                a periodic axis n_d/2 must stay even); iso: all axes halve
 *                together while every axis qualifies.  An axis of length 1
 *                (a 2D problem, Fig. 2) takes no part: it never halves, and
 *                iso halves the other axes together.
 *   C4 coarse b  finite-volume rediscretisation: coarse face = (1/c_d) times
 *                the sum of the fine faces that make it up; or, as the option
 *                for study (coarse_op 1), the Galerkin operator R A P with
 *                piecewise-constant P and R = P^T, whose coarse face is that
 *                sum without the 1/c_d.
 *   C5 omega     w0 = 1; after each V-cycle rho = |r_k| / |r_prev|; rho < 1
 *                accepts and sets w = min(1, grow w); otherwise the cycle is
 *                rejected (iterate restored), w = max(w_min, shrink w), and a
 *                rejection at w_min is divergence.
 *   C6 V-cycle   V(nu1, nu2), zero guess on coarse levels, restriction = sum
 *                over children, prolongation = piecewise-constant injection,
 *                nu_c sweeps on the coarsest level after projecting its
 *                right-hand side to zero mean over active cells; or, as the
 *                option for study (coarse_mode 1), the exact minimum-norm
 *                solve p = A^+ b of the coarsest level, A^+ the Moore-Penrose
 *                pseudo-inverse of its operator.
 *   C7 stop      |b - A p|_2 / |b|_2 <= tol, checked after each V-cycle.
 *   C8 gauge     at exit p -= mean over active cells; inactive cells p = 0.
 *
 * Layout: arrays are [nz][ny][nx], x fastest; b_d[I] is the coefficient on
 * the lower d-face of cell I.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_NOT_CONVERGED 3
#define OR_DIVERGED 4
#define OR_MAX_LEVELS 32

typedef struct {
    int n[3];          /* nx, ny, nz */
    int per[3];        /* periodic flags */
} grid_t;

static long cells(const grid_t* g) { return (long)g->n[0] * g->n[1] * g->n[2]; }

static long idx(const grid_t* g, int i, int j, int k)
{
    return ((long)k * g->n[1] + j) * g->n[0] + i;
}

/* neighbour of cell (c[0],c[1],c[2]) one step along axis d in direction s
 * (+1 / -1); returns 0 if it does not exist (Neumann boundary). */
static int neighbour(const grid_t* g, const int c[3], int d, int s, int out[3])
{
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2];
    out[d] += s;
    if (out[d] < 0 || out[d] >= g->n[d]) {
        if (!g->per[d]) return 0;
        out[d] = (out[d] + g->n[d]) % g->n[d];
    }
    return 1;
}

/* coefficient of the face between cell c and its neighbour along d, s */
static double face(const grid_t* g, const double* const beta[3], const int c[3], int d, int s)
{
    int f[3] = {c[0], c[1], c[2]};
    if (s > 0) {                       /* upper face = lower face of the next cell */
        f[d] += 1;
        if (f[d] == g->n[d]) {
            if (!g->per[d]) return 0.0;
            f[d] = 0;
        }
    } else if (c[d] == 0 && !g->per[d]) {
        return 0.0;                    /* lower wall face */
    }
    return beta[d][idx(g, f[0], f[1], f[2])];
}

static double diag(const grid_t* g, const double* const beta[3], const int c[3])
{
    double s = 0.0;
    for (int d = 0; d < 3; ++d) s += face(g, beta, c, d, -1) + face(g, beta, c, d, +1);
    return s;
}

/* sum over faces of beta_f * p(neighbour across f) */
static double flux_sum(const grid_t* g, const double* const beta[3], const double* p, const int c[3])
{
    double s = 0.0;
    for (int d = 0; d < 3; ++d)
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            int nb[3];
            if (!neighbour(g, c, d, sgn, nb)) continue;
            double bf = face(g, beta, c, d, sgn);
            if (bf != 0.0) s += bf * p[idx(g, nb[0], nb[1], nb[2])];
        }
    return s;
}

/* C1: (A p)_I */
static void apply_A(const grid_t* g, const double* const beta[3], const double* p, double* out)
{
    int c[3];
    for (c[2] = 0; c[2] < g->n[2]; ++c[2])
        for (c[1] = 0; c[1] < g->n[1]; ++c[1])
            for (c[0] = 0; c[0] < g->n[0]; ++c[0]) {
                long I = idx(g, c[0], c[1], c[2]);
                out[I] = flux_sum(g, beta, p, c) - diag(g, beta, c) * p[I];
            }
}

static void residual(const grid_t* g, const double* const beta[3], const double* b,
                     const double* p, double* r)
{
    apply_A(g, beta, p, r);
    long N = cells(g);
    for (long I = 0; I < N; ++I) r[I] = b[I] - r[I];
}

static double norm2(const double* v, long N)
{
    double s = 0.0;
    for (long I = 0; I < N; ++I) s += v[I] * v[I];
    return sqrt(s);
}

/* C2: one colour of the under-relaxed Gauss-Seidel sweep, in place */
static void half_sweep(const grid_t* g, const double* const beta[3], const double* b,
                       double* p, double omega, int colour)
{
    int c[3];
    for (c[2] = 0; c[2] < g->n[2]; ++c[2])
        for (c[1] = 0; c[1] < g->n[1]; ++c[1])
            for (c[0] = 0; c[0] < g->n[0]; ++c[0]) {
                if (((c[0] + c[1] + c[2]) & 1) != colour) continue;
                double dg = diag(g, beta, c);
                if (dg == 0.0) continue;
                long I = idx(g, c[0], c[1], c[2]);
                double gs = (flux_sum(g, beta, p, c) - b[I]) / dg;
                p[I] = (1.0 - omega) * p[I] + omega * gs;
            }
}

static void sweep(const grid_t* g, const double* const beta[3], const double* b, double* p, double omega)
{
    half_sweep(g, beta, b, p, omega, 0);
    half_sweep(g, beta, b, p, omega, 1);
}

/* mean over active cells (sum of faces > 0) and their count */
static double active_mean(const grid_t* g, const double* const beta[3], const double* v, long* count)
{
    int c[3];
    double s = 0.0;
    long n = 0;
    for (c[2] = 0; c[2] < g->n[2]; ++c[2])
        for (c[1] = 0; c[1] < g->n[1]; ++c[1])
            for (c[0] = 0; c[0] < g->n[0]; ++c[0])
                if (diag(g, beta, c) > 0.0) {
                    s += v[idx(g, c[0], c[1], c[2])];
                    ++n;
                }
    if (count) *count = n;
    return n ? s / (double)n : 0.0;
}

/* v -= mean over active cells; inactive cells set to 0 */
static void project_active(const grid_t* g, const double* const beta[3], double* v)
{
    double m = active_mean(g, beta, v, NULL);
    int c[3];
    for (c[2] = 0; c[2] < g->n[2]; ++c[2])
        for (c[1] = 0; c[1] < g->n[1]; ++c[1])
            for (c[0] = 0; c[0] < g->n[0]; ++c[0]) {
                long I = idx(g, c[0], c[1], c[2]);
                v[I] = diag(g, beta, c) > 0.0 ? v[I] - m : 0.0;
            }
}

/* C3: the coarsening factor of each axis from a level of size n */
static int axis_halves(int n, int periodic, int n_min)
{
    if (n % 2) return 0;
    if (n / 2 < n_min) return 0;
    if (periodic && (n / 2) % 2) return 0;
    return 1;
}

static int schedule(const int n0[3], const int per[3], int aniso, int n_min, int max_levels,
                    int dims[][3], int fac[][3])
{
    int L = 0;
    int n[3] = {n0[0], n0[1], n0[2]};
    for (;;) {
        dims[L][0] = n[0]; dims[L][1] = n[1]; dims[L][2] = n[2];
        fac[L][0] = fac[L][1] = fac[L][2] = 1;
        ++L;
        if (L >= max_levels) break;
        int h[3], any = 0, all = 1;
        for (int d = 0; d < 3; ++d) {
            h[d] = axis_halves(n[d], per[d], n_min);
            any |= h[d];
            if (n[d] > 1) all &= h[d];   /* a length-1 axis is not part of the grid */
        }
        if (!any || (!aniso && !all)) break;
        for (int d = 0; d < 3; ++d) {
            fac[L - 1][d] = h[d] ? 2 : 1;
            n[d] /= fac[L - 1][d];
        }
    }
    return L;
}

/* C4: coarse face coefficients by finite-volume rediscretisation (galerkin 0),
 * or those of R A P with piecewise-constant P (galerkin 1: no 1/c_d) */
static void coarsen_beta(const grid_t* fg, const double* const fb[3], const int c[3],
                         const grid_t* cg, double* const cb[3], int galerkin)
{
    int J[3];
    for (int d = 0; d < 3; ++d) {
        for (J[2] = 0; J[2] < cg->n[2]; ++J[2])
            for (J[1] = 0; J[1] < cg->n[1]; ++J[1])
                for (J[0] = 0; J[0] < cg->n[0]; ++J[0]) {
                    /* fine faces on the plane I_d = c_d J_d spanning the coarse face */
                    int lo[3], hi[3];
                    for (int e = 0; e < 3; ++e) {
                        lo[e] = c[e] * J[e];
                        hi[e] = (e == d) ? lo[e] + 1 : lo[e] + c[e];
                    }
                    double s = 0.0;
                    int I[3];
                    for (I[2] = lo[2]; I[2] < hi[2]; ++I[2])
                        for (I[1] = lo[1]; I[1] < hi[1]; ++I[1])
                            for (I[0] = lo[0]; I[0] < hi[0]; ++I[0])
                                s += fb[d][idx(fg, I[0], I[1], I[2])];
                    cb[d][idx(cg, J[0], J[1], J[2])] = galerkin ? s : s / (double)c[d];
                }
    }
}

/* C6: b_c[J] = sum over the children of J of r */
static void restrict_sum(const grid_t* fg, const double* r, const int c[3], const grid_t* cg, double* bc)
{
    memset(bc, 0, sizeof(double) * (size_t)cells(cg));
    int I[3];
    for (I[2] = 0; I[2] < fg->n[2]; ++I[2])
        for (I[1] = 0; I[1] < fg->n[1]; ++I[1])
            for (I[0] = 0; I[0] < fg->n[0]; ++I[0])
                bc[idx(cg, I[0] / c[0], I[1] / c[1], I[2] / c[2])] += r[idx(fg, I[0], I[1], I[2])];
}

/* C6: p[I] += e[floor(I / c)] */
static void prolong_add(const grid_t* fg, double* p, const int c[3], const grid_t* cg, const double* e)
{
    int I[3];
    for (I[2] = 0; I[2] < fg->n[2]; ++I[2])
        for (I[1] = 0; I[1] < fg->n[1]; ++I[1])
            for (I[0] = 0; I[0] < fg->n[0]; ++I[0])
                p[idx(fg, I[0], I[1], I[2])] += e[idx(cg, I[0] / c[0], I[1] / c[1], I[2] / c[2])];
}

typedef struct {
    int coarsen;        /* 0 iso, 1 aniso */
    int n_min;
    int nu1, nu2, nu_c;
    int max_cycles;
    double omega0, omega_min, shrink, grow;
    int coarse_mode;    /* 0: nu_c sweeps on the coarsest level; 1: minimum-norm dense solve */
    int coarse_op;      /* 0: finite-volume coarse coefficients; 1: Galerkin R A P (C4) */
} or_options;

/* ------------------------------------------------------------------------ */
/* C6 option: the coarsest level solved exactly in the least-squares,        */
/* minimum-norm sense, p = A^+ b.  A^+ = V diag(1/lambda) V^T over the        */
/* eigenpairs of the symmetric operator with |lambda| above a relative        */
/* threshold (the null space -- constants per connected component of the      */
/* cells -- gets 0).  Eigenpairs by the cyclic Jacobi method (Golub and Van   */
/* Loan, Matrix Computations, Sec. 8.5): rotations in every (p, q) plane      */
/* until the off-diagonal part is negligible.                                 */
/* ------------------------------------------------------------------------ */

/* dense operator of one grid, column j = A e_j (n x n, row-major) */
static void dense_A(const grid_t* g, const double* const beta[3], double* M)
{
    long n = cells(g);
    double* e = calloc((size_t)n, sizeof(double));
    double* col = malloc(sizeof(double) * (size_t)n);
    for (long j = 0; j < n; ++j) {
        e[j] = 1.0;
        apply_A(g, beta, e, col);
        for (long i = 0; i < n; ++i) M[i * n + j] = col[i];
        e[j] = 0.0;
    }
    free(e);
    free(col);
}

/* symmetric eigendecomposition of S (n x n, destroyed: its diagonal ends as the
 * eigenvalues); V receives the eigenvectors as columns */
static void jacobi_eigen(double* S, double* V, long n)
{
    for (long i = 0; i < n; ++i)
        for (long j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (long i = 0; i < n * n; ++i) fro += S[i] * S[i];
    fro = sqrt(fro);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (long p = 0; p < n; ++p)
            for (long q = p + 1; q < n; ++q) off += 2.0 * S[p * n + q] * S[p * n + q];
        if (sqrt(off) <= 1e-15 * fro) break;
        for (long p = 0; p < n; ++p)
            for (long q = p + 1; q < n; ++q) {
                double apq = S[p * n + q];
                if (apq == 0.0) continue;
                /* rotation (c, s) that zeroes S[p][q] (Golub-Van Loan Alg. 8.5.1) */
                double tau = (S[q * n + q] - S[p * n + p]) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                /* S <- J^T S J with J the rotation in the (p, q) plane */
                for (long k = 0; k < n; ++k) {
                    double skp = S[k * n + p], skq = S[k * n + q];
                    S[k * n + p] = c * skp - sn * skq;
                    S[k * n + q] = sn * skp + c * skq;
                }
                for (long k = 0; k < n; ++k) {
                    double spk = S[p * n + k], sqk = S[q * n + k];
                    S[p * n + k] = c * spk - sn * sqk;
                    S[q * n + k] = sn * spk + c * sqk;
                }
                for (long k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - sn * vkq;
                    V[k * n + q] = sn * vkp + c * vkq;
                }
            }
    }
}

/* Moore-Penrose pseudo-inverse of the operator of grid g (n x n, row-major) */
static double* pseudo_inverse(const grid_t* g, const double* const beta[3])
{
    long n = cells(g);
    double* S = malloc(sizeof(double) * (size_t)(n * n));
    double* V = malloc(sizeof(double) * (size_t)(n * n));
    double* P = calloc((size_t)(n * n), sizeof(double));
    dense_A(g, beta, S);
    jacobi_eigen(S, V, n);
    double lmax = 0.0;
    for (long i = 0; i < n; ++i) lmax = fmax(lmax, fabs(S[i * n + i]));
    for (long m = 0; m < n; ++m) {
        double lam = S[m * n + m];
        if (!(fabs(lam) > 1e-10 * lmax)) continue;          /* null space */
        for (long i = 0; i < n; ++i)
            for (long j = 0; j < n; ++j) P[i * n + j] += V[i * n + m] * V[j * n + m] / lam;
    }
    free(S);
    free(V);
    return P;
}

/* p = A^+ b */
static void pinv_apply(const double* P, long n, const double* b, double* p)
{
    for (long i = 0; i < n; ++i) {
        double s = 0.0;
        for (long j = 0; j < n; ++j) s += P[i * n + j] * b[j];
        p[i] = s;
    }
}

typedef struct {
    int levels;
    int dims[OR_MAX_LEVELS][3];
    int fac[OR_MAX_LEVELS][3];
    grid_t g[OR_MAX_LEVELS];
    double* beta[OR_MAX_LEVELS][3];
    double* b[OR_MAX_LEVELS];
    double* p[OR_MAX_LEVELS];
    double* r[OR_MAX_LEVELS];
    double* pinv;       /* coarse_mode 1: A^+ of the coarsest level */
} hierarchy_t;

static void free_hierarchy(hierarchy_t* h)
{
    for (int l = 0; l < h->levels; ++l) {
        for (int d = 0; d < 3; ++d) free(h->beta[l][d]);
        free(h->b[l]); free(h->p[l]); free(h->r[l]);
    }
    free(h->pinv);
}

/* fine coefficients with the wall faces of Neumann axes zeroed, then C4 per level */
static int build_hierarchy(hierarchy_t* h, const int n[3], const int per[3], const or_options* o,
                           const double* bx, const double* by, const double* bz)
{
    memset(h, 0, sizeof(*h));
    h->levels = schedule(n, per, o->coarsen, o->n_min, OR_MAX_LEVELS, h->dims, h->fac);
    for (int l = 0; l < h->levels; ++l) {
        grid_t* g = &h->g[l];
        for (int d = 0; d < 3; ++d) { g->n[d] = h->dims[l][d]; g->per[d] = per[d]; }
        long N = cells(g);
        for (int d = 0; d < 3; ++d) h->beta[l][d] = calloc((size_t)N, sizeof(double));
        h->b[l] = calloc((size_t)N, sizeof(double));
        h->p[l] = calloc((size_t)N, sizeof(double));
        h->r[l] = calloc((size_t)N, sizeof(double));
        if (!h->b[l] || !h->p[l] || !h->r[l] || !h->beta[l][0] || !h->beta[l][1] || !h->beta[l][2]) {
            h->levels = l + 1;
            free_hierarchy(h);
            return OR_ERR_ARG;
        }
    }
    grid_t* g0 = &h->g[0];
    const double* src[3] = {bx, by, bz};
    int c[3];
    for (int d = 0; d < 3; ++d)
        for (c[2] = 0; c[2] < g0->n[2]; ++c[2])
            for (c[1] = 0; c[1] < g0->n[1]; ++c[1])
                for (c[0] = 0; c[0] < g0->n[0]; ++c[0]) {
                    long I = idx(g0, c[0], c[1], c[2]);
                    h->beta[0][d][I] = (c[d] == 0 && !per[d]) ? 0.0 : src[d][I];
                }
    for (int l = 0; l + 1 < h->levels; ++l)
        coarsen_beta(&h->g[l], (const double* const*)h->beta[l], h->fac[l], &h->g[l + 1], h->beta[l + 1],
                     o->coarse_op);
    if (o->coarse_mode == 1) {
        int c = h->levels - 1;
        h->pinv = pseudo_inverse(&h->g[c], (const double* const*)h->beta[c]);
    }
    return OR_OK;
}

/* C6: one V-cycle on level l starting from h->p[l] with right-hand side h->b[l] */
static void vcycle(hierarchy_t* h, int l, const or_options* o, double omega)
{
    const grid_t* g = &h->g[l];
    const double* const* beta = (const double* const*)h->beta[l];
    if (l == h->levels - 1) {
        project_active(g, beta, h->b[l]);
        if (o->coarse_mode == 1)
            pinv_apply(h->pinv, cells(g), h->b[l], h->p[l]);
        else
            for (int s = 0; s < o->nu_c; ++s) sweep(g, beta, h->b[l], h->p[l], omega);
        return;
    }
    for (int s = 0; s < o->nu1; ++s) sweep(g, beta, h->b[l], h->p[l], omega);
    residual(g, beta, h->b[l], h->p[l], h->r[l]);
    restrict_sum(g, h->r[l], h->fac[l], &h->g[l + 1], h->b[l + 1]);
    memset(h->p[l + 1], 0, sizeof(double) * (size_t)cells(&h->g[l + 1]));
    vcycle(h, l + 1, o, omega);
    prolong_add(g, h->p[l], h->fac[l], &h->g[l + 1], h->p[l + 1]);
    for (int s = 0; s < o->nu2; ++s) sweep(g, beta, h->b[l], h->p[l], omega);
}

typedef struct {
    int cycles;         /* V-cycles run, rejected ones included */
    int status;
    int levels;
    double rel_res;     /* |b - A p| / |b| of the returned iterate */
    double omega;       /* relaxation factor after the last cycle */
    double bnorm;
} or_info;

/*
 * Full solve (C5-C8).  b: right-hand side in grid units (not modified).
 * p: initial guess on entry, gauged solution on exit.  history (optional,
 * max_cycles + 1 entries each): relative residual of the accepted iterate
 * after each cycle (entry 0 = initial), omega used by each cycle, and the
 * accept flag of each cycle.
 */
int or_solve(int nx, int ny, int nz, const int* periodic, const or_options* o,
             const double* bx, const double* by, const double* bz,
             const double* b_in, double* p, double tol, or_info* info,
             double* hist_res, double* hist_omega, int* hist_accept)
{
    const int n[3] = {nx, ny, nz};
    const int per[3] = {periodic[0] != 0, periodic[1] != 0, periodic[2] != 0};
    if (nx < 1 || ny < 1 || nz < 1 || !o || !b_in || !p) return OR_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (per[d] && n[d] % 2) return OR_ERR_ARG;
    hierarchy_t h;
    if (build_hierarchy(&h, n, per, o, bx, by, bz) != OR_OK) return OR_ERR_ARG;
    const grid_t* g = &h.g[0];
    const double* const* beta = (const double* const*)h.beta[0];
    long N = cells(g);
    double* b = malloc(sizeof(double) * (size_t)N);
    double* cand = malloc(sizeof(double) * (size_t)N);
    double* r = malloc(sizeof(double) * (size_t)N);
    memcpy(b, b_in, sizeof(double) * (size_t)N);
    project_active(g, beta, b);                  /* compatible right-hand side */
    int c[3];
    for (c[2] = 0; c[2] < g->n[2]; ++c[2])
        for (c[1] = 0; c[1] < g->n[1]; ++c[1])
            for (c[0] = 0; c[0] < g->n[0]; ++c[0])
                if (!(diag(g, beta, c) > 0.0)) p[idx(g, c[0], c[1], c[2])] = 0.0;

    or_info inf = {0, OR_OK, h.levels, 0.0, o->omega0, 0.0};
    double bnorm = norm2(b, N);
    inf.bnorm = bnorm;
    if (bnorm == 0.0) {
        memset(p, 0, sizeof(double) * (size_t)N);
        if (hist_res) hist_res[0] = 0.0;
    } else {
        residual(g, beta, b, p, r);
        double r_prev = norm2(r, N);
        if (hist_res) hist_res[0] = r_prev / bnorm;
        double omega = o->omega0;
        int status = (r_prev / bnorm <= tol) ? OR_OK : OR_NOT_CONVERGED;
        for (int k = 1; k <= o->max_cycles && status == OR_NOT_CONVERGED; ++k) {
            memcpy(cand, p, sizeof(double) * (size_t)N);
            memcpy(h.p[0], cand, sizeof(double) * (size_t)N);
            memcpy(h.b[0], b, sizeof(double) * (size_t)N);
            vcycle(&h, 0, o, omega);
            residual(g, beta, b, h.p[0], r);
            double rk = norm2(r, N);
            int accept = rk < r_prev;            /* NaN rejects */
            if (hist_omega) hist_omega[k - 1] = omega;
            if (hist_accept) hist_accept[k - 1] = accept;
            inf.cycles = k;
            if (accept) {
                memcpy(p, h.p[0], sizeof(double) * (size_t)N);
                r_prev = rk;
                omega = fmin(1.0, o->grow * omega);
            } else {
                if (omega <= o->omega_min) {
                    status = OR_DIVERGED;
                } else {
                    omega = fmax(o->omega_min, o->shrink * omega);
                }
            }
            if (hist_res) hist_res[k] = r_prev / bnorm;
            if (status != OR_DIVERGED && r_prev / bnorm <= tol) status = OR_OK;
        }
        inf.status = status;
        inf.omega = omega;
        inf.rel_res = r_prev / bnorm;
        project_active(g, beta, p);              /* C8 gauge */
    }
    if (info) *info = inf;
    free(b); free(cand); free(r);
    free_hierarchy(&h);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* single steps, exposed so that each can be pinned on its own                 */
/* ------------------------------------------------------------------------ */

int or_apply_A(int nx, int ny, int nz, const int* periodic, const double* bx, const double* by,
               const double* bz, const double* p, double* out)
{
    grid_t g = {{nx, ny, nz}, {periodic[0] != 0, periodic[1] != 0, periodic[2] != 0}};
    const double* beta[3] = {bx, by, bz};
    apply_A(&g, beta, p, out);
    return OR_OK;
}

int or_half_sweep(int nx, int ny, int nz, const int* periodic, const double* bx, const double* by,
                  const double* bz, const double* b, double* p, double omega, int colour)
{
    grid_t g = {{nx, ny, nz}, {periodic[0] != 0, periodic[1] != 0, periodic[2] != 0}};
    const double* beta[3] = {bx, by, bz};
    half_sweep(&g, beta, b, p, omega, colour);
    return OR_OK;
}

int or_sweep(int nx, int ny, int nz, const int* periodic, const double* bx, const double* by,
             const double* bz, const double* b, double* p, double omega)
{
    grid_t g = {{nx, ny, nz}, {periodic[0] != 0, periodic[1] != 0, periodic[2] != 0}};
    const double* beta[3] = {bx, by, bz};
    sweep(&g, beta, b, p, omega);
    return OR_OK;
}

int or_schedule(int nx, int ny, int nz, const int* periodic, int aniso, int n_min,
                int* dims_out, int* fac_out)
{
    const int n[3] = {nx, ny, nz};
    const int per[3] = {periodic[0] != 0, periodic[1] != 0, periodic[2] != 0};
    int dims[OR_MAX_LEVELS][3], fac[OR_MAX_LEVELS][3];
    int L = schedule(n, per, aniso, n_min, OR_MAX_LEVELS, dims, fac);
    memcpy(dims_out, dims, sizeof(int) * 3 * (size_t)L);
    memcpy(fac_out, fac, sizeof(int) * 3 * (size_t)L);
    return L;
}

int or_coarsen_beta(int nx, int ny, int nz, const int* periodic, const int* fac,
                    const double* bx, const double* by, const double* bz,
                    double* cbx, double* cby, double* cbz, int galerkin)
{
    grid_t fg = {{nx, ny, nz}, {periodic[0] != 0, periodic[1] != 0, periodic[2] != 0}};
    grid_t cg = {{nx / fac[0], ny / fac[1], nz / fac[2]}, {fg.per[0], fg.per[1], fg.per[2]}};
    const double* fb[3] = {bx, by, bz};
    double* cb[3] = {cbx, cby, cbz};
    coarsen_beta(&fg, fb, fac, &cg, cb, galerkin);
    return OR_OK;
}

int or_restrict(int nx, int ny, int nz, const int* fac, const double* r, double* bc)
{
    grid_t fg = {{nx, ny, nz}, {0, 0, 0}};
    grid_t cg = {{nx / fac[0], ny / fac[1], nz / fac[2]}, {0, 0, 0}};
    restrict_sum(&fg, r, fac, &cg, bc);
    return OR_OK;
}

int or_prolong_add(int nx, int ny, int nz, const int* fac, const double* e, double* p)
{
    grid_t fg = {{nx, ny, nz}, {0, 0, 0}};
    grid_t cg = {{nx / fac[0], ny / fac[1], nz / fac[2]}, {0, 0, 0}};
    prolong_add(&fg, p, fac, &cg, e);
    return OR_OK;
}

/* one V-cycle from p (in/out) with the given omega, no control logic */
int or_vcycle(int nx, int ny, int nz, const int* periodic, const or_options* o,
              const double* bx, const double* by, const double* bz,
              const double* b, double* p, double omega)
{
    const int n[3] = {nx, ny, nz};
    const int per[3] = {periodic[0] != 0, periodic[1] != 0, periodic[2] != 0};
    hierarchy_t h;
    if (build_hierarchy(&h, n, per, o, bx, by, bz) != OR_OK) return OR_ERR_ARG;
    long N = cells(&h.g[0]);
    memcpy(h.p[0], p, sizeof(double) * (size_t)N);
    memcpy(h.b[0], b, sizeof(double) * (size_t)N);
    vcycle(&h, 0, o, omega);
    memcpy(p, h.p[0], sizeof(double) * (size_t)N);
    free_hierarchy(&h);
    return OR_OK;
}

/* the coarsest-level step of coarse_mode 1 on one grid: p = A^+ b */
int or_pinv_apply(int nx, int ny, int nz, const int* periodic, const double* bx, const double* by,
                  const double* bz, const double* b, double* p)
{
    grid_t g = {{nx, ny, nz}, {periodic[0] != 0, periodic[1] != 0, periodic[2] != 0}};
    const double* beta[3] = {bx, by, bz};
    double* P = pseudo_inverse(&g, beta);
    pinv_apply(P, cells(&g), b, p);
    free(P);
    return OR_OK;
}
