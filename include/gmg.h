/*
 * gmg.h -- C ABI of the GB300 geometric-multigrid pressure-Poisson solver.
 *
 * The problem (the paper's Sec. 3.1 names it: the variable-coefficient Poisson
 * equation of immersed-boundary flows; its Sec. 3 solves it by geometric
 * multigrid) is, on a cell-centred nx x ny x nz grid in grid units,
 *
 *     (A p)_I = sum over the six faces f of cell I of beta_f (p_nb(f) - p_I) = b_I
 *
 * with one coefficient per face.  Solves run V-cycles (Sec. 3) with the
 * adaptive under-relaxed red-black Gauss-Seidel smoother (Sec. 3.1) on an
 * isotropically or anisotropically coarsened hierarchy (Sec. 3.2) until
 * |b - A p|_2 <= tol |b|_2.
 *
 * Layout.  Every grid array is C-contiguous [nz][ny][nx] (x fastest).  bx[I]
 * is the coefficient on the lower x-face of cell I (between I - e_x and I);
 * by, bz likewise.  On a non-periodic (Neumann) axis the lower wall faces are
 * ignored whatever they hold and the upper wall faces do not exist; on a
 * periodic axis the lower face of cell 0 joins it to cell n - 1.
 *
 * Memory.  Unless an entry point says "host", every pointer is CUDA device
 * memory of the device that was current at gmg_create.  The caller owns its
 * arrays; the library copies what it keeps (the coefficients) and owns the
 * multigrid workspace.  All work is ordered on the stream given at creation
 * (a cudaStream_t passed as void*; NULL = the legacy default stream).
 *
 * Errors.  Every call returns a gmg_status.  GMG_ERR_ARG and GMG_ERR_CUDA
 * leave a message for gmg_last_error.  A CUDA error inside a call is reported
 * as GMG_ERR_CUDA and the handle should then be destroyed.
 */
#ifndef GMG_H
#define GMG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GMG_OK = 0,
    GMG_ERR_ARG = 1,            /* bad argument (dimensions, null pointer, option range) */
    GMG_ERR_CUDA = 2,           /* a CUDA call failed */
    GMG_ERR_NOT_CONVERGED = 3,  /* max_cycles reached; p holds the best iterate */
    GMG_ERR_DIVERGED = 4,       /* a cycle grew the residual at omega_min, or omega is not a positive
                                   finite number; p holds the best iterate */
    GMG_ERR_NONFINITE = 5       /* the right-hand side holds NaN or Inf; p is left untouched */
} gmg_status;

enum { GMG_COARSEN_ISO = 0, GMG_COARSEN_ANISO = 1 };

/*
 * Coarsest-level treatment of the V-cycle (Sec. 3: the coarse-grid correction;
 * Sec. 3.2 ties the iso/aniso effect to how well the coarsest level reduces
 * the low frequencies).  SWEEPS: its right-hand side is projected to zero mean
 * over active cells and nu_c red-black sweeps run from zero.  DENSE: after the
 * same projection it is solved exactly in the minimum-norm least-squares
 * sense, p = A^+ b, with the Moore-Penrose pseudo-inverse of the coarsest
 * operator built on the device at gmg_set_coeffs (FP64, about n^3 operations
 * for n coarsest cells; kept in FP32, n^2 floats per problem).  DENSE needs a
 * hierarchy of at least two levels and a coarsest level of at most 1024
 * cells (GMG_ERR_ARG at create otherwise).
 */
enum { GMG_COARSE_SWEEPS = 0, GMG_COARSE_DENSE = 1 };

/*
 * Coarse operator (the paper does not state one).  GMG_COARSE_OP_FV (default):
 * finite-volume rediscretisation, each coarse face coefficient 1/c_d times the
 * sum of the fine faces it covers (c_d = 2 on a coarsened axis, else 1).
 * GMG_COARSE_OP_GALERKIN, for study: the Galerkin operator R A P with
 * piecewise-constant prolongation P and R = P^T, the same sums without the
 * 1/c_d.  On a cell-centred grid that operator over-weights the coarse
 * correction, so the V-cycles converge several times more slowly (the
 * solution is the same).
 */
enum { GMG_COARSE_OP_FV = 0, GMG_COARSE_OP_GALERKIN = 1 };

/*
 * Precision modes.  The FP32 V-cycle levels sum squared residuals in FP32 over
 * a few cells per thread before the FP64 tile partials, so their norms keep
 * full relative precision while per-cell residuals lie between about 1e-19 and
 * 1e19 (squares within FP32's normal range).  The IR modes scale the inner
 * right-hand side to unit norm, and their outer FP64 residual is summed in
 * FP64, so they have no such range limit.
 */
enum {
    GMG_FP32 = 0,       /* FP32 storage and arithmetic throughout */
    GMG_FP32_BF16 = 1,  /* FP32, with BF16 storage of the corrections on levels >= 1 */
    GMG_IR64 = 2,       /* FP64 outer iterative refinement around FP32 (+BF16) V-cycles */
    GMG_IR64_FP32 = 3   /* FP64 outer iterative refinement around FP32 V-cycles */
};

typedef struct {
    int coarsen;        /* GMG_COARSEN_ISO or GMG_COARSEN_ANISO (default ANISO) */
    int n_min;          /* an axis is halved only while n/2 >= n_min (default 4) */
    int nu1, nu2;       /* pre- and post-smoothing sweeps per level (default 2, 2) */
    int nu_c;           /* sweeps on the coarsest level (default 16) */
    int precision;      /* GMG_FP32 ... GMG_IR64_FP32 (default GMG_FP32) */
    int max_cycles;     /* V-cycle limit per solve, rejected cycles included (default 100) */
    double omega0;      /* initial relaxation factor (default 1) */
    double omega_min;   /* floor of the relaxation factor (default 0.25) */
    double shrink;      /* factor applied to omega after a rejected cycle (default 0.7) */
    double grow;        /* factor applied after an accepted cycle, capped at 1 (default 1.1) */
    int use_graph;      /* replay the V-cycle from a captured CUDA graph (default 1) */
    int cycles_per_sync;/* at most this many V-cycles queued between two reads of the status; the solver
                           queues as many as the contraction seen so far predicts (default 8) */
    double ir_inner_rtol; /* IR modes: inner V-cycles stop at this residual reduction (default 1e-4) */
    int autotune;       /* time launch shapes at gmg_set_coeffs and keep the fastest (default 1) */
    int coarse_mode;    /* coarsest level: GMG_COARSE_SWEEPS (default) or GMG_COARSE_DENSE */
    int coarse_op;      /* coarse operator: GMG_COARSE_OP_FV (default) or GMG_COARSE_OP_GALERKIN */
} gmg_options;

typedef struct {
    int cycles;         /* V-cycles run (rejected ones included) */
    int status;         /* gmg_status of the solve */
    int levels;         /* multigrid levels */
    int outer;          /* FP64 refinement steps (IR modes), else 0 */
    int launches;       /* kernels this call launched (graph replays counted per kernel node) */
    double rel_res;     /* |b - A p|_2 / |b|_2 of the returned p (before the gauge shift) */
    double omega;       /* relaxation factor after the last cycle */
    double bnorm;       /* |b|_2 after the zero-mean projection */
} gmg_info;

typedef struct gmg_solver* gmg_handle;
typedef struct gmg_batch_solver* gmg_batch;

/*
 * Departures from the sketch of this interface in the design notes: no
 * GMG_ERR_SINGULAR_RHS status (the right-hand side is projected onto the
 * operator's range, so a singular operator never makes it unsolvable; NaN or
 * Inf in sigma gives GMG_ERR_NONFINITE instead), and no reject_on_growth
 * switch (a cycle that grows the residual is always rejected: the adaptive
 * relaxation rule of Sec. 3.1 relies on it).
 */

/* Fills *opt with the defaults listed above. */
void gmg_default_options(gmg_options* opt);

/*
 * Plans a solver for one grid.  periodic: 3 flags (x, y, z); a periodic axis
 * must have even length.  Every axis must have length >= 1.  opt may be NULL
 * (defaults).  stream: cudaStream_t (or NULL).  Allocates the hierarchy on
 * the current device.  Errors: GMG_ERR_ARG (dimensions, options, odd periodic
 * length, h NULL), GMG_ERR_CUDA (allocation).
 */
int gmg_create(gmg_handle* h, int nx, int ny, int nz, const int* periodic,
               const gmg_options* opt, void* stream);

/*
 * Copies the face coefficients (three device arrays of nx*ny*nz floats, see
 * Layout) and builds the coarse-level coefficients by finite-volume
 * rediscretisation (coarse face = sum of its fine faces / coarsening factor).
 * Must precede gmg_solve.  Coefficients must be finite and >= 0.
 */
int gmg_set_coeffs(gmg_handle h, const float* bx, const float* by, const float* bz);

/*
 * Solves A p = b, where b is sigma projected to zero mean over the active
 * cells (cells whose face coefficients do not all vanish) and set to 0 on the
 * inactive ones.  sigma and p are device arrays of nx*ny*nz float (FP32 modes)
 * or double (IR modes).  p: initial guess on entry; on exit the iterate with
 * the smallest residual, shifted to zero mean over active cells, 0 on
 * inactive cells.  tol: relative residual target (> 0).  info may be NULL.
 * Blocks the calling host thread until the solve ends.  Returns the solve's
 * status (GMG_OK, GMG_ERR_NOT_CONVERGED, GMG_ERR_DIVERGED, GMG_ERR_NONFINITE)
 * or an error.
 */
int gmg_solve(gmg_handle h, const void* sigma, void* p, double tol, gmg_info* info);

/*
 * As gmg_solve, with sigma and p in HOST memory (pageable or pinned): the
 * call copies sigma and the initial guess to the device, solves, and copies
 * p back, all on the handle's stream.
 */
int gmg_solve_host(gmg_handle h, const void* sigma_host, void* p_host, double tol, gmg_info* info);

/*
 * The comparison solver of the paper (Sec. 3 and Table 1: preconditioned
 * conjugate gradients, general-purpose but with global inner products in every
 * iteration and an iteration count that grows with the grid): CG on the same
 * operator, right-hand-side projection and exit gauge as gmg_solve, with the
 * Jacobi (diagonal) preconditioner, which the paper does not name.  FP32
 * vectors, FP64 inner-product partials; alpha, beta and the stop test
 * (|b - A p| / |b| <= tol, the recursively updated residual) stay on the
 * device, and iterations run in CUDA graphs of 16.
 *
 * h: a single-problem handle with precision GMG_FP32 or GMG_FP32_BF16 and its
 * coefficients set (only the finest level is used).  sigma, p: device float
 * arrays of nx*ny*nz, as for gmg_solve (p: initial guess in, solution out).
 * max_iter >= 1 bounds the iterations.  info->cycles reports CG iterations,
 * info->levels 1.  Returns GMG_OK, GMG_ERR_NOT_CONVERGED (max_iter reached),
 * GMG_ERR_DIVERGED (the search direction lost definiteness or the residual is
 * not finite), GMG_ERR_NONFINITE, GMG_ERR_ARG (IR-precision handle, batch-like
 * misuse, max_iter < 1, tol <= 0) or GMG_ERR_CUDA.  The first call allocates
 * six work vectors of nx*ny*nz floats, kept by the handle.
 */
int gmg_pcg_solve(gmg_handle h, const void* sigma, void* p, double tol, int max_iter, gmg_info* info);

/*
 * The paper's GMG-PCG (Table 1): the multigrid V-cycle of gmg_solve (same
 * hierarchy, coarse coefficients, restriction and prolongation) with PCG as
 * the smoother instead of the adaptive red-black Gauss-Seidel: nu1 and nu2
 * Jacobi-PCG iterations before and after the coarse correction and nu_c on
 * the coarsest level (whose right-hand side is projected to zero mean), each
 * a fresh run from the level's current iterate that also stops once its
 * residual has fallen to 1e-5 of its start.  Cycles are always accepted (no
 * relaxation factor); the solve stops when |b - A p| / |b| <= tol, evaluated
 * after every cycle.  Each cycle is one CUDA graph replay.
 *
 * h: a single-problem GMG_FP32 handle with its coefficients set; sigma, p as
 * for gmg_solve.  info->cycles reports V-cycles.  Returns GMG_OK,
 * GMG_ERR_NOT_CONVERGED (max_cycles), GMG_ERR_NONFINITE, GMG_ERR_ARG or
 * GMG_ERR_CUDA.  The first call allocates six work vectors per level.
 */
int gmg_gmgpcg_solve(gmg_handle h, const void* sigma, void* p, double tol, gmg_info* info);

/*
 * Per-cycle record of the last gmg_solve / gmg_solve_host (the comparison
 * solvers gmg_pcg_solve and gmg_gmgpcg_solve record none): rel_res[k] (k = 0 .. cycles; entry 0
 * is the initial iterate's relative residual, entry k the accepted iterate's
 * after cycle k), omega[k] and accepted[k] (k = 0 .. cycles-1) for cycle k+1.
 * Host arrays of capacity cap (+1 for rel_res).  Returns the number of cycles
 * recorded (<= cap), or -1 on a bad argument.
 */
int gmg_history(gmg_handle h, double* rel_res, double* omega, int* accepted, int cap);

/* Number of levels and their dimensions (host array of 3*levels ints, may be NULL). */
int gmg_levels(gmg_handle h, int* dims);

/* The bottom of the V-cycle as planned at creation or at the last
 * gmg_set_coeffs (the autotuner may move it): *level = the first level that the
 * bottom kernel runs, *ranks = 1 when one CTA runs it, or the number of CTAs of
 * the thread-block cluster that splits its levels of more than 1024 cells by
 * rows (then the smaller levels run in the cluster's first CTA); both 0 when no
 * bottom kernel runs (one level, or a coarsest level too large for one CTA,
 * which then runs as grid sweeps).  GMG_ERR_ARG on a null argument. */
int gmg_bottom_form(gmg_handle h, int* level, int* ranks);

/* Releases the handle and its device memory. */
int gmg_destroy(gmg_handle h);

/* Message of the last error on this handle (or of the last failed create when h is NULL). */
const char* gmg_last_error(gmg_handle h);

/*
 * The autotuner's results, process-wide (no counterpart in the paper: launch
 * shapes are a property of this implementation).  gmg_set_coeffs with
 * autotune = 1 times the z-chunk depth of each pipelined kernel per level
 * geometry; for a single problem, where the bottom kernel starts and whether
 * one CTA or a thread-block cluster runs it; for a batch, how its batched
 * levels are cut into z-chunks (whole V-cycles timed).  It keeps them in a
 * table that later handles of the same shapes reuse without timing.
 *
 * gmg_tune_export writes the table as text: one line per entry,
 *   "z kind nx ny nz px py pz zchunk"   (kind 0 sweep, 1 sweep with correction,
 *                                        2 residual; kind 3 keeps the coarse-grid
 *                                        correction's form, 1 separate, 2 fused)
 *   "b nx ny nz px py pz coarsen n_min precision nu_c coarse level ranks"
 *                                       (coarse = coarse_mode + 2 coarse_op)
 *                                       (first level of the bottom kernel; ranks 1:
 *                                        one CTA, > 1: a cluster of that many CTAs
 *                                        splits its larger levels; a line without
 *                                        ranks reads as 1)
 *   "c nprob hash choice"               (a batch of nprob >= 2 problems, hash: a
 *                                        30-bit hash of their geometries and the
 *                                        hierarchy options; choice = 2 (t + 1) + g:
 *                                        t = -1, each batched level keeps its
 *                                        geometry's z-chunks, t >= 1, every column
 *                                        of a batched level is cut into the fewest
 *                                        chunks that give the launch t tiles; g = 1,
 *                                        one block per tile in the z-marching
 *                                        launches, g = 0, a persistent grid)
 * into buf (host, capacity cap bytes, NUL-terminated) and its length without
 * the NUL into *len.  buf == NULL only reports the length.  GMG_ERR_ARG when
 * cap is too small (nothing written).
 *
 * gmg_tune_import merges such text into the table (entries of the same key
 * are replaced; a "b" line of level 0 removes its key's entry), so that a
 * later process reuses an earlier one's launch shapes: same shapes, same
 * launches, same results bit for bit.  GMG_ERR_ARG,
 * with the table unchanged, on a malformed line.  Neither call touches the GPU.
 */
int gmg_tune_export(char* buf, size_t cap, size_t* len);
int gmg_tune_import(const char* text);

/* ----------------------------------------------------------------------------
 * Batched solves: many independent problems of uneven sizes, one launch per
 * multigrid phase for all of them (levels of equal depth are smoothed,
 * restricted and prolongated together; each problem keeps its own omega,
 * residuals and convergence; converged problems are masked).
 * -------------------------------------------------------------------------- */

/*
 * dims: nprob x 3 ints (nx, ny, nz); periodic: nprob x 3 flags (or NULL for
 * all walls); opt shared by all problems (any precision: the FP64 refinement
 * modes run their outer steps per problem and the V-cycles of all unfinished
 * problems together).
 */
int gmg_batch_create(gmg_batch* b, int nprob, const int* dims, const int* periodic,
                     const gmg_options* opt, void* stream);

/* bx, by, bz: host arrays of nprob device pointers, each to that problem's faces. */
int gmg_batch_set_coeffs(gmg_batch b, const float* const* bx, const float* const* by,
                         const float* const* bz);

/*
 * sigma, p: host arrays of nprob device pointers, to float arrays (GMG_FP32,
 * GMG_FP32_BF16) or double arrays (GMG_IR64, GMG_IR64_FP32), as for gmg_solve.
 * infos: host array of nprob gmg_info (may be NULL).  Returns GMG_OK if every
 * problem converged, else the first failing problem's status.
 */
int gmg_batch_solve(gmg_batch b, const void* const* sigma, void* const* p, double tol,
                    gmg_info* infos);

int gmg_batch_destroy(gmg_batch b);
const char* gmg_batch_last_error(gmg_batch b);

/* ----------------------------------------------------------------------------
 * Single multigrid steps on caller buffers (the kernels the solver is built
 * from), for users assembling their own cycles and for step-by-step checks.
 * Each is asynchronous on `stream`; geometry arguments as for gmg_create.
 * -------------------------------------------------------------------------- */

/*
 * One red-black Gauss-Seidel sweep under-relaxed by omega (Sec. 3.1): red
 * cells ((i+j+k) even) are updated from p_in, then black cells from the new
 * red values: p <- (1-omega) p + omega (sum_f b_f p_nb - b) / sum_f b_f, cells
 * whose faces all vanish keep their value.  p_out must not alias p_in.
 */
int gmg_op_sweep(int nx, int ny, int nz, const int* periodic, const float* bx, const float* by,
                 const float* bz, const float* b, const float* p_in, float* p_out, double omega,
                 void* stream);

/*
 * The same sweep as gmg_op_sweep, run as two in-place launches (red cells,
 * then black cells) with one thread per cell.  It gives bit-identical results
 * and serves as the check that the single-launch sweep has no race.  p is
 * updated in place.
 */
int gmg_op_sweep_reference(int nx, int ny, int nz, const int* periodic, const float* bx,
                           const float* by, const float* bz, const float* b, float* p, double omega,
                           void* stream);

/*
 * Residual r = b - A p of a fine grid, summed over the children of each coarse
 * cell (Sec. 3: coarse-grid correction; restriction = sum over children):
 * b_coarse[J] = sum_{I in J} r_I, where the coarse grid is (nx/fx, ny/fy,
 * nz/fz) with factors f in {1, 2} dividing the axis.  If rr is not NULL, the
 * host receives sum over fine cells of r_I^2 (the call then synchronises the
 * stream).
 */
int gmg_op_residual_restrict(int nx, int ny, int nz, const int* periodic, const int* factors,
                             const float* bx, const float* by, const float* bz, const float* b,
                             const float* p, float* b_coarse, double* rr, void* stream);

/*
 * The residual of the FP64 iterative refinement, r = b - A p, on FP64 arrays b
 * and p (device doubles of nx*ny*nz; faces FP32 as for gmg_op_sweep).
 * definition 0 is the evaluation the solver runs: the six neighbour differences
 * p_nb - p_I in FP64, then the products, their sum and b - A p in double-length
 * FP32 arithmetic (hi + lo pairs of FP32, about 44 significant bits; cells
 * whose values leave the FP32 exponent range are evaluated in FP64).
 * definition 1 evaluates everything in FP64 (the reference the first is
 * checked against).  r_out (device double array) receives r, r32_out (device
 * float array) r rounded to FP32; either may be NULL.  If rr is not NULL the
 * host receives the sum of the squares of the FP32 r (FP64 sum; the call then
 * synchronises the stream).  GMG_ERR_ARG for bad dimensions, null arrays or a
 * definition other than 0 or 1.
 */
int gmg_op_residual64(int nx, int ny, int nz, const int* periodic, const float* bx, const float* by,
                      const float* bz, const double* b, const double* p, double* r_out, float* r32_out,
                      double* rr, int definition, void* stream);

/* p[I] += e[I / f] on the fine grid (piecewise-constant prolongation, Sec. 3). */
int gmg_op_prolong_add(int nx, int ny, int nz, const int* factors, const float* e, float* p,
                       void* stream);

/*
 * Coarse face coefficients of the grid coarsened by factors (Sec. 3.2): the
 * coarse d-face is the sum of the fine d-faces it covers divided by f_d (the
 * finite-volume operator, GMG_COARSE_OP_FV); wall faces of Neumann axes are 0.
 */
int gmg_op_coarsen_coeffs(int nx, int ny, int nz, const int* periodic, const int* factors,
                          const float* bx, const float* by, const float* bz, float* cbx,
                          float* cby, float* cbz, void* stream);

/*
 * |b - A p|_2^2 summed in FP64 on the device, returned to the host in *rr
 * (synchronises the stream).  Uses a library-owned device buffer for the
 * per-block partial sums, allocated on first use per device.
 */
int gmg_op_residual_norm(int nx, int ny, int nz, const int* periodic, const float* bx,
                         const float* by, const float* bz, const float* b, const float* p,
                         double* rr, void* stream);

/*
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot let a library allocate device memory: real-time loops that must
 * never meet the device-wide synchronisation that cudaMalloc / cudaFree may
 * cause, and programs whose device-memory budget is fixed before they start.
 *
 * Same quantity as gmg_op_residual_norm, |b - A p|_2^2 with FP64 partial sums,
 * but its scratch (one FP64 partial sum per 32x4x2-cell tile, plus the total)
 * lives in a fixed array inside the library image: at most 65536 partial
 * sums, i.e. about 16.7 M cells.  Every GPU that loads the library holds that
 * array (about 512 KB) until the process exits.  The call allocates and frees
 * nothing.  It always runs the per-cell residual kernel; gmg_op_residual_norm
 * runs the z-marching kernel when rows are a multiple of 4 cells and the
 * arrays 16-byte aligned, which groups the FP32 squares differently, so the
 * two results may then differ in the last digits (relative ~1e-7).
 *
 * Errors: GMG_ERR_ARG for bad dimensions, a null pointer, or a grid needing
 * more than 65536 partial sums (message in gmg_last_error(NULL));
 * GMG_ERR_CUDA if a CUDA call fails.
 *
 * The first call on a device looks up the array's device address on that
 * device (cudaGetSymbolAddress, with that device current).  All calls on a
 * device share the one array and each overwrites what the previous call left
 * there: calls that overlap on the GPU (concurrent streams, or several host
 * threads) race and must be serialised by the caller.  The call synchronises `stream` and copies the
 * total to *rr (host memory) before it returns.
 */
int gmg_op_residual_norm_noalloc(int nx, int ny, int nz, const int* periodic, const float* bx,
                                 const float* by, const float* bz, const float* b,
                                 const float* p, double* rr, void* stream);

/* ----------------------------------------------------------------------------
 * Test hooks (no counterpart in the paper): host-side fault injection for the
 * failure paths, so that tests need no GPU fault.
 * -------------------------------------------------------------------------- */

/*
 * Arms the handle so that its next solve writes NaN into every problem's
 * device-resident relaxation factor just before V-cycle `cycle` (>= 1) is
 * launched (a host-to-device copy ordered on the handle's stream between two
 * cycles; one shot).  The control rule treats a relaxation factor that is not
 * a positive finite number as corrupt state: that cycle is rejected and the
 * solve returns GMG_ERR_DIVERGED with the best accepted iterate.
 * GMG_ERR_ARG if h is NULL or cycle < 1.
 */
int gmg_test_poison_omega(gmg_handle h, int cycle);

/*
 * Poll limit of the ring-slot waits of the pipelined sweep and residual
 * kernels on the current device (a consumer waiting for a plane, a producer
 * waiting for a free slot); tries < 0 restores the default (about two seconds
 * of polling).  With 0 every such wait gives up at once: the block records the
 * fault, waits (with the full limit) for the copies it already issued, and
 * returns; the next status read of a solve reports GMG_ERR_CUDA ("the launch
 * timed out and was terminated") and the handle should be destroyed.  The
 * setting is process-wide for the device.  GMG_ERR_CUDA if the device
 * variable cannot be written.
 */
int gmg_test_ring_wait_tries(int tries);

/*
 * Largest thread-block cluster the cluster form of the bottom may use in
 * handles planned after this call: 16 or 8 (the form's fallback where a device
 * cannot co-schedule 16 CTAs), 0 restores the default (the largest the device
 * co-schedules).  Process-wide.  GMG_ERR_ARG for any other value.
 */
int gmg_test_cluster_ranks(int ranks);

#ifdef __cplusplus
}
#endif
#endif /* GMG_H */
