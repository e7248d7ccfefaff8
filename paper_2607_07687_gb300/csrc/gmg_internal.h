// gmg_internal.h -- device-side task descriptors and kernel launchers of the
// GB300 multigrid solver (private to the library).
//
// Every kernel works on a list of tasks (one task = one grid level of one
// problem) so that a single launch serves one problem or a whole batch of
// problems of uneven sizes.  Blocks walk the concatenated tiles of all tasks
// (persistent grid-stride loop); tile_off[t] is the first tile of task t.  A
// launch over a single task passes it by value instead (no device copy).
//
// Iterate buffers of the finest level rotate: a task names a buffer by role
// (0 = accepted iterate, 1 and 2 = work) and the live assignment is
// buf[(role + *rot) % 3], so accepting a V-cycle changes *rot instead of
// copying the grid.  Coarse levels use rot == nullptr (fixed roles).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <string>
#include <utility>

#include "gmg_hw.h"

namespace gmg {

constexpr int kMaxLevels = 32;
constexpr int kThreads = 256;           // threads per block of the grid kernels

// sweep tile (cells): TX x TY columns marching through a z-chunk
constexpr int kSweepTX = 32;
constexpr int kSweepTY = 8;
// plane rings of the pipelined sweeps (p, b, x/y/z faces, merged red plane),
// R plane slots each
constexpr int kSweepRing = 6;
constexpr size_t kSweepSmemBytes = sizeof(float) * (kSweepTX + 8) * (kSweepTY + 4) * 6 * kSweepRing;
// the pipelined residual stages the same rings without the merged plane, in
// kResRing slots: 48 KB a block, so that 4 blocks (24 warps) share an SM, where
// 6 slots left room for 3 (18 warps; the 512^3 residual took 0.72 instead of
// 0.62 ms)
constexpr int kResRing = 5;
constexpr size_t kResidualSmemBytes = sizeof(float) * (kSweepTX + 8) * (kSweepTY + 4) * 5 * kResRing;
// residual tile (fine cells)
constexpr int kResTX = 32;
constexpr int kResTY = 4;
constexpr int kResTZ = 2;
// elementwise kernels: cells per tile
constexpr int kElemTile = 4096;

enum RunStatus { kRunning = -1, kOk = 0, kNotConverged = 3, kDiverged = 4, kNonFinite = 5 };

using bf16 = __nv_bfloat16;

struct Geo {
    int n[3];      // nx, ny, nz
    int per[3];    // periodic flags
};

// Tensor maps of one FP32 level for the tensor-memory-accelerator plane
// copies of the pipelined sweep and residual: 3-D maps (x, y, z) with a box of
// one (kSweepTX + 8) x (kSweepTY + 4) plane, zero fill outside the grid.
// Lives in device memory; p[r] maps iterate buffer r.
struct TmaPlanes {
    CUtensorMap p[3];
    CUtensorMap b, x, y, z;
};

// Per-problem solve state, resident in device memory.
struct Ctl {
    double omega;        // relaxation factor used by the next cycle
    double omega_min, shrink, grow;
    double bnorm;        // |b|_2 of the (inner) right-hand side
    double r_prev;       // residual norm of the accepted iterate
    double tol;          // relative residual target of this (inner) solve
    double r_last;       // residual norm of the latest candidate
    double hist_scale;   // history entry = residual norm * hist_scale
    double mean;         // mean used by the last projection / gauge
    double stat_cnt;     // number of active cells
    double outer_bnorm;  // IR: |b64|
    double outer_r;      // IR: |b64 - A p64| of the current p64
    int rot;             // rotation of the finest-level iterate roles
    int cycles;          // cycles run in this (inner) solve
    int total_cycles;    // cycles over all inner solves (IR)
    int status;          // RunStatus of the (inner) solve
    int done;            // 1: every kernel skips this problem
    int max_cycles;      // cycle limit of this (inner) solve
    int res_role;        // role holding the candidate at the end of a cycle
    int nonfinite;       // count of non-finite right-hand-side entries
    int zero_out;        // 1: the solution is identically zero (|b| = 0)
    int outer_status;    // IR: status of the whole solve
    int hist_cap;
    int pad;
    double* hist_res;    // [hist_cap + 1] relative residual after each cycle
    double* hist_omega;  // [hist_cap] omega used by each cycle
    int* hist_acc;       // [hist_cap] accept flag of each cycle
};

// One red-black sweep of one level: p_out = S(p_in [+ P corr]).
template <class TP, class TC>
struct SweepTask {
    Geo g;
    const float* bx;
    const float* by;
    const float* bz;
    const float* b;
    TP* buf[3];
    const int* rot;      // nullptr: roles fixed
    int in_role;         // -1: zero input (coarse levels, first sweep)
    int out_role;
    const TC* corr;      // coarse correction added to the input, or nullptr
    int cf[3];           // coarsening factors of corr
    int tiles_x, tiles_y, zchunk, nchunks;
    float omega;         // used when ctl == nullptr
    const Ctl* ctl;
    const TmaPlanes* tma;  // plane copies by TMA (FP32, 16-byte rows), or nullptr
};

// Residual of one level, restricted to the next level and/or summed in squares.
template <class TP>
struct ResTask {
    Geo g;
    const float* bx;
    const float* by;
    const float* bz;
    const float* b;
    TP* buf[3];
    const int* rot;
    int role;            // -1: zero iterate (residual = b)
    float* bc;           // coarse right-hand side, or nullptr (norm only)
    int cf[3];
    int tiles_x, tiles_y, tiles_z;
    int zchunk;          // marching kernel: cells per z-chunk (tiles_z chunks of 32 x 8 columns)
    double* partials;    // one per tile of this task, or nullptr
    const Ctl* ctl;
    const TmaPlanes* tma;  // plane copies by TMA (marching kernel), or nullptr
};

// Coarse-grid correction of one level as its own pass (the alternative to folding
// it into the first post-smoothing sweep): buf[role] += e[I / c], rows of a
// multiple of 4 cells, 16-byte aligned arrays.
struct ProlongTask {
    Geo g;               // fine level
    int cf[3];           // coarsening factors (cf[0] in {1, 2})
    const float* e;      // coarse correction
    float* buf[3];
    const int* rot;      // nullptr: roles fixed
    int role;
};

// Zero-mean projection of one level's right-hand side over its active cells
// (coarsest levels too large for the bottom kernel; their sweeps then run as k_sweep).
struct LevelProjTask {
    Geo g;
    const float* bx;
    const float* by;
    const float* bz;
    float* b;
    const Ctl* ctl;
};

// The bottom of the V-cycle (levels lb .. L-1 of one problem) in one CTA, or in
// one thread-block cluster whose CTAs split the larger of those levels.
constexpr int kBottomThreads = 1024;
constexpr int kBottomMaxCells = 10240;   // 5 floats per cell of shared memory: 200 KB
static_assert(kBottomMaxCells < (1 << 23), "bottom cell indices are decoded with an FP32 estimate");
// Cluster form: a level of more than kBottomThreads cells is split by rows over
// the cluster's CTAs (distributed level, 10 floats per cell: iterate,
// right-hand side, residual, six face coefficients and the diagonal); the
// smaller levels below it run in CTA 0 as in the one-CTA form.  Each CTA holds
// at most kClusterMaxFloats floats (200 KB).
constexpr int kClusterMaxRanks = 16;
constexpr int kDistArrays = 10;
constexpr int kClusterMaxFloats = 51200;
constexpr int kClusterMaxCells = 1 << 22;   // largest distributed level (FP32 index decoding)

struct BottomLevel {
    Geo g;
    int cf[3];           // coarsening factors to the next level
    const float* bx;
    const float* by;
    const float* bz;
    int off;             // offset (floats) of the level's block in shared memory
    int walls_zeroed;    // 1: the stored faces already read 0 on walls (coarse levels)
    float inv_nx;        // 1 / nx and 1 / (nx ny): cell index -> (x, y, z) by multiplication
    float inv_nxy;
    int cpr;             // distributed level: cells per CTA (a whole number of rows)
    float inv_cpr;       // 1 / cpr
};

// coarse_mode 1: the coarsest level (at most kDenseMaxCells cells) is solved by
// its pseudo-inverse, built at gmg_set_coeffs
constexpr int kDenseMaxCells = 1024;
static_assert(kDenseMaxCells <= kBottomThreads, "one thread per coarsest cell in the dense solve");

template <class TP>
struct BottomTask {
    int nlev;            // levels lb .. L-1; the last one is the coarsest
    BottomLevel lev[kMaxLevels];
    const float* b;      // right-hand side of level lb (written by the finer level)
    TP* out;             // result of level lb (read by the finer level's correction)
    int nu1, nu2, nu_c;
    const Ctl* ctl;
    const float* pinv;   // A^+ of the coarsest level (n x n, symmetric), or nullptr: nu_c sweeps
    int nd;              // cluster form: levels 0 .. nd-1 are distributed (0: one-CTA form)
    int ranks;           // cluster form: CTAs per cluster (the layout's cpr assumes it)
};

struct CtlTask;

template <class Task>
struct TaskList {
    const Task* tasks;   // device array, or nullptr: use `single`
    const int* tile_off; // device prefix of tile counts (ntasks + 1)
    int ntasks;
    int total;           // total tiles
    int vec;             // 4: every task's rows split into aligned 16-byte chunks
    int corr;            // sweeps: 1 if any task adds a coarse correction
    int march;           // residuals: 1 = z-marching kernel (tiles of 32 x 8 columns x zchunk)
    // z-marching norm residual of the fine level: the last block to finish applies
    // the cycle's control rule for these tasks (nullptr: a separate launch does);
    // `arrivals` counts finished blocks and is reset to 0 by that last block
    const CtlTask* ctl_tasks;
    int nctl;
    unsigned* arrivals;
    Task single;
};

// Caller right-hand side -> solver right-hand side, and initial guess copy-in.
template <class TS>
struct ProjTask {
    int64_t n;           // cells
    const uint8_t* mask; // 1 on active cells
    const TS* sigma;
    float* b32;          // FP32 right-hand side, or nullptr
    double* b64;         // FP64 right-hand side, or nullptr
    const TS* p_in;      // caller initial guess, or nullptr (zero)
    float* p32;          // FP32 iterate, or nullptr
    double* p64;         // FP64 iterate, or nullptr (may alias p_in)
    double* partials;    // 3 per tile: sum sigma (active), active count, non-finite count
    double* bpartials;   // 1 per tile: sum b^2
    int tiles;
    Ctl* ctl;
};

// Accepted iterate -> caller array, shifted to zero mean over active cells.
template <class TP, class TD>
struct GaugeTask {
    int64_t n;
    const uint8_t* mask;
    TP* buf[3];
    const int* rot;
    TD* dst;
    double* partials;    // 1 per tile
    int tiles;
    Ctl* ctl;
};

struct CtlTask {
    Ctl* ctl;
    const double* partials;    // residual partials
    int nparts;
    const double* bpartials;   // |b|^2 partials (init only)
    int nbparts;
    const double* ppartials;   // projection partials (3 per tile)
    int npparts;
};

// FP64 iterative refinement on one fine grid.
struct IrTask {
    Geo g;
    const float* bx;
    const float* by;
    const float* bz;
    const double* b64;
    double* p64;
    float* b32;          // inner right-hand side (FP32 r), or nullptr
    double* r64;         // r in full, or nullptr (single-step op)
    float* ebuf[3];      // inner iterate roles (role 0 cleared), ebuf[0] may be nullptr
    const int* rot;
    double* partials;    // one per block of the residual launch (at most one per tile)
    int tiles_x, tiles_y, tiles_z;
    Ctl* ctl;
    double* scale;       // device scalar: inner = outer residual * scale
};

// Scalars of the conjugate-gradient solve kept on the device.
struct PcgScal {
    double rz;           // rho . z of the current residual
    double alpha, beta;
    int smoother;        // 1: tolerances relative to the run's first residual, not to |b|
    int pad;
};

// One Jacobi-preconditioned CG solve on one level (the comparison solver).
struct PcgTask {
    Geo g;
    const float* bx;
    const float* by;
    const float* bz;
    const float* b;      // projected right-hand side
    float* x;            // iterate
    float* r;            // rho = A x - b
    float* z;            // D^-1 rho
    float* q;            // A d
    float* inv_diag;     // D^-1 (0 where no face is open)
    const float* d_src;  // previous direction
    float* d_dst;        // new direction
    double* part;        // 3 per block
    int nparts;
    int zc;              // z-chunk of a block
    Ctl* ctl;            // status, bnorm, r_prev (|rho|), tol, cycles (= iterations), max_cycles
    PcgScal* scal;
};

int pcg_blocks(const Geo& g, int zc);
cudaError_t launch_pcg_start(const PcgTask& t, bool restart, cudaStream_t s);
cudaError_t launch_pcg_iteration(const PcgTask& t, cudaStream_t s);
// arm a run on the device: done = 0, status running, cycles = 0, max_cycles, tol
cudaError_t launch_pcg_arm(Ctl* ctl, PcgScal* scal, int max_it, double tol, int smoother, cudaStream_t s);

// Message returned by gmg_last_error(NULL) for calls without a handle.
void set_api_error(const char* msg);

// Geometry checks shared by every entry point: dimensions >= 1, at most 2^31 - 1
// cells, even length on periodic axes.  GMG_OK, or GMG_ERR_ARG with msg set.
int validate_geometry(int nx, int ny, int nz, const int* periodic, std::string& msg);

// Blocks of the persistent grid-stride kernels for `tiles` tiles: at most
// kResident blocks per SM of the current device.
int persistent_grid(int64_t tiles);

// Ring-slot waits of the pipelined kernels (a consumer waiting for a plane, a
// producer waiting for a free slot) give up after this many mbarrier polls;
// tries < 0 restores the default.  The waits for copies already in flight keep
// their full limit.  Applies to the current device.
cudaError_t set_ring_wait_tries(int tries);

// ---------------------------------------------------------------- launchers

// Launch with programmatic stream serialization: the kernel may be scheduled
// as its predecessor in the stream finishes, before the predecessor's completion
// is signalled, and must execute griddepcontrol.wait (dev::pdl_wait) before it
// touches memory that another kernel writes or reads.  A cluster size > 1 adds
// the thread-block cluster dimension.
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, int cluster,
                       Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    int n = 0;
    at[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
    if (cluster > 1) {
        at[n].id = cudaLaunchAttributeClusterDimension;
        at[n].val.clusterDim.x = (unsigned)cluster;
        at[n].val.clusterDim.y = 1;
        at[n].val.clusterDim.z = 1;
        ++n;
    }
    cfg.attrs = at;
    cfg.numAttrs = n;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <class TP, class TC>
cudaError_t launch_sweep(const TaskList<SweepTask<TP, TC>>& tl, int grid, cudaStream_t s);

// Host: tensor maps of the seven arrays of an FP32 level (null pointers get an
// unused zero map); false if the driver refuses one (the kernels then copy planes
// with per-thread asynchronous copies).  The geometry needs rows of a multiple of
// 4 cells and 16-byte aligned arrays.
bool encode_tma_planes(TmaPlanes* out, const Geo& g, const float* const p[3], const float* b, const float* bx,
                       const float* by, const float* bz);

// Device flag set when a pipelined kernel gave up waiting for its plane copies
// (the kernel then drained its copies and returned); 0 otherwise.
int* wait_fault_flag();
template <class TP>
cudaError_t launch_residual(const TaskList<ResTask<TP>>& tl, int grid, cudaStream_t s);

cudaError_t launch_project_level(const LevelProjTask* tasks, int ntasks, cudaStream_t s);

template <class TP>
cudaError_t launch_bottom(const BottomTask<TP>* tasks, int ntasks, size_t smem, cudaStream_t s);
// cluster form: one cluster of `ranks` CTAs per task
template <class TP>
cudaError_t launch_bottom_cluster(const BottomTask<TP>* tasks, int ntasks, int ranks, size_t smem, cudaStream_t s);
// CTAs per cluster that the current device can co-schedule for the cluster form
// with its full shared-memory budget (16 or 8), or 0 when it cannot
int bottom_cluster_ranks();
// test hook: the largest cluster size bottom_cluster_ranks may return (16 or 8)
void set_cluster_cap(int ranks);

// Reference variant of the sweep: one in-place launch per colour.
cudaError_t launch_sweep_two_pass(Geo g, const float* bx, const float* by, const float* bz,
                                  const float* b, float* p, float omega, cudaStream_t s);

// A^+ of one grid's operator (at most kDenseMaxCells cells) in FP32, n x n
// row-major (symmetric), from its face coefficients (walls already zero);
// synchronises the stream.
cudaError_t build_dense_pinv(const Geo& g, const float* bx, const float* by, const float* bz, float* pinv,
                             cudaStream_t s);

// coarse face coefficients of the next level: finite volume (galerkin 0) or the
// Galerkin operator's (galerkin 1)
cudaError_t launch_coarsen_coeffs(Geo fine, const int cf[3], const float* bx, const float* by,
                                  const float* bz, float* cbx, float* cby, float* cbz, int galerkin,
                                  cudaStream_t s);
cudaError_t launch_prolong_add(Geo fine, const int cf[3], const float* e, float* p, cudaStream_t s);
cudaError_t launch_prolong_rows(const ProlongTask& t, cudaStream_t s);
cudaError_t launch_active_mask(Geo g, const float* bx, const float* by, const float* bz,
                               uint8_t* mask, cudaStream_t s);
cudaError_t launch_sum_partials(const double* partials, int n, double* out, cudaStream_t s);
cudaError_t launch_check_coeffs(int64_t n, const float* bx, const float* by, const float* bz,
                                int* bad, cudaStream_t s);

template <class TS>
cudaError_t launch_project_sum(const TaskList<ProjTask<TS>>& tl, int grid, cudaStream_t s);
template <class TS>
cudaError_t launch_project_apply(const TaskList<ProjTask<TS>>& tl, int grid, cudaStream_t s);
cudaError_t launch_project_finalize(const CtlTask* t, int nprob, cudaStream_t s);
cudaError_t launch_control_init(const CtlTask* t, int nprob, cudaStream_t s);
cudaError_t launch_control_cycle(const CtlTask* t, int nprob, cudaStream_t s);

template <class TP, class TD>
cudaError_t launch_gauge_sum(const TaskList<GaugeTask<TP, TD>>& tl, int grid, cudaStream_t s);
template <class TP, class TD>
cudaError_t launch_gauge_apply(const TaskList<GaugeTask<TP, TD>>& tl, int grid, cudaStream_t s);
cudaError_t launch_gauge_finalize(const CtlTask* t, int nprob, cudaStream_t s);

// r = b64 - A p64 (double-length FP32 after FP64 differences), or, with
// fp64_definition, the all-FP64 evaluation it is checked against
cudaError_t launch_ir_residual(const IrTask& t, int grid, cudaStream_t s, bool fp64_definition = false);
cudaError_t launch_ir_begin_inner(const IrTask& t, int nparts, double tol, double inner_rtol,
                                  int max_cycles, cudaStream_t s);
cudaError_t launch_ir_update(const IrTask& t, cudaStream_t s);

}  // namespace gmg
