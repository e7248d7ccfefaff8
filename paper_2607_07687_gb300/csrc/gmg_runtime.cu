// gmg_runtime.cu -- host runtime and C ABI of the GB300 multigrid solver.
//
// A solve (Sec. 3 of the paper: V-cycles = smoothing + coarse-grid correction;
// Sec. 3.1: adaptive under-relaxed red-black Gauss-Seidel; Sec. 3.2: iso or
// anisotropic coarsening) is planned once per handle:
//   * the coarsening schedule (each axis halves while its length is even and
//     length/2 >= n_min; a periodic axis also stays even; isotropic mode
//     halves all axes together while all qualify, an axis of length 1 (a 2D
//     problem) taking no part);
//   * device buffers of every level and the coefficient hierarchy;
//   * a fixed list of launches for one V-cycle (sweeps, residual+restriction,
//     coarsest solve, prolongation folded into the first post-sweep, fine
//     residual norm, control), recorded once into a CUDA graph.
// Each V-cycle is one graph replay; the relaxation factor, the accepted-iterate
// rotation and the done flag live in device memory, so the host only reads an
// 8-byte-aligned status block every `cycles_per_sync` cycles.
#include "gmg_internal.h"
#include "../../include/gmg.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

using namespace gmg;

namespace {

constexpr int kResident = 8;    // CTAs per SM targeted by the persistent grids

thread_local std::string g_create_error;

int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Tensor maps of one call's arrays (single-step ops), or nullptr when the plane
// copies stay per-thread.  Maps live in device memory in a small cache keyed by
// geometry and pointers, so repeated calls on the same arrays upload nothing;
// an evicted entry is released with cudaFree, which waits for kernels using it.
std::mutex g_map_mutex;
struct MapEntry {
    std::vector<uintptr_t> key;
    TmaPlanes* dev;
    uint64_t used;
};
std::vector<MapEntry> g_map_cache;
uint64_t g_map_clock = 0;
constexpr size_t kMapCacheEntries = 16;

TmaPlanes* op_tensor_maps(const Geo& g, const float* p, const float* b, const float* bx, const float* by,
                          const float* bz, bool vec4, cudaStream_t s)
{
    if (!vec4) return nullptr;
    int dev = 0;
    cudaGetDevice(&dev);
    const std::vector<uintptr_t> key = {(uintptr_t)dev, (uintptr_t)g.n[0], (uintptr_t)g.n[1], (uintptr_t)g.n[2],
                                        (uintptr_t)p, (uintptr_t)b, (uintptr_t)bx, (uintptr_t)by, (uintptr_t)bz};
    std::lock_guard<std::mutex> lock(g_map_mutex);
    for (MapEntry& m : g_map_cache)
        if (m.key == key) {
            m.used = ++g_map_clock;
            return m.dev;
        }
    TmaPlanes h;
    const float* pb[3] = {p, nullptr, nullptr};
    if (!encode_tma_planes(&h, g, pb, b, bx, by, bz)) return nullptr;
    if (g_map_cache.size() >= kMapCacheEntries) {
        auto it = std::min_element(g_map_cache.begin(), g_map_cache.end(),
                                   [](const MapEntry& a, const MapEntry& c) { return a.used < c.used; });
        cudaFree(it->dev);
        g_map_cache.erase(it);
    }
    TmaPlanes* d = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&d), sizeof(h)) != cudaSuccess) return nullptr;
    if (cudaMemcpyAsync(d, &h, sizeof(h), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    g_map_cache.push_back({key, d, ++g_map_clock});
    return d;
}

}  // namespace

namespace gmg {

int sm_count()
{
    constexpr int kDevices = 64;
    static std::atomic<int> cached[kDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < kDevices) {
        const int c = cached[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
    if (dev >= 0 && dev < kDevices) cached[dev].store(n, std::memory_order_relaxed);
    return n;
}

int persistent_grid(int64_t tiles)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sm_count() * kResident));
}

// Grids of the z-marching kernels (k_sweep_ws, k_residual_ws) of one problem:
// one block per tile.  The hardware starts the blocks in tile order as earlier
// ones finish, so tiles that share halo rows (neighbours in x and y sit close in
// that order) stream the same planes at about the same time and their halos come
// from L2; blocks of a persistent grid, each walking a fixed stride of tiles,
// drift apart over many tiles and read the halos from DRAM again (512^3
// triple-periodic sweep: DRAM reads 1.08 instead of 1.63 times the inputs).
// Levels of at most one tile per resident block launch the same grid either way.
// A batched launch takes one block per tile only where its autotuner chose it
// (`batch_one_block`): with the short z-chunks a problem tuned alone gets, each
// block would pay a pipeline start for a few planes (64-problem batch 12 % slower).
template <class TC>
int sweep_grid(const TaskList<SweepTask<float, TC>>& tl, bool batch_one_block = false)
{
    return tl.vec >= 4 && (tl.ntasks <= 1 || batch_one_block) ? std::max(1, tl.total) : persistent_grid(tl.total);
}

int residual_grid(const TaskList<ResTask<float>>& tl, bool batch_one_block = false)
{
    return tl.march && (tl.ntasks <= 1 || batch_one_block) ? std::max(1, tl.total) : persistent_grid(tl.total);
}

}  // namespace gmg

namespace {

// ------------------------------------------------------------ schedule (C3)

bool axis_halves(int n, int periodic, int n_min)
{
    if (n % 2) return false;
    if (n / 2 < n_min) return false;
    if (periodic && (n / 2) % 2) return false;
    return true;
}

int plan_levels(const Geo& g0, int aniso, int n_min, Geo* geo, int (*cf)[3])
{
    int L = 0;
    Geo g = g0;
    for (;;) {
        geo[L] = g;
        cf[L][0] = cf[L][1] = cf[L][2] = 1;
        ++L;
        if (L >= kMaxLevels) break;
        bool h[3], any = false, all = true;
        for (int d = 0; d < 3; ++d) {
            h[d] = axis_halves(g.n[d], g.per[d], n_min);
            any |= h[d];
            if (g.n[d] > 1) all &= h[d];   // an axis of length 1 (a 2D problem) is not coarsened
        }
        if (!any || (!aniso && !all)) break;
        for (int d = 0; d < 3; ++d) {
            cf[L - 1][d] = h[d] ? 2 : 1;
            g.n[d] /= cf[L - 1][d];
        }
    }
    return L;
}

int64_t cells(const Geo& g) { return (int64_t)g.n[0] * g.n[1] * g.n[2]; }

// NVTX range over a host-side phase (set-up, autotuning, a solve, a refinement
// step), for profilers that filter or group launches by range
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// rows of a multiple of 4 cells and 16-byte aligned arrays: the sweep copies
// 16-byte chunks; otherwise single floats
template <class TC>
int sweep_vec(const SweepTask<float, TC>& t)
{
    if (t.g.n[0] % 4) return 1;
    if (!aligned16(t.bx) || !aligned16(t.by) || !aligned16(t.bz) || !aligned16(t.b)) return 1;
    for (int r = 0; r < 3; ++r)
        if (!aligned16(t.buf[r])) return 1;
    return 4;
}
template <class TC>
int sweep_vec(const SweepTask<bf16, TC>&) { return 1; }

struct SweepTiling {
    int tx, ty, zchunk, nchunks;
    int64_t tiles() const { return (int64_t)tx * ty * nchunks; }
};

// ------------------------------------------------------------ autotuned shapes
// z-chunk depth per (kernel kind, level geometry), filled by Engine::tune from
// timed trial launches and shared by every handle of the process.
enum TuneKind { kTuneSweep = 0, kTuneSweepCorr = 1, kTuneResidual = 2, kTuneCorrForm = 3 };
// kTuneCorrForm entries: 1 = correction as its own pass before a plain sweep, 2 = folded into the sweep
enum { kCorrSeparate = 1, kCorrFused = 2 };

struct TuneKey {
    int kind, n0, n1, n2, p0, p1, p2;
    bool operator<(const TuneKey& o) const
    {
        const int a[7] = {kind, n0, n1, n2, p0, p1, p2}, b[7] = {o.kind, o.n0, o.n1, o.n2, o.p0, o.p1, o.p2};
        return std::lexicographical_compare(a, a + 7, b, b + 7);
    }
};

std::mutex g_tune_mutex;
std::map<TuneKey, int> g_tuned_zchunk;
// tuned start and form of the bottom per (fine geometry, hierarchy options):
// every handle of the same problem shape then runs the same cycle, bit for bit
struct BottomChoice {
    int level;   // first level of the bottom kernel
    int ranks;   // 1: one CTA; > 1: the cluster form
};
std::map<std::vector<int>, BottomChoice> g_tuned_lb;
// tuned z-chunk policy and grid of a batch per (problem count, 30-bit hash of the
// problems' geometries and the hierarchy options): 2 (target tiles per batched
// launch + 1) + 1 if one block per tile (target -1: the depths of each level's
// geometry)
std::map<std::pair<int, int>, int> g_tuned_batch;

TuneKey tune_key(int kind, const Geo& g) { return {kind, g.n[0], g.n[1], g.n[2], g.per[0], g.per[1], g.per[2]}; }

int tuned_zchunk(int kind, const Geo& g)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned_zchunk.find(tune_key(kind, g));
    return it == g_tuned_zchunk.end() ? 0 : it->second;
}

// heuristic depth: the chunk count that minimises rounds x (chunk + 3 planes of
// pipeline fill), a round being one tile on each of the 3 CTA slots per SM the
// pipelined kernels occupy; chunks of >= 4 planes
int default_zchunk(const Geo& g)
{
    const int64_t cols = (int64_t)ceil_div(g.n[0], kSweepTX) * ceil_div(g.n[1], kSweepTY);
    const int64_t slots = (int64_t)sm_count() * 3;
    int best_zc = g.n[2];
    double best = 1e300;
    for (int nc = 1; nc <= std::max(1, g.n[2] / 4); ++nc) {
        const int zc = ceil_div(g.n[2], nc);
        const int64_t tiles = cols * ceil_div(g.n[2], zc);
        const double cost = (double)((tiles + slots - 1) / slots) * (zc + 3);
        if (cost < best * 0.999) {
            best = cost;
            best_zc = zc;
        }
    }
    return best_zc;
}

SweepTiling sweep_tiling(const Geo& g, int kind = kTuneSweep, int zchunk = 0)
{
    SweepTiling t;
    t.tx = ceil_div(g.n[0], kSweepTX);
    t.ty = ceil_div(g.n[1], kSweepTY);
    if (zchunk <= 0) zchunk = tuned_zchunk(kind, g);
    if (zchunk <= 0) zchunk = default_zchunk(g);
    t.zchunk = std::min(zchunk, g.n[2]);
    t.nchunks = ceil_div(g.n[2], t.zchunk);
    return t;
}

struct ResTiling {
    int tx, ty, tz;
    int zchunk;   // marching tiling only
    int64_t tiles() const { return (int64_t)tx * ty * tz; }
};

// 32 x 4 x 2 cell tiles of the per-cell residual kernel
ResTiling res_tiling(const Geo& g)
{
    return {ceil_div(g.n[0], kResTX), ceil_div(g.n[1], kResTY), ceil_div(g.n[2], kResTZ), 0};
}

// FP32 levels with rows of a multiple of 4 cells use the z-marching residual
bool res_marches(const Geo& g, bool fp32) { return fp32 && g.n[0] % 4 == 0; }

// 32 x 8 columns x z-chunks of even length (coarse z-pairs never straddle chunks)
ResTiling march_tiling(const Geo& g, int zchunk = 0)
{
    ResTiling t;
    t.tx = ceil_div(g.n[0], kSweepTX);
    t.ty = ceil_div(g.n[1], kSweepTY);
    if (zchunk <= 0) zchunk = tuned_zchunk(kTuneResidual, g);
    if (zchunk <= 0) zchunk = default_zchunk(g);
    t.zchunk = std::min(zchunk, g.n[2]);
    if (t.zchunk % 2 && t.zchunk < g.n[2]) ++t.zchunk;
    t.tz = ceil_div(g.n[2], t.zchunk);
    return t;
}

ResTiling level_res_tiling(const Geo& g, bool fp32) { return res_marches(g, fp32) ? march_tiling(g) : res_tiling(g); }

// ------------------------------------------------------------ plan structures

struct LevelMem {
    Geo g;
    int cf[3];
    float* beta[3] = {nullptr, nullptr, nullptr};
    float* b = nullptr;
    void* buf[3] = {nullptr, nullptr, nullptr};
    TmaPlanes* tma = nullptr;     // device tensor maps of the FP32 arrays, or nullptr
};

struct ProblemMem {
    Geo g0;
    int L = 0;
    LevelMem lev[kMaxLevels];
    uint8_t* mask = nullptr;
    int64_t n0 = 0;
    int elem_tiles = 0;
    double* norm_part = nullptr;    // fine residual norm partials
    int norm_tiles = 0;              // partials the finest residual writes (current tiling)
    int norm_cap = 0;                // partials the buffer holds
    int res_zchunk0 = 0;             // z-chunk depth of the finest residual, fixed per handle
    double* proj_part = nullptr;    // 3 per element tile
    double* bpart = nullptr;        // 1 per element tile
    double* gauge_part = nullptr;   // 1 per element tile
    double* b64 = nullptr;          // IR right-hand side
    double* ir_part = nullptr;
    Ctl* ctl = nullptr;             // device
    double* hist_res = nullptr;
    double* hist_omega = nullptr;
    int* hist_acc = nullptr;
    float* pinv = nullptr;          // coarse_mode 1: A^+ of the coarsest level
};

enum OpKind { kSweepFF, kSweepFB, kSweepBB, kResF, kResB, kBottomF, kBottomB, kProjLevel, kControl, kProlong };

struct LaunchOp {
    OpKind kind;
    int grid = 1;
    TaskList<SweepTask<float, float>> s_ff{};
    TaskList<SweepTask<float, bf16>> s_fb{};
    TaskList<SweepTask<bf16, bf16>> s_bb{};
    TaskList<ResTask<float>> r_f{};
    TaskList<ResTask<bf16>> r_b{};
    const BottomTask<float>* bot_f = nullptr;
    const BottomTask<bf16>* bot_b = nullptr;
    size_t smem = 0;
    int ranks = 1;   // bottom: CTAs per task (> 1: cluster form)
    const LevelProjTask* lp = nullptr;
    const CtlTask* ctl = nullptr;
    ProlongTask pro{};
    int n = 0;
};

struct Engine {
    std::vector<ProblemMem> P;
    gmg_options opt{};
    cudaStream_t stream = nullptr;
    bool bf16_coarse = false;
    bool ir = false;
    int device = 0;
    std::vector<int> res_role;      // per problem: role of the candidate after a cycle
    void* stage[2] = {nullptr, nullptr};   // device staging of gmg_solve_host
    std::vector<void*> allocs;
    std::vector<LaunchOp> cycle;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    Ctl* ctl_dev = nullptr;         // nprob
    Ctl* ctl_host = nullptr;        // pinned mirror
    int* fault_host = nullptr;      // pinned copy of the plane-copy wait fault flag
    int* fault_dev = nullptr;
    CtlTask* cycle_ctl = nullptr;   // device: per-cycle control tasks
    CtlTask* init_ctl = nullptr;    // device: init / projection / gauge tasks
    CtlTask* gauge_ctl = nullptr;
    bool coeffs_set = false;
    int poison_cycle = 0;           // test hook: before this V-cycle of the next solve, omega = NaN
    std::string err;
    int last_cycles = 0;
    long long launches = 0;     // kernels launched since the counter was reset

    // conjugate-gradient comparison solver (problem 0): r, z, q, D^-1, d0, d1
    float* pcg_buf[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double* pcg_part = nullptr;
    PcgScal* pcg_scal = nullptr;
    cudaGraphExec_t pcg_exec = nullptr;
    static constexpr int kPcgZChunk = 8;      // z-planes per block of the CG kernels
    static constexpr int kPcgGraphIters = 16; // iterations per graph replay (even: d0/d1 alternate)
    static constexpr int kPcgMaxRestarts = 64; // true-residual checks per solve

    ~Engine() { release(); }

    void release()
    {
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        graph_exec = nullptr;
        graph = nullptr;
        if (pcg_exec) cudaGraphExecDestroy(pcg_exec);
        pcg_exec = nullptr;
        if (gp_exec) cudaGraphExecDestroy(gp_exec);
        gp_exec = nullptr;
        gp_lev.clear();
        gp_probe = nullptr;
        gp_proj = nullptr;
        for (float*& b : pcg_buf) b = nullptr;
        for (void* a : allocs) cudaFree(a);
        allocs.clear();
        if (ctl_host) cudaFreeHost(ctl_host);
        ctl_host = nullptr;
        if (fault_host) cudaFreeHost(fault_host);
        fault_host = nullptr;
    }

    int fail(int code, const char* fmt, ...)
    {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        err = buf;
        return code;
    }

    int cuda_fail(cudaError_t e, const char* what)
    {
        return fail(GMG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    }

    template <class T>
    T* dalloc(size_t count)
    {
        void* p = nullptr;
        if (count == 0) count = 1;
        if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) return nullptr;
        allocs.push_back(p);
        return static_cast<T*>(p);
    }

    template <class T>
    T* upload(const std::vector<T>& v)
    {
        T* d = dalloc<T>(v.size());
        if (!d) return nullptr;
        if (cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
            return nullptr;
        return d;
    }

    // ---------------------------------------------------------------- planning

    int plan(int nprob, const int* dims, const int* periodic, const gmg_options& o, cudaStream_t s)
    {
        opt = o;
        stream = s;
        bf16_coarse = o.precision == GMG_FP32_BF16 || o.precision == GMG_IR64;
        ir = o.precision == GMG_IR64 || o.precision == GMG_IR64_FP32;
        cudaGetDevice(&device);
        P.resize(nprob);
        int64_t total_norm = 0, total_elem = 0;
        for (int p = 0; p < nprob; ++p) {
            ProblemMem& M = P[p];
            for (int d = 0; d < 3; ++d) {
                M.g0.n[d] = dims[3 * p + d];
                M.g0.per[d] = periodic ? (periodic[3 * p + d] != 0) : 0;
            }
            Geo geo[kMaxLevels];
            int cf[kMaxLevels][3];
            M.L = plan_levels(M.g0, o.coarsen == GMG_COARSEN_ANISO, o.n_min, geo, cf);
            M.n0 = cells(M.g0);
            if (o.coarse_mode == GMG_COARSE_DENSE) {
                const int64_t nc = cells(geo[M.L - 1]);
                if (M.L < 2)
                    return fail(GMG_ERR_ARG, "coarse_mode DENSE needs at least two levels (problem %d does not coarsen)", p);
                if (nc > kDenseMaxCells)
                    return fail(GMG_ERR_ARG,
                                "coarse_mode DENSE needs a coarsest level of at most %d cells (problem %d: %lld)",
                                kDenseMaxCells, p, (long long)nc);
                if (!(M.pinv = dalloc<float>((size_t)(nc * nc)))) return fail(GMG_ERR_CUDA, "out of device memory");
            }
            for (int l = 0; l < M.L; ++l) {
                LevelMem& Lm = M.lev[l];
                Lm.g = geo[l];
                for (int d = 0; d < 3; ++d) Lm.cf[d] = cf[l][d];
                const int64_t n = cells(geo[l]);
                for (int d = 0; d < 3; ++d)
                    if (!(Lm.beta[d] = dalloc<float>(n))) return fail(GMG_ERR_CUDA, "out of device memory");
                if (!(Lm.b = dalloc<float>(n))) return fail(GMG_ERR_CUDA, "out of device memory");
                const int nb = l == 0 ? 3 : 2;
                for (int r = 0; r < nb; ++r) {
                    void* q = (l > 0 && bf16_coarse) ? (void*)dalloc<bf16>(n) : (void*)dalloc<float>(n);
                    if (!q) return fail(GMG_ERR_CUDA, "out of device memory");
                    Lm.buf[r] = q;
                }
                if (!(l > 0 && bf16_coarse)) {
                    TmaPlanes h;
                    const float* pb[3] = {static_cast<const float*>(Lm.buf[0]), static_cast<const float*>(Lm.buf[1]),
                                          static_cast<const float*>(Lm.buf[2])};
                    if (encode_tma_planes(&h, Lm.g, pb, Lm.b, Lm.beta[0], Lm.beta[1], Lm.beta[2])) {
                        if (!(Lm.tma = dalloc<TmaPlanes>(1))) return fail(GMG_ERR_CUDA, "out of device memory");
                        if (cudaMemcpy(Lm.tma, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess)
                            return fail(GMG_ERR_CUDA, "tensor map upload failed");
                    }
                }
            }
            if (!(M.mask = dalloc<uint8_t>(M.n0))) return fail(GMG_ERR_CUDA, "out of device memory");
            M.elem_tiles = ceil_div(M.n0, kElemTile);
            // room for the finest tiling any z-chunk depth can give
            M.norm_cap = (int)std::max<int64_t>(res_tiling(M.g0).tiles(), march_tiling(M.g0, 1).tiles());
            total_norm += M.norm_cap;
            total_elem += M.elem_tiles;
            if (ir) {
                if (!(M.b64 = dalloc<double>(M.n0))) return fail(GMG_ERR_CUDA, "out of device memory");
                if (!(M.ir_part = dalloc<double>(res_tiling(M.g0).tiles())))
                    return fail(GMG_ERR_CUDA, "out of device memory");
            }
            const int cap = std::max(1, o.max_cycles);
            M.hist_res = dalloc<double>(cap + 1);
            M.hist_omega = dalloc<double>(cap);
            M.hist_acc = dalloc<int>(cap);
            if (!M.hist_res || !M.hist_omega || !M.hist_acc) return fail(GMG_ERR_CUDA, "out of device memory");
        }
        double* norm = dalloc<double>(total_norm);
        double* proj = dalloc<double>(3 * total_elem);
        double* bp = dalloc<double>(total_elem);
        double* gp = dalloc<double>(total_elem);
        ctl_dev = dalloc<Ctl>(nprob);
        if (!norm || !proj || !bp || !gp || !ctl_dev) return fail(GMG_ERR_CUDA, "out of device memory");
        if (cudaMallocHost(&ctl_host, sizeof(Ctl) * nprob) != cudaSuccess)
            return fail(GMG_ERR_CUDA, "out of pinned host memory");
        if (cudaMallocHost(&fault_host, sizeof(int)) != cudaSuccess)
            return fail(GMG_ERR_CUDA, "out of pinned host memory");
        *fault_host = 0;
        fault_dev = wait_fault_flag();
        std::memset(ctl_host, 0, sizeof(Ctl) * nprob);
        int64_t on = 0, oe = 0;
        for (int p = 0; p < nprob; ++p) {
            ProblemMem& M = P[p];
            M.norm_part = norm + on;
            M.proj_part = proj + 3 * oe;
            M.bpart = bp + oe;
            M.gauge_part = gp + oe;
            M.ctl = ctl_dev + p;
            on += M.norm_cap;
            oe += M.elem_tiles;
        }
        if (upload_ctl_tasks() != GMG_OK) return fail(GMG_ERR_CUDA, "upload failed");
        return build_cycle();
    }

    // tiling of the finest level's residual, as fixed by upload_ctl_tasks
    static ResTiling res0_tiling(const ProblemMem& M)
    {
        return M.res_zchunk0 > 0 ? march_tiling(M.g0, M.res_zchunk0) : res_tiling(M.g0);
    }

    // control tasks: how many residual partials each problem's finest level
    // writes (this follows the tuned tiling)
    int upload_ctl_tasks()
    {
        const int nprob = (int)P.size();
        std::vector<CtlTask> cyc(nprob), ini(nprob), gau(nprob);
        for (int p = 0; p < nprob; ++p) {
            ProblemMem& M = P[p];
            M.res_zchunk0 = res_marches(M.g0, true) ? march_tiling(M.g0, batch_zchunk(p, 0)).zchunk : 0;
            M.norm_tiles = (int)res0_tiling(M).tiles();
            if (M.norm_tiles > M.norm_cap) return GMG_ERR_CUDA;
            cyc[p] = CtlTask{M.ctl, M.norm_part, M.norm_tiles, nullptr, 0, nullptr, 0};
            ini[p] = CtlTask{M.ctl, M.norm_part, M.norm_tiles, M.bpart, M.elem_tiles, M.proj_part, M.elem_tiles};
            gau[p] = CtlTask{M.ctl, nullptr, 0, nullptr, 0, M.gauge_part, M.elem_tiles};
        }
        if (cycle_ctl) drop(cycle_ctl);
        if (init_ctl) drop(init_ctl);
        if (gauge_ctl) drop(gauge_ctl);
        cycle_ctl = init_ctl = gauge_ctl = nullptr;
        if (!(cycle_ctl = upload(cyc)) || !(init_ctl = upload(ini)) || !(gauge_ctl = upload(gau))) return GMG_ERR_CUDA;
        return GMG_OK;
    }

    // device array + prefix of tile counts for a multi-task list
    template <class Task>
    int make_list(const std::vector<Task>& tasks, const std::vector<int64_t>& tiles, TaskList<Task>& tl)
    {
        tl = TaskList<Task>{};
        tl.ntasks = (int)tasks.size();
        tl.vec = 1;
        tl.corr = 0;
        int64_t tot = 0;
        std::vector<int> off(tasks.size() + 1);
        for (size_t i = 0; i < tasks.size(); ++i) {
            off[i] = (int)tot;
            tot += tiles[i];
        }
        off[tasks.size()] = (int)tot;
        tl.total = (int)tot;
        if (tasks.size() == 1) {
            tl.tasks = nullptr;
            tl.tile_off = nullptr;
            tl.single = tasks[0];
            return GMG_OK;
        }
        tl.tasks = upload(tasks);
        tl.tile_off = upload(off);
        if (!tl.tasks || !tl.tile_off) return fail(GMG_ERR_CUDA, "upload failed");
        return GMG_OK;
    }

    // role bookkeeping: on level 0 roles {0 accepted, 1, 2} rotate; on coarse
    // levels physical buffers {0, 1}; -1 = zero input.
    static int next_out(int level, int in)
    {
        if (level == 0) return in == 1 ? 2 : 1;
        return in == 0 ? 1 : 0;
    }

    template <class TP, class TC>
    SweepTask<TP, TC> sweep_task(int p, int l, int in, int out, bool with_corr)
    {
        const ProblemMem& M = P[p];
        const LevelMem& Lm = M.lev[l];
        SweepTask<TP, TC> t{};
        t.g = Lm.g;
        t.bx = Lm.beta[0];
        t.by = Lm.beta[1];
        t.bz = Lm.beta[2];
        t.b = Lm.b;
        for (int r = 0; r < 3; ++r) t.buf[r] = static_cast<TP*>(Lm.buf[r]);
        t.rot = l == 0 ? &M.ctl->rot : nullptr;
        t.in_role = in;
        t.out_role = out;
        t.corr = nullptr;
        t.cf[0] = t.cf[1] = t.cf[2] = 1;
        if (with_corr) {
            t.corr = static_cast<const TC*>(M.lev[l + 1].buf[coarse_result_[p][l + 1]]);
            for (int d = 0; d < 3; ++d) t.cf[d] = Lm.cf[d];
        }
        const SweepTiling st = sweep_tiling(Lm.g, with_corr ? kTuneSweepCorr : kTuneSweep, batch_zchunk(p, l));
        t.tiles_x = st.tx;
        t.tiles_y = st.ty;
        t.zchunk = st.zchunk;
        t.nchunks = st.nchunks;
        t.omega = 1.0f;
        t.ctl = M.ctl;
        t.tma = std::is_same<TP, float>::value ? Lm.tma : nullptr;
        return t;
    }

    // the coarse-grid correction of level l as its own pass into the iterate of `role`
    ProlongTask prolong_task(int p, int l, int role) const
    {
        const ProblemMem& M = P[p];
        const LevelMem& Lm = M.lev[l];
        ProlongTask t{};
        t.g = Lm.g;
        for (int d = 0; d < 3; ++d) t.cf[d] = Lm.cf[d];
        t.e = static_cast<const float*>(M.lev[l + 1].buf[coarse_result_[p][l + 1]]);
        for (int r = 0; r < 3; ++r) t.buf[r] = static_cast<float*>(Lm.buf[r]);
        t.rot = l == 0 ? &M.ctl->rot : nullptr;
        t.role = role;
        return t;
    }

    // a single FP32 problem whose level l (rows of a multiple of 4 cells, FP32 correction)
    // may take its correction as a separate pass: the autotuner decides
    bool corr_separable(int l) const
    {
        if (P.size() != 1 || bf16_coarse) return false;
        const LevelMem& Lm = P[0].lev[l];
        if (Lm.g.n[0] % 4 || Lm.cf[0] > 2) return false;
        for (int r = 0; r < 3; ++r)
            if (Lm.buf[r] && !aligned16(Lm.buf[r])) return false;
        return aligned16(P[0].lev[l + 1].buf[0]) && aligned16(P[0].lev[l + 1].buf[1]);
    }

    template <class TP>
    ResTask<TP> res_task(int p, int l, int role, bool restrict_to_next, double* partials)
    {
        const ProblemMem& M = P[p];
        const LevelMem& Lm = M.lev[l];
        ResTask<TP> t{};
        t.g = Lm.g;
        t.bx = Lm.beta[0];
        t.by = Lm.beta[1];
        t.bz = Lm.beta[2];
        t.b = Lm.b;
        for (int r = 0; r < 3; ++r) t.buf[r] = static_cast<TP*>(Lm.buf[r]);
        t.rot = l == 0 ? &M.ctl->rot : nullptr;
        t.role = role;
        t.bc = restrict_to_next ? M.lev[l + 1].b : nullptr;
        for (int d = 0; d < 3; ++d) t.cf[d] = restrict_to_next ? Lm.cf[d] : 1;
        constexpr bool fp32 = std::is_same<TP, float>::value;
        const int bzc = batch_zchunk(p, l);
        const ResTiling rt = (l == 0 && M.res_zchunk0 > 0)        ? res0_tiling(M)
                             : (bzc > 0 && res_marches(Lm.g, fp32)) ? march_tiling(Lm.g, bzc)
                                                                   : level_res_tiling(Lm.g, fp32);
        t.tiles_x = rt.tx;
        t.tiles_y = rt.ty;
        t.tiles_z = rt.tz;
        t.zchunk = rt.zchunk;
        t.partials = partials;
        t.ctl = M.ctl;
        t.tma = std::is_same<TP, float>::value ? Lm.tma : nullptr;
        return t;
    }

    // residual launches of level l for `probs`: problems whose level marches and
    // those that do not go to separate launches
    int res_ops(int l, const std::vector<int>& probs, const std::vector<int>& role, bool restrict_to_next,
                bool norm, std::vector<LaunchOp>& ops)
    {
        const bool bf = l > 0 && bf16_coarse;
        for (int m = 0; m < 2; ++m) {
            std::vector<int> sel;
            for (size_t i = 0; i < probs.size(); ++i)
                if ((int)res_marches(P[probs[i]].lev[l].g, !bf) == m) sel.push_back((int)i);
            if (sel.empty()) continue;
            LaunchOp op;
            std::vector<int64_t> tiles;
            int rc;
            if (bf) {
                std::vector<ResTask<bf16>> v;
                for (int i : sel) {
                    const int p = probs[i];
                    v.push_back(res_task<bf16>(p, l, role[i], restrict_to_next, norm ? P[p].norm_part : nullptr));
                    tiles.push_back(level_res_tiling(P[p].lev[l].g, false).tiles());
                }
                op.kind = kResB;
                if ((rc = make_list(v, tiles, op.r_b))) return rc;
                op.grid = persistent_grid(op.r_b.total);
            } else {
                std::vector<ResTask<float>> v;
                for (int i : sel) {
                    const int p = probs[i];
                    v.push_back(res_task<float>(p, l, role[i], restrict_to_next, norm ? P[p].norm_part : nullptr));
                    tiles.push_back((int64_t)v.back().tiles_x * v.back().tiles_y * v.back().tiles_z);
                }
                op.kind = kResF;
                if ((rc = make_list(v, tiles, op.r_f))) return rc;
                op.r_f.march = m;
                op.grid = residual_grid(op.r_f, batch_one_block_);
            }
            ops.push_back(op);
        }
        return GMG_OK;
    }

    std::vector<std::vector<int>> coarse_result_;   // [p][l] buffer holding the level's result
    std::vector<int> stop_;                         // [p] first level not run by grid kernels
    int forced_lb_ = 0;                             // tuned start of the bottom (0: smallest one-CTA fit)
    int forced_ranks_ = 1;                          // tuned form of the bottom (> 1: cluster form)
    std::vector<int> fit_lb_;                       // [p] smallest one-CTA fit, -1 if none
    int bottom_level_ = 0, bottom_ranks_ = 0;       // problem 0's bottom as planned (0: none)
    unsigned* arrivals_ = nullptr;                  // block counter of the norm residual with the control rule
    bool tuned_ = false;
    int batch_target_ = -1;                         // batches: tiles each level's launch aims for (-1: per-geometry depths)
    bool batch_one_block_ = false;                  // batches: one block per tile in the z-marching launches

    // z-chunk depth of problem p's level l in a batched launch: every column of the
    // level's launch gets the same number of chunks, the fewest that give the launch
    // batch_target_ tiles (0: the depth tuned or chosen for the level's geometry
    // alone, as a single problem uses)
    // 30-bit FNV-1a hash of the batch's geometries and hierarchy options: the key of
    // its z-chunk policy in the tuning table
    int batch_hash() const
    {
        uint32_t h = 2166136261u;
        auto mix = [&](int v) {
            for (int i = 0; i < 4; ++i) {
                h ^= (uint32_t)(v >> (8 * i)) & 0xffu;
                h *= 16777619u;
            }
        };
        for (const ProblemMem& Q : P)
            for (int d = 0; d < 3; ++d) {
                mix(Q.g0.n[d]);
                mix(Q.g0.per[d]);
            }
        for (int v : {opt.coarsen, opt.n_min, opt.precision, opt.nu1, opt.nu2, opt.nu_c, opt.coarse_mode,
                      opt.coarse_op})
            mix(v);
        return (int)(h & ((1u << 30) - 1));
    }

    int batch_zchunk(int p, int l) const
    {
        if (P.size() < 2 || batch_target_ < 0) return 0;
        int64_t cols = 0;
        int nz_max = 1;
        for (const ProblemMem& Q : P) {
            if (l >= Q.L) continue;
            const Geo& g = Q.lev[l].g;
            cols += (int64_t)ceil_div(g.n[0], kSweepTX) * ceil_div(g.n[1], kSweepTY);
            nz_max = std::max(nz_max, g.n[2]);
        }
        int nc = 1;
        while (cols * nc < batch_target_ && nc < nz_max) ++nc;
        return ceil_div(P[p].lev[l].g.n[2], nc);
    }

    int add_sweeps(int l, const std::vector<int>& probs, int in, int out, bool with_corr)
    {
        const bool coarse_bf = l > 0 && bf16_coarse;
        const bool corr_bf = with_corr && bf16_coarse;   // the correction comes from level l+1 >= 1
        LaunchOp op;
        std::vector<int64_t> tiles;
        for (int p : probs)
            tiles.push_back(sweep_tiling(P[p].lev[l].g, with_corr ? kTuneSweepCorr : kTuneSweep, batch_zchunk(p, l))
                                .tiles());
        int rc;
        if (coarse_bf) {
            std::vector<SweepTask<bf16, bf16>> v;
            for (int p : probs) v.push_back(sweep_task<bf16, bf16>(p, l, in, out, with_corr));
            op.kind = kSweepBB;
            if ((rc = make_list(v, tiles, op.s_bb))) return rc;
            op.s_bb.vec = 4;
            for (const auto& t : v) op.s_bb.vec = std::min(op.s_bb.vec, sweep_vec(t));
            op.s_bb.corr = with_corr ? 1 : 0;
            op.grid = persistent_grid(op.s_bb.total);
        } else if (corr_bf) {
            std::vector<SweepTask<float, bf16>> v;
            for (int p : probs) v.push_back(sweep_task<float, bf16>(p, l, in, out, with_corr));
            op.kind = kSweepFB;
            if ((rc = make_list(v, tiles, op.s_fb))) return rc;
            op.s_fb.vec = 4;
            for (const auto& t : v) op.s_fb.vec = std::min(op.s_fb.vec, sweep_vec(t));
            op.s_fb.corr = with_corr ? 1 : 0;
            op.grid = sweep_grid(op.s_fb, batch_one_block_);
        } else {
            std::vector<SweepTask<float, float>> v;
            for (int p : probs) v.push_back(sweep_task<float, float>(p, l, in, out, with_corr));
            op.kind = kSweepFF;
            if ((rc = make_list(v, tiles, op.s_ff))) return rc;
            op.s_ff.vec = 4;
            for (const auto& t : v) op.s_ff.vec = std::min(op.s_ff.vec, sweep_vec(t));
            op.s_ff.corr = with_corr ? 1 : 0;
            op.grid = sweep_grid(op.s_ff, batch_one_block_);
        }
        cycle.push_back(op);
        return GMG_OK;
    }

    int add_residual(int l, const std::vector<int>& probs, int role, bool restrict_to_next, bool norm)
    {
        std::vector<LaunchOp> ops;
        int rc = res_ops(l, probs, std::vector<int>(probs.size(), role), restrict_to_next, norm, ops);
        if (rc) return rc;
        for (auto& op : ops) cycle.push_back(op);
        return GMG_OK;
    }

    // Cluster form of the bottom of problem M from level lb with `ranks` CTAs: the
    // number of distributed levels (the leading levels of more than kBottomThreads
    // cells) and, in *floats, the shared floats of one CTA; 0 when the form does not
    // apply (no distributed level, a coarsest level too large for one CTA, or more
    // than kClusterMaxFloats floats)
    static int cluster_layout(const ProblemMem& M, int lb, int ranks, int* floats)
    {
        if (ranks < 2 || ranks > kClusterMaxRanks || lb < 1 || lb >= M.L) return 0;
        int nd = 0;
        int64_t off = 0;
        for (int l = lb; l < M.L; ++l) {
            const Geo& g = M.lev[l].g;
            const int64_t n = cells(g);
            if (n > kBottomThreads) {
                if (l != lb + nd || n > kClusterMaxCells) return 0;
                const int64_t rows = (int64_t)g.n[1] * g.n[2];
                off += (int64_t)kDistArrays * ((rows + ranks - 1) / ranks) * g.n[0];
                ++nd;
            } else {
                off += 5 * n;
            }
        }
        if (nd == 0 || nd == M.L - lb || off > kClusterMaxFloats) return 0;
        if (floats) *floats = (int)off;
        return nd;
    }

    int build_cycle()
    {
        const int nprob = (int)P.size();
        int Lmax = 0;
        for (auto& M : P) Lmax = std::max(Lmax, M.L);
        coarse_result_.assign(nprob, std::vector<int>(kMaxLevels, 0));
        // per problem: levels from `stop` down run in one CTA (bottom kernel) when
        // they fit in its shared memory; otherwise only the coarsest level is
        // special (grid sweeps); a problem that does not coarsen runs sweeps only
        stop_.assign(nprob, 0);
        fit_lb_.assign(nprob, -1);
        std::vector<int> bottom(nprob, -1);
        std::vector<int> bottom_nd(nprob, 0);   // > 0: the cluster form with that many distributed levels
        const int ranks = nprob == 1 && forced_ranks_ > 1 ? bottom_cluster_ranks() : 0;
        for (int p = 0; p < nprob; ++p) {
            const ProblemMem& M = P[p];
            if (M.L == 1) continue;
            int64_t acc = 0;
            int lb = -1;
            for (int l = M.L - 1; l >= 1; --l) {
                acc += cells(M.lev[l].g);
                if (acc > kBottomMaxCells) break;
                lb = l;
            }
            fit_lb_[p] = lb;
            const int nd = ranks > 1 ? cluster_layout(M, forced_lb_, ranks, nullptr) : 0;
            if (nd > 0) {
                lb = forced_lb_;
                bottom_nd[p] = nd;
            } else if (lb >= 1 && forced_lb_ > lb && forced_lb_ < M.L) {
                lb = forced_lb_;
            }
            bottom[p] = lb;
            stop_[p] = lb >= 1 ? lb : M.L - 1;
            if (p == 0) {
                bottom_level_ = lb >= 1 ? lb : 0;
                bottom_ranks_ = lb < 1 ? 0 : (nd > 0 ? ranks : 1);
            }
        }
        std::vector<int> pre(kMaxLevels, 0);   // role/buffer of the pre-smoothed iterate per level
        // descent
        for (int l = 0; l + 1 < Lmax; ++l) {
            std::vector<int> probs;
            for (int p = 0; p < nprob; ++p)
                if (l < stop_[p]) probs.push_back(p);
            if (probs.empty()) continue;
            int cur = l == 0 ? 0 : -1;
            for (int s = 0; s < opt.nu1; ++s) {
                const int out = next_out(l, cur < 0 ? (l == 0 ? 0 : 1) : cur);
                int rc = add_sweeps(l, probs, cur, out, false);
                if (rc) return rc;
                cur = out;
            }
            pre[l] = cur;
            int rc = add_residual(l, probs, cur, true, false);
            if (rc) return rc;
        }
        res_role.assign(nprob, 0);
        {
            std::vector<BottomTask<float>> bf;
            std::vector<BottomTask<bf16>> bb;
            size_t smem = 0;
            int cluster_ranks = 1;
            std::vector<int> single;
            std::vector<std::vector<int>> big(kMaxLevels);   // by coarsest level index
            for (int p = 0; p < nprob; ++p) {
                const ProblemMem& M = P[p];
                if (M.L == 1) {
                    single.push_back(p);
                    continue;
                }
                if (bottom[p] < 1) {
                    big[M.L - 1].push_back(p);
                    continue;
                }
                const int lb = bottom[p];
                BottomTask<float> t{};
                t.nlev = M.L - lb;
                t.nd = bottom_nd[p];
                t.ranks = t.nd > 0 ? ranks : 1;
                int off = 0;
                for (int k = 0; k < t.nlev; ++k) {
                    const LevelMem& Lm = M.lev[lb + k];
                    BottomLevel& B = t.lev[k];
                    B.g = Lm.g;
                    for (int d = 0; d < 3; ++d) B.cf[d] = Lm.cf[d];
                    B.bx = Lm.beta[0];
                    B.by = Lm.beta[1];
                    B.bz = Lm.beta[2];
                    B.off = off;
                    B.walls_zeroed = lb + k > 0;   // coarse faces are built with walls read as 0
                    B.inv_nx = 1.0f / (float)Lm.g.n[0];
                    B.inv_nxy = 1.0f / (float)(Lm.g.n[0] * Lm.g.n[1]);
                    if (k < t.nd) {                // rows split over the cluster's CTAs
                        const int rows = Lm.g.n[1] * Lm.g.n[2];
                        B.cpr = (rows + t.ranks - 1) / t.ranks * Lm.g.n[0];
                        B.inv_cpr = 1.0f / (float)B.cpr;
                        off += kDistArrays * B.cpr;
                    } else {
                        off += 5 * (int)cells(Lm.g);
                    }
                }
                if (t.nd > 0) cluster_ranks = t.ranks;
                smem = std::max(smem, sizeof(float) * (size_t)off);
                t.b = M.lev[lb].b;
                t.nu1 = opt.nu1;
                t.nu2 = opt.nu2;
                t.nu_c = opt.nu_c;
                t.ctl = M.ctl;
                t.pinv = M.pinv;
                coarse_result_[p][lb] = 0;
                if (bf16_coarse) {
                    BottomTask<bf16> tb{};
                    tb.nlev = t.nlev;
                    tb.nd = t.nd;
                    tb.ranks = t.ranks;
                    for (int k = 0; k < t.nlev; ++k) tb.lev[k] = t.lev[k];
                    tb.b = t.b;
                    tb.out = static_cast<bf16*>(M.lev[lb].buf[0]);
                    tb.nu1 = t.nu1;
                    tb.nu2 = t.nu2;
                    tb.nu_c = t.nu_c;
                    tb.ctl = t.ctl;
                    tb.pinv = t.pinv;
                    bb.push_back(tb);
                } else {
                    t.out = static_cast<float*>(M.lev[lb].buf[0]);
                    bf.push_back(t);
                }
            }
            if (!bf.empty()) {
                LaunchOp op;
                op.kind = kBottomF;
                op.bot_f = upload(bf);
                op.n = (int)bf.size();
                op.smem = smem;
                op.ranks = cluster_ranks;
                if (!op.bot_f) return fail(GMG_ERR_CUDA, "upload failed");
                cycle.push_back(op);
            }
            if (!bb.empty()) {
                LaunchOp op;
                op.kind = kBottomB;
                op.bot_b = upload(bb);
                op.n = (int)bb.size();
                op.smem = smem;
                op.ranks = cluster_ranks;
                if (!op.bot_b) return fail(GMG_ERR_CUDA, "upload failed");
                cycle.push_back(op);
            }
            // coarsest levels too large for one CTA: projection, then nu_c grid sweeps
            for (int l = 1; l < kMaxLevels; ++l) {
                if (big[l].empty()) continue;
                std::vector<LevelProjTask> lp;
                for (int p : big[l]) {
                    const LevelMem& Lm = P[p].lev[l];
                    lp.push_back(LevelProjTask{Lm.g, Lm.beta[0], Lm.beta[1], Lm.beta[2], Lm.b, P[p].ctl});
                }
                LaunchOp op;
                op.kind = kProjLevel;
                op.lp = upload(lp);
                op.n = (int)lp.size();
                if (!op.lp) return fail(GMG_ERR_CUDA, "upload failed");
                cycle.push_back(op);
                int cur = -1;
                for (int s = 0; s < opt.nu_c; ++s) {
                    const int out = next_out(l, cur < 0 ? 1 : cur);
                    int rc = add_sweeps(l, big[l], cur, out, false);
                    if (rc) return rc;
                    cur = out;
                }
                for (int p : big[l]) coarse_result_[p][l] = cur;
            }
            if (!single.empty()) {
                int cur = 0;
                for (int s = 0; s < opt.nu_c; ++s) {
                    const int out = next_out(0, cur);
                    int rc = add_sweeps(0, single, cur, out, false);
                    if (rc) return rc;
                    cur = out;
                }
                for (int p : single) res_role[p] = cur;
            }
        }
        // ascent
        for (int l = Lmax - 2; l >= 0; --l) {
            std::vector<int> probs;
            for (int p = 0; p < nprob; ++p)
                if (l < stop_[p]) probs.push_back(p);
            if (probs.empty()) continue;
            int cur = pre[l];
            // the correction: folded into the first post-sweep, or (tuned) its own pass
            const bool separate = corr_separable(l) && cur >= 0 &&
                                  tuned_zchunk(kTuneCorrForm, P[0].lev[l].g) == kCorrSeparate;
            if (separate) {
                LaunchOp op;
                op.kind = kProlong;
                op.pro = prolong_task(0, l, cur);
                cycle.push_back(op);
            }
            for (int s = 0; s < opt.nu2; ++s) {
                const int out = next_out(l, cur < 0 ? (l == 0 ? 0 : 1) : cur);
                int rc = add_sweeps(l, probs, cur, out, s == 0 && !separate);
                if (rc) return rc;
                cur = out;
            }
            for (int p : probs) {
                coarse_result_[p][l] = cur;
                if (l == 0) res_role[p] = cur;
            }
        }
        // fine residual norm of the candidate, then the control rule: for one
        // problem on the z-marching residual, inside that launch (its last block)
        {
            std::vector<int> probs(nprob);
            for (int p = 0; p < nprob; ++p) probs[p] = p;
            std::vector<LaunchOp> ops;
            int rc = res_ops(0, probs, res_role, false, true, ops);
            if (rc) return rc;
            const bool fold = nprob == 1 && ops.size() == 1 && ops[0].kind == kResF && ops[0].r_f.march;
            if (fold) {
                if (!arrivals_) {
                    arrivals_ = dalloc<unsigned>(1);
                    if (!arrivals_ || cudaMemset(arrivals_, 0, sizeof(unsigned)) != cudaSuccess)
                        return fail(GMG_ERR_CUDA, "arrival counter allocation failed");
                }
                ops[0].r_f.ctl_tasks = cycle_ctl;
                ops[0].r_f.nctl = nprob;
                ops[0].r_f.arrivals = arrivals_;
            }
            for (auto& op : ops) cycle.push_back(op);
            if (!fold) {
                LaunchOp c;
                c.kind = kControl;
                c.ctl = cycle_ctl;
                c.n = nprob;
                cycle.push_back(c);
            }
        }
        return GMG_OK;
    }

    cudaError_t launch(const LaunchOp& op)
    {
        ++launches;
        switch (op.kind) {
        case kSweepFF: return launch_sweep(op.s_ff, op.grid, stream);
        case kSweepFB: return launch_sweep(op.s_fb, op.grid, stream);
        case kSweepBB: return launch_sweep(op.s_bb, op.grid, stream);
        case kResF: return launch_residual(op.r_f, op.grid, stream);
        case kResB: return launch_residual(op.r_b, op.grid, stream);
        case kBottomF:
            return op.ranks > 1 ? launch_bottom_cluster(op.bot_f, op.n, op.ranks, op.smem, stream)
                                : launch_bottom(op.bot_f, op.n, op.smem, stream);
        case kBottomB:
            return op.ranks > 1 ? launch_bottom_cluster(op.bot_b, op.n, op.ranks, op.smem, stream)
                                : launch_bottom(op.bot_b, op.n, op.smem, stream);
        case kProjLevel: return launch_project_level(op.lp, op.n, stream);
        case kControl: return launch_control_cycle(op.ctl, op.n, stream);
        case kProlong: return launch_prolong_rows(op.pro, stream);
        }
        return cudaErrorInvalidValue;
    }

    cudaError_t run_cycle_eager()
    {
        for (const LaunchOp& op : cycle) {
            cudaError_t e = launch(op);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }

    cudaError_t ensure_graph()
    {
        if (graph_exec) return cudaSuccess;
        cudaStream_t cap;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaStream_t saved = stream;
            const long long counted = launches;
            stream = cap;
            cudaError_t le = run_cycle_eager();
            stream = saved;
            launches = counted;
            e = cudaStreamEndCapture(cap, &graph);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&graph_exec, graph, 0);
        cudaStreamDestroy(cap);
        return e;
    }

    cudaError_t run_cycle()
    {
        if (opt.use_graph) {
            cudaError_t e = ensure_graph();
            if (e != cudaSuccess) return e;
            launches += (long long)cycle.size();
            return cudaGraphLaunch(graph_exec, stream);
        }
        return run_cycle_eager();
    }

    // ---------------------------------------------------------------- coefficients

    int set_coeffs(const float* const* bx, const float* const* by, const float* const* bz)
    {
        NvtxRange range("gmg_set_coeffs");
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "gmg_set_coeffs: pending error from an earlier call");
        int* bad = dalloc<int>(1);
        if (!bad) return fail(GMG_ERR_CUDA, "out of device memory");
        const char* step = "memset";
        e = cudaMemsetAsync(bad, 0, sizeof(int), stream);
        for (size_t p = 0; p < P.size() && e == cudaSuccess; ++p) {
            ProblemMem& M = P[p];
            const size_t bytes = sizeof(float) * (size_t)M.n0;
            const float* src[3] = {bx[p], by[p], bz[p]};
            step = "coefficient copy";
            for (int d = 0; d < 3 && e == cudaSuccess; ++d)
                e = cudaMemcpyAsync(M.lev[0].beta[d], src[d], bytes, cudaMemcpyDeviceToDevice, stream);
            if (e == cudaSuccess) {
                step = "coefficient check";
                e = launch_check_coeffs(M.n0, M.lev[0].beta[0], M.lev[0].beta[1], M.lev[0].beta[2], bad, stream);
            }
            step = "coarsening";
            for (int l = 0; l + 1 < M.L && e == cudaSuccess; ++l)
                e = launch_coarsen_coeffs(M.lev[l].g, M.lev[l].cf, M.lev[l].beta[0], M.lev[l].beta[1],
                                          M.lev[l].beta[2], M.lev[l + 1].beta[0], M.lev[l + 1].beta[1],
                                          M.lev[l + 1].beta[2], opt.coarse_op == GMG_COARSE_OP_GALERKIN, stream);
            if (e == cudaSuccess) {
                step = "active mask";
                e = launch_active_mask(M.g0, M.lev[0].beta[0], M.lev[0].beta[1], M.lev[0].beta[2], M.mask, stream);
            }
            if (e == cudaSuccess && M.pinv) {
                step = "coarsest pseudo-inverse";
                const LevelMem& C = M.lev[M.L - 1];
                e = build_dense_pinv(C.g, C.beta[0], C.beta[1], C.beta[2], M.pinv, stream);
            }
            if (e != cudaSuccess) return fail(GMG_ERR_CUDA, "gmg_set_coeffs (problem %zu, %s): %s", p, step,
                                              cudaGetErrorString(e));
        }
        int hbad = 0;
        step = "readback";
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        drop(bad);
        if (e != cudaSuccess) return fail(GMG_ERR_CUDA, "gmg_set_coeffs (%s): %s", step, cudaGetErrorString(e));
        if (hbad) return fail(GMG_ERR_ARG, "face coefficients must be finite and >= 0");
        coeffs_set = true;
        if (opt.autotune && !tuned_) {
            tuned_ = true;
            const int rc = tune();
            if (rc != GMG_OK) return rc;
        }
        return GMG_OK;
    }

    // ---------------------------------------------------------------- autotuner

    // mean time of one call of f after two warm-up calls (ms), or a huge value on error
    float time_ms(const std::function<cudaError_t()>& f, int reps)
    {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaError_t e = f();
        if (e == cudaSuccess) e = f();
        if (e == cudaSuccess) e = cudaEventRecord(a, stream);
        for (int i = 0; i < reps && e == cudaSuccess; ++i) e = f();
        if (e == cudaSuccess) e = cudaEventRecord(b, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 1e30f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return e == cudaSuccess ? ms / reps : 1e30f;
    }

    // free the launch lists of the current cycle plan and its graph
    void reset_cycle()
    {
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        graph_exec = nullptr;
        graph = nullptr;
        for (const LaunchOp& op : cycle) {
            const void* ptrs[] = {op.s_ff.tasks, op.s_ff.tile_off, op.s_fb.tasks, op.s_fb.tile_off, op.s_bb.tasks,
                                  op.s_bb.tile_off, op.r_f.tasks, op.r_f.tile_off, op.r_b.tasks, op.r_b.tile_off,
                                  op.bot_f, op.bot_b, op.lp};
            for (const void* q : ptrs)
                if (q) drop(q);
        }
        cycle.clear();
    }

    // a control state under which timed V-cycles never finish: tolerance below
    // zero, no divergence floor, no cycle limit, no history
    cudaError_t upload_timing_ctl()
    {
        for (size_t p = 0; p < P.size(); ++p) {
            Ctl c = initial_ctl(P[p], -1.0);
            c.omega_min = -1.0;
            c.r_prev = 1.0;
            c.bnorm = 1.0;
            c.max_cycles = 1 << 30;
            c.hist_cap = 0;
            ctl_host[p] = c;
        }
        return cudaMemcpy(ctl_dev, ctl_host, sizeof(Ctl) * P.size(), cudaMemcpyHostToDevice);
    }

    int tune()
    {
        NvtxRange range("gmg autotune");
        // timed launches run on zeros: right-hand sides and iterates of every level
        for (auto& M : P)
            for (int l = 0; l < M.L; ++l) {
                const size_t n = (size_t)cells(M.lev[l].g);
                const size_t es = (l > 0 && bf16_coarse) ? sizeof(bf16) : sizeof(float);
                cudaMemsetAsync(M.lev[l].b, 0, n * sizeof(float), stream);
                for (int r = 0; r < 3; ++r)
                    if (M.lev[l].buf[r]) cudaMemsetAsync(M.lev[l].buf[r], 0, n * es, stream);
            }
        if (upload_timing_ctl() != cudaSuccess) return fail(GMG_ERR_CUDA, "autotune: control upload failed");
        // 1) z-chunk depth of each grid-kernel level, per kernel kind
        for (size_t p = 0; p < P.size(); ++p) {
            const ProblemMem& M = P[p];
            // a single problem may move the bottom's start down (step 2), which turns
            // the levels above it into grid levels: tune every level but the coarsest
            const int grid_levels = P.size() == 1 ? std::max(stop_[p], M.L - 1) : stop_[p];
            for (int l = 0; l < grid_levels; ++l) {
                if (l > 0 && bf16_coarse) continue;   // BF16 levels keep the heuristic depth
                const Geo g = M.lev[l].g;
                std::vector<int> cand;
                for (int zc : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256})
                    if (zc < g.n[2]) cand.push_back(zc);
                cand.push_back(g.n[2]);
                const int in = l == 0 ? 0 : 1, out = l == 0 ? 1 : 0;
                for (int kind : {kTuneSweep, kTuneSweepCorr, kTuneResidual}) {
                    if (tuned_zchunk(kind, g)) continue;
                    if (kind == kTuneResidual && !res_marches(g, true)) continue;
                    float best = 1e30f;
                    int best_zc = 0;
                    int last_chunks = -1;
                    for (int zc : cand) {
                        const SweepTiling st = sweep_tiling(g, kind, zc);
                        const int chunks = kind == kTuneResidual ? march_tiling(g, zc).tz : st.nchunks;
                        if (chunks == last_chunks) continue;   // same launch as the previous candidate
                        last_chunks = chunks;
                        float ms;
                        if (kind == kTuneResidual) {
                            ResTask<float> t = res_task<float>((int)p, l, in, true, nullptr);
                            const ResTiling rt = march_tiling(g, zc);
                            t.tiles_z = rt.tz;
                            t.zchunk = rt.zchunk;
                            TaskList<ResTask<float>> tl{};
                            tl.ntasks = 1;
                            tl.total = (int)rt.tiles();
                            tl.single = t;
                            tl.march = 1;
                            ms = time_ms([&] { return launch_residual(tl, residual_grid(tl), stream); }, 5);
                        } else if (kind == kTuneSweepCorr && bf16_coarse) {
                            SweepTask<float, bf16> t = sweep_task<float, bf16>((int)p, l, in, out, true);
                            t.zchunk = st.zchunk;
                            t.nchunks = st.nchunks;
                            TaskList<SweepTask<float, bf16>> tl{};
                            tl.ntasks = 1;
                            tl.total = (int)st.tiles();
                            tl.single = t;
                            tl.vec = sweep_vec(t);
                            tl.corr = 1;
                            ms = time_ms([&] { return launch_sweep(tl, sweep_grid(tl), stream); }, 5);
                        } else {
                            SweepTask<float, float> t =
                                sweep_task<float, float>((int)p, l, in, out, kind == kTuneSweepCorr);
                            t.zchunk = st.zchunk;
                            t.nchunks = st.nchunks;
                            TaskList<SweepTask<float, float>> tl{};
                            tl.ntasks = 1;
                            tl.total = (int)st.tiles();
                            tl.single = t;
                            tl.vec = sweep_vec(t);
                            tl.corr = kind == kTuneSweepCorr ? 1 : 0;
                            ms = time_ms([&] { return launch_sweep(tl, sweep_grid(tl), stream); }, 5);
                        }
                        if (ms < best) {
                            best = ms;
                            best_zc = zc;
                        }
                    }
                    if (best_zc > 0) {
                        std::lock_guard<std::mutex> lock(g_tune_mutex);
                        g_tuned_zchunk[tune_key(kind, g)] = best_zc;
                    }
                }
                // the correction folded into the first post-sweep against its own pass plus a plain sweep
                if (l + 1 < M.L && corr_separable(l) && !tuned_zchunk(kTuneCorrForm, g)) {
                    SweepTask<float, float> tf = sweep_task<float, float>((int)p, l, in, out, true);
                    TaskList<SweepTask<float, float>> lf{};
                    lf.ntasks = 1;
                    lf.total = (int)sweep_tiling(g, kTuneSweepCorr).tiles();
                    lf.single = tf;
                    lf.vec = sweep_vec(tf);
                    lf.corr = 1;
                    SweepTask<float, float> tp = sweep_task<float, float>((int)p, l, in, out, false);
                    TaskList<SweepTask<float, float>> lp{};
                    lp.ntasks = 1;
                    lp.total = (int)sweep_tiling(g, kTuneSweep).tiles();
                    lp.single = tp;
                    lp.vec = sweep_vec(tp);
                    const ProlongTask pt = prolong_task((int)p, l, in);
                    const float fused =
                        time_ms([&] { return launch_sweep(lf, sweep_grid(lf), stream); }, 5);
                    const float split = time_ms([&] {
                        cudaError_t e2 = launch_prolong_rows(pt, stream);
                        return e2 == cudaSuccess ? launch_sweep(lp, sweep_grid(lp), stream) : e2;
                    }, 5);
                    std::lock_guard<std::mutex> lock(g_tune_mutex);
                    g_tuned_zchunk[tune_key(kTuneCorrForm, g)] = split < fused ? kCorrSeparate : kCorrFused;
                }
            }
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "autotune (z-chunks)");
        // 2) where the bottom starts and in which form (one problem): time whole
        // V-cycle graphs of each candidate
        forced_lb_ = 0;
        forced_ranks_ = 1;
        reset_cycle();
        if (upload_ctl_tasks() != GMG_OK) return fail(GMG_ERR_CUDA, "autotune: control task upload failed");
        int rc = build_cycle();
        if (rc != GMG_OK) return rc;
        const std::vector<int> lb_key = {P[0].g0.n[0], P[0].g0.n[1], P[0].g0.n[2], P[0].g0.per[0], P[0].g0.per[1],
                                         P[0].g0.per[2], opt.coarsen, opt.n_min, opt.precision, opt.nu_c,
                                         opt.coarse_mode + 2 * opt.coarse_op};
        BottomChoice cached{0, 1};
        {
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            auto it = g_tuned_lb.find(lb_key);
            if (it != g_tuned_lb.end()) cached = it->second;
        }
        std::vector<BottomChoice> cand;   // one-CTA starts from the smallest fit; cluster starts
        if (P.size() == 1 && P[0].L > 1 && cached.level == 0) {
            if (fit_lb_[0] >= 1)
                for (int lb = fit_lb_[0]; lb < P[0].L; ++lb) cand.push_back({lb, 1});
            const int ranks = bottom_cluster_ranks();
            for (int lb = 1; lb < P[0].L; ++lb)
                if (cluster_layout(P[0], lb, ranks, nullptr) > 0) cand.push_back({lb, ranks});
        }
        if (P.size() == 1 && cached.level > 0) {
            forced_lb_ = cached.level;
            forced_ranks_ = cached.ranks;
            reset_cycle();
            if ((rc = build_cycle()) != GMG_OK) return rc;
        } else if (cand.size() > 1) {
            std::vector<float> ms(cand.size());
            float best = 1e30f;
            for (size_t i = 0; i < cand.size(); ++i) {
                forced_lb_ = cand[i].level;
                forced_ranks_ = cand[i].ranks;
                reset_cycle();
                if ((rc = build_cycle()) != GMG_OK) return rc;
                if (upload_timing_ctl() != cudaSuccess) return fail(GMG_ERR_CUDA, "autotune: control upload failed");
                ms[i] = time_ms([&] { return run_cycle(); }, 5);
                best = std::min(best, ms[i]);
            }
            // within 2 % of the fastest (the spread of these short timings) take the
            // bottom that starts highest, cluster before one CTA: the fewest launches
            // per cycle, so the choice does not flip with timing noise
            BottomChoice best_c{0, 1};
            for (size_t i = 0; i < cand.size(); ++i) {
                if (ms[i] > 1.02f * best) continue;
                const BottomChoice& c = cand[i];
                if (best_c.level == 0 || c.level < best_c.level ||
                    (c.level == best_c.level && c.ranks > best_c.ranks))
                    best_c = c;
            }
            forced_lb_ = best_c.level;
            forced_ranks_ = best_c.ranks;
            {
                std::lock_guard<std::mutex> lock(g_tune_mutex);
                g_tuned_lb[lb_key] = best_c;
            }
            reset_cycle();
            if ((rc = build_cycle()) != GMG_OK) return rc;
        }
        // 3) a batch: z-chunks of its batched levels.  The depths tuned per geometry
        // above fit a problem that runs alone, which splits its few columns into many
        // short chunks; one launch over many problems has columns enough, and fewer,
        // deeper chunks pay less for halo planes and pipeline starts.  Whole V-cycles
        // are timed with the per-geometry depths and with each level's columns cut
        // into the fewest chunks that give its launch one chunk a column or 1, 2 or
        // 4 waves of blocks, each on the persistent grid and with one block per tile.
        if (P.size() > 1) {
            const std::pair<int, int> key{(int)P.size(), batch_hash()};
            int cached_choice = -1;
            {
                std::lock_guard<std::mutex> lock(g_tune_mutex);
                auto it = g_tuned_batch.find(key);
                if (it != g_tuned_batch.end()) cached_choice = it->second;
            }
            const int slots = sm_count() * 3;
            // choice = 2 (target + 1) + (1 if one block per tile)
            std::vector<int> choices;
            if (cached_choice >= 0) {
                choices = {cached_choice};
            } else {
                for (int target : {-1, 1, slots, 2 * slots, 4 * slots})
                    for (int one : {0, 1}) choices.push_back(2 * (target + 1) + one);
            }
            float best = 1e30f;
            int best_choice = 0;
            for (int choice : choices) {
                if (choices.size() == 1) {
                    best_choice = choice;
                    break;
                }
                batch_target_ = choice / 2 - 1;
                batch_one_block_ = choice % 2 == 1;
                reset_cycle();
                if (upload_ctl_tasks() != GMG_OK) return fail(GMG_ERR_CUDA, "autotune: control task upload failed");
                if ((rc = build_cycle()) != GMG_OK) return rc;
                if (upload_timing_ctl() != cudaSuccess) return fail(GMG_ERR_CUDA, "autotune: control upload failed");
                const float ms = time_ms([&] { return run_cycle(); }, 5);
                if (ms < best) {
                    best = ms;
                    best_choice = choice;
                }
            }
            batch_target_ = best_choice / 2 - 1;
            batch_one_block_ = best_choice % 2 == 1;
            {
                std::lock_guard<std::mutex> lock(g_tune_mutex);
                g_tuned_batch[key] = best_choice;
            }
            reset_cycle();
            if (upload_ctl_tasks() != GMG_OK) return fail(GMG_ERR_CUDA, "autotune: control task upload failed");
            if ((rc = build_cycle()) != GMG_OK) return rc;
        }
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e, "autotune");
        return GMG_OK;
    }

    // ---------------------------------------------------------------- solves

    Ctl initial_ctl(const ProblemMem& M, double tol) const
    {
        Ctl c{};
        c.omega = opt.omega0;
        c.omega_min = opt.omega_min;
        c.shrink = opt.shrink;
        c.grow = opt.grow;
        c.tol = tol;
        c.max_cycles = opt.max_cycles;
        c.res_role = res_role[&M - P.data()];
        c.status = kRunning;
        c.done = 0;
        c.hist_cap = opt.max_cycles;
        c.hist_res = M.hist_res;
        c.hist_omega = M.hist_omega;
        c.hist_acc = M.hist_acc;
        c.outer_status = kRunning;
        return c;
    }

    // control blocks to the host; a pipelined kernel that gave up waiting for its
    // plane copies turns into cudaErrorLaunchTimeout
    cudaError_t read_ctl()
    {
        cudaError_t e = cudaMemcpyAsync(ctl_host, ctl_dev, sizeof(Ctl) * P.size(), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess && fault_dev)
            e = cudaMemcpyAsync(fault_host, fault_dev, sizeof(int), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e == cudaSuccess && fault_dev && *fault_host) {
            *fault_host = 0;
            cudaMemsetAsync(fault_dev, 0, sizeof(int), stream);   // reported once
            e = cudaErrorLaunchTimeout;
        }
        return e;
    }

    bool all_done() const
    {
        for (size_t p = 0; p < P.size(); ++p)
            if (!ctl_host[p].done) return false;
        return true;
    }

    // projection of sigma to zero mean over active cells + iterate copy-in
    template <class TS>
    cudaError_t project(const TS* const* sigma, const TS* const* p_in, bool to64, TS* const* p64_dst)
    {
        std::vector<ProjTask<TS>> v(P.size());
        std::vector<int64_t> tiles(P.size());
        for (size_t p = 0; p < P.size(); ++p) {
            ProblemMem& M = P[p];
            ProjTask<TS> t{};
            t.n = M.n0;
            t.mask = M.mask;
            t.sigma = sigma[p];
            t.b32 = to64 ? nullptr : M.lev[0].b;
            t.b64 = to64 ? M.b64 : nullptr;
            t.p_in = p_in[p];
            t.p32 = to64 ? nullptr : static_cast<float*>(M.lev[0].buf[0]);
            t.p64 = to64 ? reinterpret_cast<double*>(p64_dst[p]) : nullptr;
            t.partials = M.proj_part;
            t.bpartials = M.bpart;
            t.tiles = M.elem_tiles;
            t.ctl = M.ctl;
            v[p] = t;
            tiles[p] = M.elem_tiles;
        }
        TaskList<ProjTask<TS>> tl;
        if (make_list(v, tiles, tl)) return cudaErrorMemoryAllocation;
        launches += 3;
        cudaError_t e = launch_project_sum(tl, persistent_grid(tl.total), stream);
        if (e == cudaSuccess) e = launch_project_finalize(init_ctl, (int)P.size(), stream);
        if (e == cudaSuccess) e = launch_project_apply(tl, persistent_grid(tl.total), stream);
        if (tl.tasks) {   // the lists are rebuilt per solve: free them after the launches ran
            cudaStreamSynchronize(stream);
            drop(tl.tasks);
            drop(tl.tile_off);
        }
        return e;
    }

    template <class T>
    void drop(const T* ptr)
    {
        auto it = std::find(allocs.begin(), allocs.end(), (void*)ptr);
        if (it != allocs.end()) {
            cudaFree(*it);
            allocs.erase(it);
        }
    }

    template <class TP, class TD>
    cudaError_t gauge(TD* const* dst, bool fine64)
    {
        std::vector<GaugeTask<TP, TD>> v(P.size());
        std::vector<int64_t> tiles(P.size());
        for (size_t p = 0; p < P.size(); ++p) {
            ProblemMem& M = P[p];
            GaugeTask<TP, TD> t{};
            t.n = M.n0;
            t.mask = M.mask;
            if (fine64) {
                t.buf[0] = t.buf[1] = t.buf[2] = reinterpret_cast<TP*>(dst[p]);
                t.rot = nullptr;
            } else {
                for (int r = 0; r < 3; ++r) t.buf[r] = static_cast<TP*>(M.lev[0].buf[r]);
                t.rot = &M.ctl->rot;
            }
            t.dst = dst[p];
            t.partials = M.gauge_part;
            t.tiles = M.elem_tiles;
            t.ctl = M.ctl;
            v[p] = t;
            tiles[p] = M.elem_tiles;
        }
        TaskList<GaugeTask<TP, TD>> tl;
        if (make_list(v, tiles, tl)) return cudaErrorMemoryAllocation;
        launches += 3;
        cudaError_t e = launch_gauge_sum(tl, persistent_grid(tl.total), stream);
        if (e == cudaSuccess) e = launch_gauge_finalize(gauge_ctl, (int)P.size(), stream);
        if (e == cudaSuccess) e = launch_gauge_apply(tl, persistent_grid(tl.total), stream);
        if (tl.tasks) {
            cudaStreamSynchronize(stream);
            drop(tl.tasks);
            drop(tl.tile_off);
        }
        return e;
    }

    // initial residual of the copied-in iterate, then the control init
    cudaError_t init_control()
    {
        std::vector<int> probs(P.size());
        for (size_t p = 0; p < P.size(); ++p) probs[p] = (int)p;
        std::vector<LaunchOp> ops;
        if (res_ops(0, probs, std::vector<int>(P.size(), 0), false, true, ops)) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaSuccess;
        for (const LaunchOp& op : ops)
            if (e == cudaSuccess) e = launch(op);
        ++launches;
        if (e == cudaSuccess) e = launch_control_init(init_ctl, (int)P.size(), stream);
        bool uploaded = false;
        for (const LaunchOp& op : ops) uploaded |= op.r_f.tasks != nullptr;
        if (uploaded) {   // the lists are built per solve: free them once the launches ran
            cudaStreamSynchronize(stream);
            for (const LaunchOp& op : ops) {
                if (op.r_f.tasks) drop(op.r_f.tasks);
                if (op.r_f.tile_off) drop(op.r_f.tile_off);
            }
        }
        return e;
    }

    cudaError_t upload_ctl(double tol)
    {
        for (size_t p = 0; p < P.size(); ++p) ctl_host[p] = initial_ctl(P[p], tol);
        return cudaMemcpyAsync(ctl_dev, ctl_host, sizeof(Ctl) * P.size(), cudaMemcpyHostToDevice, stream);
    }

    // test hook (gmg_test_poison_omega): write NaN into every problem's device
    // relaxation factor, ordered on the stream between two V-cycles
    cudaError_t poison_omega()
    {
        static const double nan_value = std::nan("");
        for (size_t p = 0; p < P.size(); ++p) {
            cudaError_t e = cudaMemcpyAsync(&P[p].ctl->omega, &nan_value, sizeof(double), cudaMemcpyHostToDevice,
                                            stream);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }

    // V-cycles to queue before the next status read: as many as the contraction
    // seen since the last read (r0, c0: residual and cycle count then) predicts the
    // slowest unfinished problem still needs, rounded down and at least 1, at most
    // cycles_per_sync; 2 while no contraction has been seen.  A cycle queued after
    // every problem finished still costs one launch per kernel of the graph (the
    // kernels see the done flag and return); an extra status read costs less.
    int cycles_to_queue(const std::vector<double>& r0, const std::vector<int>& c0) const
    {
        const int cap = std::max(1, opt.cycles_per_sync);
        int q = 0;
        bool unknown = false;
        for (size_t p = 0; p < P.size(); ++p) {
            const Ctl& c = ctl_host[p];
            if (c.done) continue;
            const int ran = c.cycles - c0[p];
            if (ran <= 0 || !(r0[p] > 0.0) || !(c.r_prev > 0.0) || !(c.bnorm > 0.0) || !(c.tol > 0.0)) {
                unknown = true;
                continue;
            }
            const double rho = std::pow(c.r_prev / r0[p], 1.0 / ran);
            if (!(rho < 0.95)) {                 // slow, or rejected cycles: a full batch
                q = cap;
                continue;
            }
            const double need = std::log(c.tol * c.bnorm / c.r_prev) / std::log(rho);
            q = std::max(q, need >= (double)cap ? cap : (int)std::floor(need));
        }
        if (unknown) q = std::max(q, 2);
        return std::min(cap, std::max(1, q));
    }

    // cycles until every problem is done; returns the CUDA status
    cudaError_t iterate()
    {
        const int cap = std::max(1, opt.cycles_per_sync);
        std::vector<double> r0(P.size());
        std::vector<int> c0(P.size());
        int queued = 0;
        while (queued <= opt.max_cycles + cap) {
            const int q = cycles_to_queue(r0, c0);
            for (size_t p = 0; p < P.size(); ++p) {
                r0[p] = ctl_host[p].r_prev;
                c0[p] = ctl_host[p].cycles;
            }
            for (int k = 0; k < q; ++k) {
                if (++queued == poison_cycle) {
                    poison_cycle = 0;
                    cudaError_t e = poison_omega();
                    if (e != cudaSuccess) return e;
                }
                cudaError_t e = run_cycle();
                if (e != cudaSuccess) return e;
            }
            cudaError_t e = read_ctl();
            if (e != cudaSuccess) return e;
            if (all_done()) return cudaSuccess;
        }
        return read_ctl();
    }

    int solve32(const float* const* sigma, float* const* p, double tol, gmg_info* infos)
    {
        NvtxRange range("gmg_solve (FP32 V-cycles)");
        if (!coeffs_set) return fail(GMG_ERR_ARG, "gmg_set_coeffs must precede gmg_solve");
        launches = 0;
        cudaError_t e = upload_ctl(tol);
        if (e == cudaSuccess) e = project<float>(sigma, (const float* const*)p, false, nullptr);
        if (e == cudaSuccess) e = init_control();
        if (e == cudaSuccess) e = read_ctl();
        if (e == cudaSuccess && !all_done()) e = iterate();
        if (e != cudaSuccess) return cuda_fail(e, "gmg_solve");
        // gauge into the caller arrays (skipped for problems with a non-finite source)
        bool any_finite = false;
        for (size_t q = 0; q < P.size(); ++q) any_finite |= ctl_host[q].status != kNonFinite;
        if (any_finite) {
            std::vector<float*> dst(P.size());
            for (size_t q = 0; q < P.size(); ++q) dst[q] = p[q];
            e = gauge<float, float>(dst.data(), false);
            if (e == cudaSuccess) e = read_ctl();
            if (e != cudaSuccess) return cuda_fail(e, "gmg_solve (gauge)");
        }
        int worst = GMG_OK;
        for (size_t q = 0; q < P.size(); ++q) {
            const Ctl& c = ctl_host[q];
            const int st = c.status == kRunning ? kNotConverged : c.status;
            if (infos) {
                gmg_info& inf = infos[q];
                inf.cycles = c.cycles;
                inf.status = st;
                inf.levels = P[q].L;
                inf.outer = 0;
                inf.launches = (int)launches;
                inf.rel_res = c.bnorm > 0.0 ? c.r_prev / c.bnorm : 0.0;
                inf.omega = c.omega;
                inf.bnorm = c.bnorm;
            }
            if (worst == GMG_OK && st != GMG_OK) worst = st;
        }
        last_cycles = ctl_host[0].total_cycles;
        return worst;
    }

    // ---------------------------------------------------------------- PCG

    PcgTask pcg_task(int parity)
    {
        ProblemMem& M = P[0];
        PcgTask t{};
        t.g = M.lev[0].g;
        t.bx = M.lev[0].beta[0];
        t.by = M.lev[0].beta[1];
        t.bz = M.lev[0].beta[2];
        t.b = M.lev[0].b;
        t.x = static_cast<float*>(M.lev[0].buf[0]);
        t.r = pcg_buf[0];
        t.z = pcg_buf[1];
        t.q = pcg_buf[2];
        t.inv_diag = pcg_buf[3];
        t.d_src = pcg_buf[4 + parity];
        t.d_dst = pcg_buf[5 - parity];
        t.part = pcg_part;
        t.zc = kPcgZChunk;
        t.nparts = pcg_blocks(t.g, t.zc);
        t.ctl = M.ctl;
        t.scal = pcg_scal;
        return t;
    }

    cudaError_t pcg_iterations()
    {
        if (!opt.use_graph) {
            cudaError_t e = cudaSuccess;
            for (int i = 0; i < kPcgGraphIters && e == cudaSuccess; ++i) e = launch_pcg_iteration(pcg_task(i & 1), stream);
            launches += 4 * kPcgGraphIters;
            return e;
        }
        if (!pcg_exec) {
            cudaStream_t cap;
            cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
            if (e != cudaSuccess) return e;
            cudaGraph_t gr = nullptr;
            e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t le = cudaSuccess;
                for (int i = 0; i < kPcgGraphIters && le == cudaSuccess; ++i) le = launch_pcg_iteration(pcg_task(i & 1), cap);
                e = cudaStreamEndCapture(cap, &gr);
                if (le != cudaSuccess) e = le;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&pcg_exec, gr, 0);
            if (gr) cudaGraphDestroy(gr);
            cudaStreamDestroy(cap);
            if (e != cudaSuccess) return e;
        }
        launches += 4 * kPcgGraphIters;
        return cudaGraphLaunch(pcg_exec, stream);
    }

    // Jacobi-preconditioned CG on the finest level of problem 0 (the paper's PCG
    // comparison solver): projection of sigma and copy-in of the guess as for
    // gmg_solve, CG iterations in graphs of kPcgGraphIters until the device-side
    // stop test fires, the exit gauge into p.
    int pcg_solve(const float* sigma, float* p, double tol, int max_iter, gmg_info* info)
    {
        NvtxRange range("gmg_pcg_solve");
        if (!coeffs_set) return fail(GMG_ERR_ARG, "gmg_set_coeffs must precede gmg_pcg_solve");
        if (P.size() != 1) return fail(GMG_ERR_ARG, "gmg_pcg_solve: single-problem handles only");
        if (opt.precision == GMG_IR64 || opt.precision == GMG_IR64_FP32)
            return fail(GMG_ERR_ARG, "gmg_pcg_solve: FP32 handles only (precision GMG_FP32 or GMG_FP32_BF16)");
        if (max_iter < 1) return fail(GMG_ERR_ARG, "gmg_pcg_solve: max_iter must be >= 1");
        ProblemMem& M = P[0];
        if (!pcg_buf[0]) {
            for (float*& b : pcg_buf)
                if (!(b = dalloc<float>((size_t)M.n0))) return fail(GMG_ERR_CUDA, "gmg_pcg_solve: out of device memory");
            pcg_part = dalloc<double>(3 * (size_t)pcg_blocks(M.lev[0].g, kPcgZChunk));
            pcg_scal = dalloc<PcgScal>(1);
            if (!pcg_part || !pcg_scal) return fail(GMG_ERR_CUDA, "gmg_pcg_solve: out of device memory");
            if (cudaMemset(pcg_scal, 0, sizeof(PcgScal)) != cudaSuccess) return fail(GMG_ERR_CUDA, "gmg_pcg_solve");
        }
        launches = 0;
        Ctl c = initial_ctl(M, tol);
        c.max_cycles = max_iter;
        c.hist_cap = -1;
        ctl_host[0] = c;
        cudaError_t e = cudaMemcpyAsync(ctl_dev, ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, stream);
        const float* sig[1] = {sigma};
        float* pin[1] = {p};
        if (e == cudaSuccess) e = project<float>(sig, (const float* const*)pin, false, nullptr);
        if (e == cudaSuccess) {
            launches += 2;
            e = launch_pcg_start(pcg_task(0), false, stream);
        }
        if (e == cudaSuccess) e = read_ctl();
        // iterate; a pause (done while running) means the updated residual met tol:
        // restart from the current iterate, where the true residual decides
        int replays = 0, restarts = 0;
        while (e == cudaSuccess) {
            Ctl& h = ctl_host[0];
            if (h.done && h.status != kRunning) break;
            if (h.done) {
                if (++restarts > kPcgMaxRestarts) break;
                h.done = 0;
                e = cudaMemcpyAsync(ctl_dev, ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, stream);
                launches += 2;
                if (e == cudaSuccess) e = launch_pcg_start(pcg_task(0), true, stream);
            } else {
                if ((int64_t)replays++ * kPcgGraphIters > (int64_t)max_iter) break;
                e = pcg_iterations();
            }
            if (e == cudaSuccess) e = read_ctl();
        }
        if (e != cudaSuccess) return cuda_fail(e, "gmg_pcg_solve");
        if (ctl_host[0].status != kNonFinite) {
            e = gauge<float, float>(pin, false);
            if (e == cudaSuccess) e = read_ctl();
            if (e != cudaSuccess) return cuda_fail(e, "gmg_pcg_solve (gauge)");
        }
        const Ctl& r = ctl_host[0];
        const int st = r.status == kRunning ? kNotConverged : r.status;
        if (info) {
            info->cycles = r.cycles;
            info->status = st;
            info->levels = 1;
            info->outer = 0;
            info->launches = (int)launches;
            info->rel_res = r.bnorm > 0.0 ? r.r_prev / r.bnorm : 0.0;
            info->omega = 1.0;
            info->bnorm = r.bnorm;
        }
        return st;
    }

    // ---------------------------------------------------------------- GMG-PCG

    // the multigrid with PCG as its smoother (Table 1's GMG-PCG), problem 0: per
    // level the smoother's work vectors, control block and scalars
    struct SmoothLevel {
        float* v[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};   // r, z, q, D^-1, d0, d1
        double* part = nullptr;
        Ctl* ctl = nullptr;
        PcgScal* scal = nullptr;
    };
    std::vector<SmoothLevel> gp_lev;
    PcgScal* gp_probe = nullptr;                 // scalars of the fine-level residual probe
    const LevelProjTask* gp_proj = nullptr;      // zero-mean projection of the coarsest level
    cudaGraphExec_t gp_exec = nullptr;
    static constexpr double kSmoothEta = 1e-5;  // a smoothing run stops at this fraction of its start

    PcgTask gp_task(int l, int parity)
    {
        ProblemMem& M = P[0];
        const LevelMem& Lm = M.lev[l];
        SmoothLevel& S = gp_lev[l];
        PcgTask t{};
        t.g = Lm.g;
        t.bx = Lm.beta[0];
        t.by = Lm.beta[1];
        t.bz = Lm.beta[2];
        t.b = Lm.b;
        t.x = static_cast<float*>(Lm.buf[0]);
        t.r = S.v[0];
        t.z = S.v[1];
        t.q = S.v[2];
        t.inv_diag = S.v[3];
        t.d_src = S.v[4 + parity];
        t.d_dst = S.v[5 - parity];
        t.part = S.part;
        t.zc = kPcgZChunk;
        t.nparts = pcg_blocks(t.g, t.zc);
        t.ctl = S.ctl;
        t.scal = S.scal;
        return t;
    }

    cudaError_t gp_smooth(int l, int iters, cudaStream_t s)
    {
        if (iters <= 0) return cudaSuccess;
        cudaError_t e = launch_pcg_arm(gp_lev[l].ctl, gp_lev[l].scal, iters, kSmoothEta, 1, s);
        if (e == cudaSuccess) e = launch_pcg_start(gp_task(l, 0), false, s);
        for (int i = 0; i < iters && e == cudaSuccess; ++i) e = launch_pcg_iteration(gp_task(l, i & 1), s);
        return e;
    }

    // one V-cycle on stream s: PCG smoothing, residual and restriction, coarse
    // correction by prolongation, the coarsest right-hand side projected to zero mean
    cudaError_t gp_cycle(cudaStream_t s)
    {
        ProblemMem& M = P[0];
        const int L = M.L;
        cudaStream_t saved = stream;
        stream = s;
        cudaError_t e = cudaSuccess;
        for (int l = 0; l + 1 < L && e == cudaSuccess; ++l) {
            e = gp_smooth(l, opt.nu1, s);
            std::vector<LaunchOp> ops;
            if (e == cudaSuccess && res_ops(l, {0}, {0}, true, false, ops)) e = cudaErrorMemoryAllocation;
            for (const LaunchOp& op : ops)
                if (e == cudaSuccess) e = launch(op);
            if (e == cudaSuccess)
                e = cudaMemsetAsync(M.lev[l + 1].buf[0], 0, sizeof(float) * (size_t)cells(M.lev[l + 1].g), s);
        }
        if (e == cudaSuccess) e = launch_project_level(gp_proj, 1, s);
        if (e == cudaSuccess) e = gp_smooth(L - 1, opt.nu_c, s);
        for (int l = L - 2; l >= 0 && e == cudaSuccess; --l) {
            e = launch_prolong_add(M.lev[l].g, M.lev[l].cf, static_cast<const float*>(M.lev[l + 1].buf[0]),
                                   static_cast<float*>(M.lev[l].buf[0]), s);
            if (e == cudaSuccess) e = gp_smooth(l, opt.nu2, s);
        }
        stream = saved;
        return e;
    }

    int gmg_pcg_solve(const float* sigma, float* p, double tol, gmg_info* info)
    {
        NvtxRange range("gmg_gmgpcg_solve");
        if (!coeffs_set) return fail(GMG_ERR_ARG, "gmg_set_coeffs must precede gmg_gmgpcg_solve");
        if (P.size() != 1) return fail(GMG_ERR_ARG, "gmg_gmgpcg_solve: single-problem handles only");
        if (opt.precision != GMG_FP32) return fail(GMG_ERR_ARG, "gmg_gmgpcg_solve: GMG_FP32 handles only");
        ProblemMem& M = P[0];
        const int L = M.L;
        if (gp_lev.empty()) {
            gp_lev.resize(L);
            for (int l = 0; l < L; ++l) {
                const size_t n = (size_t)cells(M.lev[l].g);
                for (float*& v : gp_lev[l].v)
                    if (!(v = dalloc<float>(n))) return fail(GMG_ERR_CUDA, "gmg_gmgpcg_solve: out of device memory");
                gp_lev[l].part = dalloc<double>(3 * (size_t)pcg_blocks(M.lev[l].g, kPcgZChunk));
                gp_lev[l].ctl = dalloc<Ctl>(1);
                gp_lev[l].scal = dalloc<PcgScal>(1);
                if (!gp_lev[l].part || !gp_lev[l].ctl || !gp_lev[l].scal)
                    return fail(GMG_ERR_CUDA, "gmg_gmgpcg_solve: out of device memory");
                if (cudaMemset(gp_lev[l].ctl, 0, sizeof(Ctl)) != cudaSuccess ||
                    cudaMemset(gp_lev[l].scal, 0, sizeof(PcgScal)) != cudaSuccess)
                    return fail(GMG_ERR_CUDA, "gmg_gmgpcg_solve");
            }
            gp_probe = dalloc<PcgScal>(1);
            const LevelMem& C = M.lev[L - 1];
            gp_proj = upload(std::vector<LevelProjTask>{LevelProjTask{C.g, C.beta[0], C.beta[1], C.beta[2], C.b, nullptr}});
            if (!gp_probe || !gp_proj || cudaMemset(gp_probe, 0, sizeof(PcgScal)) != cudaSuccess)
                return fail(GMG_ERR_CUDA, "gmg_gmgpcg_solve: out of device memory");
        }
        launches = 0;
        Ctl c = initial_ctl(M, tol);
        c.hist_cap = -1;
        ctl_host[0] = c;
        cudaError_t e = cudaMemcpyAsync(ctl_dev, ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, stream);
        const float* sig[1] = {sigma};
        float* pin[1] = {p};
        if (e == cudaSuccess) e = project<float>(sig, (const float* const*)pin, false, nullptr);
        // the fine-level probe: the true residual of the current iterate against |b|
        auto probe = [&](bool first) {
            PcgTask t = gp_task(0, 0);
            t.ctl = M.ctl;
            t.scal = gp_probe;
            launches += 2;
            return launch_pcg_start(t, !first, stream);
        };
        if (e == cudaSuccess) e = probe(true);
        if (e == cudaSuccess) e = read_ctl();
        int cycles = 0;
        while (e == cudaSuccess && !ctl_host[0].done && cycles < opt.max_cycles) {
            if (opt.use_graph) {
                if (!gp_exec) {
                    cudaStream_t cap;
                    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
                    if (e != cudaSuccess) break;
                    cudaGraph_t gr = nullptr;
                    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
                    if (e == cudaSuccess) {
                        const cudaError_t le = gp_cycle(cap);
                        e = cudaStreamEndCapture(cap, &gr);
                        if (le != cudaSuccess) e = le;
                    }
                    if (e == cudaSuccess) e = cudaGraphInstantiate(&gp_exec, gr, 0);
                    if (gr) cudaGraphDestroy(gr);
                    cudaStreamDestroy(cap);
                    if (e != cudaSuccess) break;
                }
                e = cudaGraphLaunch(gp_exec, stream);
            } else {
                e = gp_cycle(stream);
            }
            ++cycles;
            if (e == cudaSuccess) e = probe(false);
            if (e == cudaSuccess) e = read_ctl();
        }
        if (e != cudaSuccess) return cuda_fail(e, "gmg_gmgpcg_solve");
        if (ctl_host[0].status != kNonFinite) {
            e = gauge<float, float>(pin, false);
            if (e == cudaSuccess) e = read_ctl();
            if (e != cudaSuccess) return cuda_fail(e, "gmg_gmgpcg_solve (gauge)");
        }
        const Ctl& r = ctl_host[0];
        const int st = r.status == kRunning ? kNotConverged : r.status;
        if (info) {
            info->cycles = cycles;
            info->status = st;
            info->levels = L;
            info->outer = 0;
            info->launches = (int)launches;
            info->rel_res = r.bnorm > 0.0 ? r.r_prev / r.bnorm : 0.0;
            info->omega = 1.0;
            info->bnorm = r.bnorm;
        }
        return st;
    }

    // FP64 iterative refinement (Sec. 3 cycles inside an FP64 outer loop) for every
    // problem of the engine: each outer step computes r64 = b64 - A p64, runs the
    // FP32 (or BF16-coarse) V-cycles of all unfinished problems together on it,
    // and adds the correction; a problem leaves the loop when its outer residual
    // meets tol (or its inner solve diverged).
    int solve64(const double* const* sigma, double* const* p, double tol, gmg_info* infos)
    {
        NvtxRange range("gmg_solve (FP64 refinement)");
        if (!coeffs_set) return fail(GMG_ERR_ARG, "gmg_set_coeffs must precede gmg_solve");
        const size_t N = P.size();
        launches = 0;
        cudaError_t e = upload_ctl(tol);
        if (e == cudaSuccess) e = project<double>(sigma, (const double* const*)p, true, p);
        // |b64| -> bnorm (partials = nullptr: the residual equals b here)
        if (e == cudaSuccess) {
            std::vector<CtlTask> tv(N);
            for (size_t q = 0; q < N; ++q)
                tv[q] = CtlTask{P[q].ctl, nullptr, 0, P[q].bpart, P[q].elem_tiles, P[q].proj_part, P[q].elem_tiles};
            CtlTask* d = upload(tv);
            if (!d) return fail(GMG_ERR_CUDA, "upload failed");
            e = launch_control_init(d, (int)N, stream);
            ++launches;
            if (e == cudaSuccess) e = read_ctl();
            drop(d);
        }
        if (e != cudaSuccess) return cuda_fail(e, "gmg_solve");
        std::vector<int> outer(N, 0), status(N, kRunning);
        std::vector<char> finished(N, 0);
        std::vector<IrTask> t(N);
        std::vector<ResTiling> rt(N);
        for (size_t q = 0; q < N; ++q) {
            Ctl& c = ctl_host[q];
            ProblemMem& M = P[q];
            if (c.done) {            // zero or non-finite source: settled by the control kernel
                finished[q] = 1;
                status[q] = c.status;
                continue;
            }
            c.outer_bnorm = c.bnorm;   // the outer |b| lives in outer_bnorm
            c.outer_r = 0.0;
            IrTask& ti = t[q];
            ti = IrTask{};
            ti.g = M.g0;
            ti.bx = M.lev[0].beta[0];
            ti.by = M.lev[0].beta[1];
            ti.bz = M.lev[0].beta[2];
            ti.b64 = M.b64;
            ti.p64 = p[q];
            ti.b32 = M.lev[0].b;
            for (int r = 0; r < 3; ++r) ti.ebuf[r] = static_cast<float*>(M.lev[0].buf[r]);
            ti.rot = &M.ctl->rot;
            ti.partials = M.ir_part;
            rt[q] = res_tiling(M.g0);
            ti.tiles_x = rt[q].tx;
            ti.tiles_y = rt[q].ty;
            ti.tiles_z = rt[q].tz;
            ti.ctl = M.ctl;
            ti.scale = nullptr;
        }
        e = cudaMemcpyAsync(ctl_dev, ctl_host, sizeof(Ctl) * N, cudaMemcpyHostToDevice, stream);
        auto outer_residual = [&](size_t q) {
            launches += 2;
            // one norm partial per block of the residual launch
            const int grid = persistent_grid(rt[q].tiles());
            cudaError_t r = launch_ir_residual(t[q], grid, stream);
            if (r == cudaSuccess) r = launch_ir_begin_inner(t[q], grid, tol, opt.ir_inner_rtol, opt.max_cycles, stream);
            return r;
        };
        for (;;) {
            // outer residual and the next inner right-hand side of every unfinished problem
            for (size_t q = 0; q < N && e == cudaSuccess; ++q)
                if (!finished[q]) e = outer_residual(q);
            if (e == cudaSuccess) e = read_ctl();
            if (e != cudaSuccess) break;
            bool any = false;
            for (size_t q = 0; q < N; ++q) {
                if (finished[q]) continue;
                if (ctl_host[q].done) {
                    finished[q] = 1;
                    status[q] = ctl_host[q].outer_status;
                } else {
                    ++outer[q];
                    any = true;
                }
            }
            if (!any) break;
            NvtxRange step("gmg refinement step (inner V-cycles)");
            e = iterate();
            for (size_t q = 0; q < N && e == cudaSuccess; ++q)
                if (!finished[q]) {
                    ++launches;
                    e = launch_ir_update(t[q], stream);
                }
            if (e == cudaSuccess) e = read_ctl();
            if (e != cudaSuccess) break;
            for (size_t q = 0; q < N && e == cudaSuccess; ++q) {
                if (finished[q] || ctl_host[q].status != kDiverged) continue;
                // keep the refinement so far and report the inner divergence
                e = outer_residual(q);
                if (e == cudaSuccess) e = read_ctl();
                status[q] = ctl_host[q].outer_status == kOk ? kOk : kDiverged;
                finished[q] = 1;
            }
            if (e != cudaSuccess) break;
        }
        if (e != cudaSuccess) return cuda_fail(e, "gmg_solve (refinement)");
        {
            std::vector<double*> dst;
            bool any_finite = false;
            for (size_t q = 0; q < N; ++q) {
                dst.push_back(p[q]);
                any_finite |= status[q] != kNonFinite;
            }
            if (any_finite) {
                e = gauge<double, double>(dst.data(), true);
                if (e == cudaSuccess) e = read_ctl();
                if (e != cudaSuccess) return cuda_fail(e, "gmg_solve (gauge)");
            }
        }
        int first_bad = GMG_OK;
        for (size_t q = 0; q < N; ++q) {
            const Ctl& c = ctl_host[q];
            const int st = status[q] == kRunning ? kNotConverged : status[q];
            if (st != kOk && first_bad == GMG_OK) first_bad = st;
            if (infos) {
                gmg_info& info = infos[q];
                info.cycles = c.total_cycles;
                info.status = st;
                info.levels = P[q].L;
                info.outer = outer[q];
                info.launches = (int)launches;
                info.rel_res = c.outer_bnorm > 0.0 ? c.outer_r / c.outer_bnorm : 0.0;
                info.omega = c.omega;
                info.bnorm = c.outer_bnorm;
            }
        }
        last_cycles = ctl_host[0].total_cycles;
        return first_bad;
    }
};

std::mutex g_op_mutex;
struct OpScratch {
    int device = -1;
    double* part = nullptr;
    int cap = 0;
    double* out = nullptr;
};
std::vector<OpScratch> g_op_scratch;

}  // namespace

int gmg::validate_geometry(int nx, int ny, int nz, const int* periodic, std::string& msg)
{
    if (nx < 1 || ny < 1 || nz < 1) {
        msg = "every dimension must be >= 1";
        return GMG_ERR_ARG;
    }
    if ((int64_t)nx * ny * nz > ((int64_t)1 << 31) - 1) {
        msg = "grids above 2^31 cells are not supported";
        return GMG_ERR_ARG;
    }
    const int n[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d)
        if (periodic && periodic[d] && n[d] % 2) {
            msg = "a periodic axis must have even length (red-black colouring)";
            return GMG_ERR_ARG;
        }
    return GMG_OK;
}

namespace {

int validate_options(const gmg_options& o, std::string& msg)
{
    if (o.coarsen != GMG_COARSEN_ISO && o.coarsen != GMG_COARSEN_ANISO) msg = "coarsen must be ISO or ANISO";
    else if (o.n_min < 1) msg = "n_min must be >= 1";
    else if (o.nu1 < 0 || o.nu2 < 1 || o.nu_c < 1) msg = "need nu1 >= 0, nu2 >= 1, nu_c >= 1";
    else if (o.precision < GMG_FP32 || o.precision > GMG_IR64_FP32) msg = "unknown precision";
    else if (o.max_cycles < 1) msg = "max_cycles must be >= 1";
    else if (!(o.omega0 > 0.0) || !(o.omega_min > 0.0) || !(o.shrink > 0.0 && o.shrink < 1.0) || !(o.grow >= 1.0))
        msg = "need omega0 > 0, omega_min > 0, 0 < shrink < 1, grow >= 1";
    else if (!(o.ir_inner_rtol > 0.0 && o.ir_inner_rtol < 1.0)) msg = "need 0 < ir_inner_rtol < 1";
    else if (o.coarse_mode != GMG_COARSE_SWEEPS && o.coarse_mode != GMG_COARSE_DENSE)
        msg = "coarse_mode must be SWEEPS or DENSE";
    else if (o.coarse_op != GMG_COARSE_OP_FV && o.coarse_op != GMG_COARSE_OP_GALERKIN)
        msg = "coarse_op must be FV or GALERKIN";
    else return GMG_OK;
    return GMG_ERR_ARG;
}

}  // namespace

namespace gmg {
void set_api_error(const char* msg) { g_create_error = msg ? msg : ""; }
}  // namespace gmg

struct gmg_solver {
    Engine eng;
};
struct gmg_batch_solver {
    Engine eng;
};

extern "C" {

void gmg_default_options(gmg_options* o)
{
    if (!o) return;
    o->coarsen = GMG_COARSEN_ANISO;
    o->n_min = 4;
    o->nu1 = 2;
    o->nu2 = 2;
    o->nu_c = 16;
    o->precision = GMG_FP32;
    o->max_cycles = 100;
    o->omega0 = 1.0;
    o->omega_min = 0.25;
    o->shrink = 0.7;
    o->grow = 1.1;
    o->use_graph = 1;
    o->cycles_per_sync = 8;
    o->ir_inner_rtol = 1e-4;
    o->autotune = 1;
    o->coarse_mode = GMG_COARSE_SWEEPS;
    o->coarse_op = GMG_COARSE_OP_FV;
}

int gmg_create(gmg_handle* h, int nx, int ny, int nz, const int* periodic, const gmg_options* opt,
               void* stream)
{
    if (!h) {
        g_create_error = "h is NULL";
        return GMG_ERR_ARG;
    }
    *h = nullptr;
    gmg_options o;
    gmg_default_options(&o);
    if (opt) o = *opt;
    int rc = validate_geometry(nx, ny, nz, periodic, g_create_error);
    if (rc == GMG_OK) rc = validate_options(o, g_create_error);
    if (rc != GMG_OK) return rc;
    gmg_solver* s = new gmg_solver;
    const int dims[3] = {nx, ny, nz};
    int per[3] = {0, 0, 0};
    if (periodic)
        for (int d = 0; d < 3; ++d) per[d] = periodic[d] != 0;
    rc = s->eng.plan(1, dims, per, o, static_cast<cudaStream_t>(stream));
    if (rc != GMG_OK) {
        g_create_error = s->eng.err;
        delete s;
        return rc;
    }
    *h = s;
    return GMG_OK;
}

int gmg_set_coeffs(gmg_handle h, const float* bx, const float* by, const float* bz)
{
    if (!h) return GMG_ERR_ARG;
    if (!bx || !by || !bz) return h->eng.fail(GMG_ERR_ARG, "null coefficient pointer");
    const float* x[1] = {bx};
    const float* y[1] = {by};
    const float* z[1] = {bz};
    return h->eng.set_coeffs(x, y, z);
}

int gmg_solve(gmg_handle h, const void* sigma, void* p, double tol, gmg_info* info)
{
    if (!h) return GMG_ERR_ARG;
    Engine& E = h->eng;
    if (!sigma || !p) return E.fail(GMG_ERR_ARG, "null sigma or p");
    if (!(tol > 0.0)) return E.fail(GMG_ERR_ARG, "tol must be > 0");
    if (E.ir) {
        const double* sg[1] = {static_cast<const double*>(sigma)};
        double* pp[1] = {static_cast<double*>(p)};
        return E.solve64(sg, pp, tol, info);
    }
    const float* s[1] = {static_cast<const float*>(sigma)};
    float* q[1] = {static_cast<float*>(p)};
    return E.solve32(s, q, tol, info);
}

int gmg_solve_host(gmg_handle h, const void* sigma_host, void* p_host, double tol, gmg_info* info)
{
    if (!h) return GMG_ERR_ARG;
    Engine& E = h->eng;
    if (!sigma_host || !p_host) return E.fail(GMG_ERR_ARG, "null sigma or p");
    const size_t bytes = (size_t)E.P[0].n0 * (E.ir ? sizeof(double) : sizeof(float));
    // staging buffers: allocated on the first call, kept with the handle
    for (int i = 0; i < 2; ++i)
        if (!E.stage[i] && !(E.stage[i] = E.dalloc<char>(bytes))) return E.fail(GMG_ERR_CUDA, "out of device memory");
    void* ds = E.stage[0];
    void* dp = E.stage[1];
    cudaError_t e = cudaMemcpyAsync(ds, sigma_host, bytes, cudaMemcpyHostToDevice, E.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, p_host, bytes, cudaMemcpyHostToDevice, E.stream);
    int rc = GMG_ERR_CUDA;
    if (e == cudaSuccess) {
        rc = gmg_solve(h, ds, dp, tol, info);
        if (rc == GMG_OK || rc == GMG_ERR_NOT_CONVERGED || rc == GMG_ERR_DIVERGED) {
            e = cudaMemcpyAsync(p_host, dp, bytes, cudaMemcpyDeviceToHost, E.stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(E.stream);
            if (e != cudaSuccess) rc = E.cuda_fail(e, "gmg_solve_host (copy back)");
        }
    } else {
        rc = E.cuda_fail(e, "gmg_solve_host");
    }
    return rc;
}

int gmg_pcg_solve(gmg_handle h, const void* sigma, void* p, double tol, int max_iter, gmg_info* info)
{
    if (!h || !sigma || !p || !(tol > 0.0)) return GMG_ERR_ARG;
    return h->eng.pcg_solve(static_cast<const float*>(sigma), static_cast<float*>(p), tol, max_iter, info);
}

int gmg_gmgpcg_solve(gmg_handle h, const void* sigma, void* p, double tol, gmg_info* info)
{
    if (!h || !sigma || !p || !(tol > 0.0)) return GMG_ERR_ARG;
    return h->eng.gmg_pcg_solve(static_cast<const float*>(sigma), static_cast<float*>(p), tol, info);
}

int gmg_history(gmg_handle h, double* rel_res, double* omega, int* accepted, int cap)
{
    if (!h || cap < 0) return -1;
    Engine& E = h->eng;
    const int n = std::min(cap, E.last_cycles);
    const ProblemMem& M = E.P[0];
    cudaError_t e = cudaSuccess;
    if (rel_res) e = cudaMemcpy(rel_res, M.hist_res, sizeof(double) * (n + 1), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && omega && n) e = cudaMemcpy(omega, M.hist_omega, sizeof(double) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && accepted && n) e = cudaMemcpy(accepted, M.hist_acc, sizeof(int) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        E.cuda_fail(e, "gmg_history");
        return -1;
    }
    return n;
}

int gmg_levels(gmg_handle h, int* dims)
{
    if (!h) return -1;
    const ProblemMem& M = h->eng.P[0];
    if (dims)
        for (int l = 0; l < M.L; ++l)
            for (int d = 0; d < 3; ++d) dims[3 * l + d] = M.lev[l].g.n[d];
    return M.L;
}

int gmg_bottom_form(gmg_handle h, int* level, int* ranks)
{
    if (!h || !level || !ranks) return GMG_ERR_ARG;
    *level = h->eng.bottom_level_;
    *ranks = h->eng.bottom_ranks_;
    return GMG_OK;
}

int gmg_destroy(gmg_handle h)
{
    delete h;
    return GMG_OK;
}

const char* gmg_last_error(gmg_handle h)
{
    if (!h) return g_create_error.c_str();
    return h->eng.err.c_str();
}

// ---------------------------------------------------------------- test hooks

int gmg_test_poison_omega(gmg_handle h, int cycle)
{
    if (!h || cycle < 1) return GMG_ERR_ARG;
    h->eng.poison_cycle = cycle;
    return GMG_OK;
}

int gmg_test_ring_wait_tries(int tries)
{
    const cudaError_t e = gmg::set_ring_wait_tries(tries);
    if (e != cudaSuccess) {
        g_create_error = std::string("gmg_test_ring_wait_tries: ") + cudaGetErrorString(e);
        return GMG_ERR_CUDA;
    }
    return GMG_OK;
}

int gmg_test_cluster_ranks(int ranks)
{
    if (ranks != 0 && ranks != 8 && ranks != 16) return GMG_ERR_ARG;
    gmg::set_cluster_cap(ranks == 0 ? gmg::kClusterMaxRanks : ranks);
    return GMG_OK;
}

// ---------------------------------------------------------------- tuning table

int gmg_tune_export(char* buf, size_t cap, size_t* len)
{
    std::string t;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        for (const auto& kv : g_tuned_zchunk) {
            const TuneKey& k = kv.first;
            t += "z " + std::to_string(k.kind) + " " + std::to_string(k.n0) + " " + std::to_string(k.n1) + " " +
                 std::to_string(k.n2) + " " + std::to_string(k.p0) + " " + std::to_string(k.p1) + " " +
                 std::to_string(k.p2) + " " + std::to_string(kv.second) + "\n";
        }
        for (const auto& kv : g_tuned_lb) {
            t += "b";
            for (int v : kv.first) t += " " + std::to_string(v);
            t += " " + std::to_string(kv.second.level) + " " + std::to_string(kv.second.ranks) + "\n";
        }
        for (const auto& kv : g_tuned_batch)
            t += "c " + std::to_string(kv.first.first) + " " + std::to_string(kv.first.second) + " " +
                 std::to_string(kv.second) + "\n";
    }
    if (len) *len = t.size();
    if (!buf) return GMG_OK;
    if (cap < t.size() + 1) return GMG_ERR_ARG;
    std::memcpy(buf, t.c_str(), t.size() + 1);
    return GMG_OK;
}

int gmg_tune_import(const char* text)
{
    if (!text) return GMG_ERR_ARG;
    std::map<TuneKey, int> zs;
    std::map<std::vector<int>, BottomChoice> bs;
    std::map<std::pair<int, int>, int> cs;
    std::istringstream in(text);
    std::string line;
    while (std::getline(in, line)) {
        std::istringstream ls(line);
        std::string tag;
        if (!(ls >> tag)) continue;                     // blank line
        std::vector<long> v;
        long x;
        while (ls >> x) v.push_back(x);
        if (!ls.eof()) return GMG_ERR_ARG;              // a token that is not an integer
        for (long a : v)
            if (a < 0 || a > (1L << 30)) return GMG_ERR_ARG;
        if (tag == "z" && v.size() == 8 && v[7] > 0) {
            zs[TuneKey{(int)v[0], (int)v[1], (int)v[2], (int)v[3], (int)v[4], (int)v[5], (int)v[6]}] = (int)v[7];
        } else if (tag == "b" && (v.size() == 12 || v.size() == 13) && v[11] < kMaxLevels &&
                   (v.size() == 12 || (v[12] >= 1 && v[12] <= kClusterMaxRanks))) {
            // level 0: forget the entry (the next handle of that shape times again)
            bs[std::vector<int>(v.begin(), v.begin() + 11)] = BottomChoice{(int)v[11], v.size() == 13 ? (int)v[12] : 1};
        } else if (tag == "c" && v.size() == 3 && v[0] >= 2) {
            cs[{(int)v[0], (int)v[1]}] = (int)v[2];
        } else {
            return GMG_ERR_ARG;
        }
    }
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (const auto& kv : zs) g_tuned_zchunk[kv.first] = kv.second;
    for (const auto& kv : cs) g_tuned_batch[kv.first] = kv.second;
    for (const auto& kv : bs) {
        if (kv.second.level == 0) g_tuned_lb.erase(kv.first);
        else g_tuned_lb[kv.first] = kv.second;
    }
    return GMG_OK;
}

// ---------------------------------------------------------------- batch

int gmg_batch_create(gmg_batch* b, int nprob, const int* dims, const int* periodic,
                     const gmg_options* opt, void* stream)
{
    if (!b || nprob < 1 || !dims) {
        g_create_error = "need b, nprob >= 1 and dims";
        return GMG_ERR_ARG;
    }
    *b = nullptr;
    gmg_options o;
    gmg_default_options(&o);
    if (opt) o = *opt;
    int rc = validate_options(o, g_create_error);
    if (rc != GMG_OK) return rc;
    for (int p = 0; p < nprob; ++p) {
        rc = validate_geometry(dims[3 * p], dims[3 * p + 1], dims[3 * p + 2], periodic ? periodic + 3 * p : nullptr,
                               g_create_error);
        if (rc != GMG_OK) return rc;
    }
    gmg_batch_solver* s = new gmg_batch_solver;
    rc = s->eng.plan(nprob, dims, periodic, o, static_cast<cudaStream_t>(stream));
    if (rc != GMG_OK) {
        g_create_error = s->eng.err;
        delete s;
        return rc;
    }
    *b = s;
    return GMG_OK;
}

int gmg_batch_set_coeffs(gmg_batch b, const float* const* bx, const float* const* by, const float* const* bz)
{
    if (!b) return GMG_ERR_ARG;
    if (!bx || !by || !bz) return b->eng.fail(GMG_ERR_ARG, "null coefficient array");
    for (size_t p = 0; p < b->eng.P.size(); ++p)
        if (!bx[p] || !by[p] || !bz[p]) return b->eng.fail(GMG_ERR_ARG, "null coefficient pointer (problem %zu)", p);
    return b->eng.set_coeffs(bx, by, bz);
}

int gmg_batch_solve(gmg_batch b, const void* const* sigma, void* const* p, double tol, gmg_info* infos)
{
    if (!b) return GMG_ERR_ARG;
    if (!sigma || !p) return b->eng.fail(GMG_ERR_ARG, "null sigma or p array");
    if (!(tol > 0.0)) return b->eng.fail(GMG_ERR_ARG, "tol must be > 0");
    const size_t n = b->eng.P.size();
    for (size_t q = 0; q < n; ++q)
        if (!sigma[q] || !p[q]) return b->eng.fail(GMG_ERR_ARG, "null sigma or p (problem %zu)", q);
    if (b->eng.ir) {
        std::vector<const double*> s(n);
        std::vector<double*> q(n);
        for (size_t k = 0; k < n; ++k) {
            s[k] = static_cast<const double*>(sigma[k]);
            q[k] = static_cast<double*>(p[k]);
        }
        return b->eng.solve64(s.data(), q.data(), tol, infos);
    }
    std::vector<const float*> s(n);
    std::vector<float*> q(n);
    for (size_t k = 0; k < n; ++k) {
        s[k] = static_cast<const float*>(sigma[k]);
        q[k] = static_cast<float*>(p[k]);
    }
    return b->eng.solve32(s.data(), q.data(), tol, infos);
}

int gmg_batch_destroy(gmg_batch b)
{
    delete b;
    return GMG_OK;
}

const char* gmg_batch_last_error(gmg_batch b)
{
    if (!b) return g_create_error.c_str();
    return b->eng.err.c_str();
}

// ---------------------------------------------------------------- single steps

static Geo make_geo(int nx, int ny, int nz, const int* periodic)
{
    Geo g;
    g.n[0] = nx;
    g.n[1] = ny;
    g.n[2] = nz;
    for (int d = 0; d < 3; ++d) g.per[d] = periodic ? (periodic[d] != 0) : 0;
    return g;
}

static int check_factors(int nx, int ny, int nz, const int* f)
{
    if (!f) return GMG_ERR_ARG;
    const int n[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d) {
        if (f[d] != 1 && f[d] != 2) return GMG_ERR_ARG;
        if (n[d] % f[d]) return GMG_ERR_ARG;
    }
    return GMG_OK;
}

int gmg_op_sweep(int nx, int ny, int nz, const int* periodic, const float* bx, const float* by,
                 const float* bz, const float* b, const float* p_in, float* p_out, double omega,
                 void* stream)
{
    std::string msg;
    if (validate_geometry(nx, ny, nz, periodic, msg) != GMG_OK) return GMG_ERR_ARG;
    if (!bx || !by || !bz || !b || !p_in || !p_out || p_in == p_out) return GMG_ERR_ARG;
    SweepTask<float, float> t{};
    t.g = make_geo(nx, ny, nz, periodic);
    t.bx = bx;
    t.by = by;
    t.bz = bz;
    t.b = b;
    t.buf[0] = const_cast<float*>(p_in);
    t.buf[1] = p_out;
    t.buf[2] = p_out;
    t.rot = nullptr;
    t.in_role = 0;
    t.out_role = 1;
    t.corr = nullptr;
    t.cf[0] = t.cf[1] = t.cf[2] = 1;
    const SweepTiling st = sweep_tiling(t.g);
    t.tiles_x = st.tx;
    t.tiles_y = st.ty;
    t.zchunk = st.zchunk;
    t.nchunks = st.nchunks;
    t.omega = (float)omega;
    t.ctl = nullptr;
    TaskList<SweepTask<float, float>> tl{};
    tl.ntasks = 1;
    tl.total = (int)st.tiles();
    tl.vec = sweep_vec(t);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TmaPlanes* dmap = op_tensor_maps(t.g, p_in, b, bx, by, bz, tl.vec == 4, s);
    t.tma = dmap;
    tl.single = t;
    cudaError_t e = launch_sweep(tl, sweep_grid(tl), s);
    return e == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

int gmg_op_sweep_reference(int nx, int ny, int nz, const int* periodic, const float* bx,
                           const float* by, const float* bz, const float* b, float* p, double omega,
                           void* stream)
{
    std::string msg;
    if (validate_geometry(nx, ny, nz, periodic, msg) != GMG_OK) return GMG_ERR_ARG;
    if (!bx || !by || !bz || !b || !p) return GMG_ERR_ARG;
    return launch_sweep_two_pass(make_geo(nx, ny, nz, periodic), bx, by, bz, b, p, (float)omega,
                                 static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? GMG_OK
               : GMG_ERR_CUDA;
}

static int op_scratch(int ntiles, double** part, double** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GMG_ERR_CUDA;
    for (auto& s : g_op_scratch)
        if (s.device == dev) {
            if (s.cap < ntiles) {
                cudaFree(s.part);
                s.part = nullptr;
                if (cudaMalloc(&s.part, sizeof(double) * ntiles) != cudaSuccess) {
                    s.cap = 0;
                    return GMG_ERR_CUDA;
                }
                s.cap = ntiles;
            }
            *part = s.part;
            *out = s.out;
            return GMG_OK;
        }
    OpScratch s;
    s.device = dev;
    if (cudaMalloc(&s.part, sizeof(double) * ntiles) != cudaSuccess) return GMG_ERR_CUDA;
    if (cudaMalloc(&s.out, sizeof(double)) != cudaSuccess) return GMG_ERR_CUDA;
    s.cap = ntiles;
    g_op_scratch.push_back(s);
    *part = s.part;
    *out = s.out;
    return GMG_OK;
}

static int op_residual(int nx, int ny, int nz, const int* periodic, const int* factors, const float* bx,
                       const float* by, const float* bz, const float* b, const float* p, float* b_coarse,
                       double* rr, void* stream)
{
    std::string msg;
    if (validate_geometry(nx, ny, nz, periodic, msg) != GMG_OK) return GMG_ERR_ARG;
    if (!bx || !by || !bz || !b || !p) return GMG_ERR_ARG;
    if (b_coarse && check_factors(nx, ny, nz, factors) != GMG_OK) return GMG_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ResTask<float> t{};
    t.g = make_geo(nx, ny, nz, periodic);
    t.bx = bx;
    t.by = by;
    t.bz = bz;
    t.b = b;
    t.buf[0] = t.buf[1] = t.buf[2] = const_cast<float*>(p);
    t.rot = nullptr;
    t.role = 0;
    t.bc = b_coarse;
    for (int d = 0; d < 3; ++d) t.cf[d] = b_coarse ? factors[d] : 1;
    const bool march = res_marches(t.g, true) && aligned16(bx) && aligned16(by) && aligned16(bz) && aligned16(b) &&
                       aligned16(p);
    const ResTiling rt = march ? march_tiling(t.g) : res_tiling(t.g);
    t.tiles_x = rt.tx;
    t.tiles_y = rt.ty;
    t.tiles_z = rt.tz;
    t.zchunk = rt.zchunk;
    t.ctl = nullptr;
    std::unique_lock<std::mutex> lock(g_op_mutex, std::defer_lock);
    double* out = nullptr;
    if (rr) {
        lock.lock();
        if (op_scratch((int)rt.tiles(), &t.partials, &out) != GMG_OK) return GMG_ERR_CUDA;
    }
    TaskList<ResTask<float>> tl{};
    tl.ntasks = 1;
    tl.total = (int)rt.tiles();
    tl.march = march ? 1 : 0;
    TmaPlanes* dmap = op_tensor_maps(t.g, p, b, bx, by, bz, march, s);
    t.tma = dmap;
    tl.single = t;
    cudaError_t e = launch_residual(tl, residual_grid(tl), s);
    if (e == cudaSuccess && rr) {
        e = launch_sum_partials(t.partials, (int)rt.tiles(), out, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(rr, out, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    return e == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

int gmg_op_residual64(int nx, int ny, int nz, const int* periodic, const float* bx, const float* by,
                      const float* bz, const double* b, const double* p, double* r_out, float* r32_out,
                      double* rr, int definition, void* stream)
{
    std::string msg;
    if (validate_geometry(nx, ny, nz, periodic, msg) != GMG_OK) return GMG_ERR_ARG;
    if (!bx || !by || !bz || !b || !p || (definition != 0 && definition != 1)) return GMG_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    IrTask t{};
    t.g = make_geo(nx, ny, nz, periodic);
    t.bx = bx;
    t.by = by;
    t.bz = bz;
    t.b64 = b;
    t.p64 = const_cast<double*>(p);
    t.b32 = r32_out;
    t.r64 = r_out;
    const ResTiling rt = res_tiling(t.g);
    t.tiles_x = rt.tx;
    t.tiles_y = rt.ty;
    t.tiles_z = rt.tz;
    const int grid = persistent_grid(rt.tiles());
    std::lock_guard<std::mutex> lock(g_op_mutex);
    double* out = nullptr;
    if (op_scratch(grid, &t.partials, &out) != GMG_OK) return GMG_ERR_CUDA;
    cudaError_t e = launch_ir_residual(t, grid, s, definition == 1);
    if (e == cudaSuccess && rr) {
        e = launch_sum_partials(t.partials, grid, out, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(rr, out, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    return e == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

int gmg_op_residual_restrict(int nx, int ny, int nz, const int* periodic, const int* factors,
                             const float* bx, const float* by, const float* bz, const float* b,
                             const float* p, float* b_coarse, double* rr, void* stream)
{
    if (!b_coarse) return GMG_ERR_ARG;
    return op_residual(nx, ny, nz, periodic, factors, bx, by, bz, b, p, b_coarse, rr, stream);
}

int gmg_op_residual_norm(int nx, int ny, int nz, const int* periodic, const float* bx,
                         const float* by, const float* bz, const float* b, const float* p,
                         double* rr, void* stream)
{
    if (!rr) return GMG_ERR_ARG;
    return op_residual(nx, ny, nz, periodic, nullptr, bx, by, bz, b, p, nullptr, rr, stream);
}

int gmg_op_prolong_add(int nx, int ny, int nz, const int* factors, const float* e, float* p, void* stream)
{
    std::string msg;
    if (validate_geometry(nx, ny, nz, nullptr, msg) != GMG_OK) return GMG_ERR_ARG;
    if (!e || !p || check_factors(nx, ny, nz, factors) != GMG_OK) return GMG_ERR_ARG;
    Geo g = make_geo(nx, ny, nz, nullptr);
    return launch_prolong_add(g, factors, e, p, static_cast<cudaStream_t>(stream)) == cudaSuccess ? GMG_OK
                                                                                                   : GMG_ERR_CUDA;
}

int gmg_op_coarsen_coeffs(int nx, int ny, int nz, const int* periodic, const int* factors,
                          const float* bx, const float* by, const float* bz, float* cbx,
                          float* cby, float* cbz, void* stream)
{
    std::string msg;
    if (validate_geometry(nx, ny, nz, periodic, msg) != GMG_OK) return GMG_ERR_ARG;
    if (!bx || !by || !bz || !cbx || !cby || !cbz || check_factors(nx, ny, nz, factors) != GMG_OK)
        return GMG_ERR_ARG;
    Geo g = make_geo(nx, ny, nz, periodic);
    return launch_coarsen_coeffs(g, factors, bx, by, bz, cbx, cby, cbz, 0, static_cast<cudaStream_t>(stream)) ==
                   cudaSuccess
               ? GMG_OK
               : GMG_ERR_CUDA;
}

}  // extern "C"
