// gmg_bottom.cu -- the bottom of the V-cycle in one CTA.
//
// The coarse levels of a hierarchy are small (a few thousand cells and
// below), where one launch per sweep costs more in launch and pipeline
// latency than in work.  k_bottom runs the whole lower part of the V-cycle
// (paper Sec. 3: smoothing and coarse-grid correction; Sec. 3.1: the
// under-relaxed red-black Gauss-Seidel smoother; Sec. 3.2: the iso- or
// anisotropically coarsened levels) for levels lb .. L-1 of one problem inside
// one CTA, with every level's iterate, right-hand side and face coefficients
// in shared memory:
//   descent  : zero guess, nu1 sweeps, residual summed over the children of
//              each coarse cell (restriction);
//   coarsest : right-hand side projected to zero mean over active cells,
//              nu_c sweeps from zero, or (coarse_mode 1) p = A^+ b with the
//              level's pseudo-inverse (a GEMV from global memory);
//   ascent   : p += e[I / c] (prolongation), nu2 sweeps;
// and writes level lb's result for the finer level's correction.  Colour
// phases are separated by block barriers; within a colour the cells are
// independent, so in-place updates are exact Gauss-Seidel.
#include <cooperative_groups.h>
#include <atomic>
#include <map>
#include <mutex>

#include "gmg_internal.h"
#include "gmg_device.cuh"

namespace cg = cooperative_groups;

namespace gmg {
namespace {

using namespace dev;

struct LevelView {
    Geo g;
    int n;
    float inv_nx, inv_nxy;
    float* p;
    float* b;
    float* x;   // lower faces, walls zeroed
    float* y;
    float* z;
};

// i / d for 0 <= i < 2^23: an FP32 estimate (FP64 runs at 1/64 of the FP32 rate
// on this part) corrected by one step.  The estimate's absolute error is below
// (i + 1/2) / d * 2^-23 < 1, so it is the quotient or off by one, and the
// remainder's sign and size tell which.
__device__ __forceinline__ int quot(int i, int d, float inv_d)
{
    int q = (int)(((float)i + 0.5f) * inv_d);
    const int r = i - q * d;
    if (r < 0) --q;
    else if (r >= d) ++q;
    return q;
}

// cell index -> (x, y, z) (a bottom level has at most kBottomMaxCells cells)
__device__ __forceinline__ void decode(const LevelView& L, int i, int& x, int& y, int& z)
{
    const int nx = L.g.n[0], nxy = L.g.n[0] * L.g.n[1];
    z = quot(i, nxy, L.inv_nxy);
    const int r = i - z * nxy;
    y = quot(r, nx, L.inv_nx);
    x = r - y * nx;
}

// neighbour of (x, y, z) along axis d in direction s, or -1 outside a wall
__device__ __forceinline__ int nbr(const Geo& g, int x, int y, int z, int d, int s)
{
    int c[3] = {x, y, z};
    c[d] += s;
    if (!wrapc(c[d], g.n[d], g.per[d])) return -1;
    return (c[2] * g.n[1] + c[1]) * g.n[0] + c[0];
}

// (A p)_i and the diagonal at cell i = (x, y, z), from shared memory; interior
// cells take their neighbours at fixed offsets, boundary cells wrap or drop them
__device__ __forceinline__ float flux_xyz(const LevelView& L, int i, int x, int y, int z, float& dg)
{
    const int nx = L.g.n[0], nxy = L.g.n[0] * L.g.n[1];
    const float p0 = L.p[i];
    int xl, xu, yl, yu, zl, zu;
    if (x > 0 && x < nx - 1 && y > 0 && y < L.g.n[1] - 1 && z > 0 && z < L.g.n[2] - 1) {
        xl = i - 1; xu = i + 1; yl = i - nx; yu = i + nx; zl = i - nxy; zu = i + nxy;
    } else {
        xl = nbr(L.g, x, y, z, 0, -1); xu = nbr(L.g, x, y, z, 0, +1);
        yl = nbr(L.g, x, y, z, 1, -1); yu = nbr(L.g, x, y, z, 1, +1);
        zl = nbr(L.g, x, y, z, 2, -1); zu = nbr(L.g, x, y, z, 2, +1);
    }
    const float fxu = xu < 0 ? 0.f : L.x[xu], fyu = yu < 0 ? 0.f : L.y[yu], fzu = zu < 0 ? 0.f : L.z[zu];
    dg = diag_sum(L.x[i], fxu, L.y[i], fyu, L.z[i], fzu);
    return face_flux(L.x[i], xl < 0 ? p0 : L.p[xl], fxu, xu < 0 ? p0 : L.p[xu], L.y[i],
                     yl < 0 ? p0 : L.p[yl], fyu, yu < 0 ? p0 : L.p[yu], L.z[i],
                     zl < 0 ? p0 : L.p[zl], fzu, zu < 0 ? p0 : L.p[zu], p0);
}

// diagonal (sum of the six face coefficients) of cell i
__device__ __forceinline__ float diag_at(const LevelView& L, int i)
{
    int x, y, z;
    decode(L, i, x, y, z);
    const int xu = nbr(L.g, x, y, z, 0, +1), yu = nbr(L.g, x, y, z, 1, +1), zu = nbr(L.g, x, y, z, 2, +1);
    return diag_sum(L.x[i], xu < 0 ? 0.f : L.x[xu], L.y[i], yu < 0 ? 0.f : L.y[yu], L.z[i],
                    zu < 0 ? 0.f : L.z[zu]);
}

// Walk cells first, first + stride, ... of a level, keeping (x, y, z) up to date
// by carries instead of divisions.
struct CellWalk {
    int i, x, y, z, dx, dy, dz;
    __device__ CellWalk(const LevelView& L, int first, int stride)
    {
        i = first;
        decode(L, first, x, y, z);
        decode(L, stride, dx, dy, dz);
    }
    __device__ __forceinline__ void next(const Geo& g, int stride)
    {
        i += stride;
        x += dx;
        int cy = 0;
        if (x >= g.n[0]) { x -= g.n[0]; cy = 1; }
        y += dy + cy;
        int cz = 0;
        if (y >= g.n[1]) { y -= g.n[1]; cz = 1; }
        z += dz + cz;
    }
};

// nu red-black sweeps of one level, every thread of the block.  A half-sweep walks
// only the cells of its colour: cell j of row (y, z) in the half-index space is
// x = 2j + ((colour + y + z) & 1) (x = nx is skipped when nx is odd).  Cells of one
// colour are independent, so the order of the walk does not change the result.
__device__ void sweeps(const LevelView& L, int count, float w)
{
    const int nx = L.g.n[0], ny = L.g.n[1], nz = L.g.n[2];
    const int hx = (nx + 1) >> 1;
    const int nh = hx * ny * nz;
    const int step = blockDim.x;
    // start (j, y, z) of this thread and the stride (dj, dy, dz), by carries afterwards
    const int j0 = threadIdx.x % hx, r0 = threadIdx.x / hx;
    const int dj = step % hx, dr = step / hx;
    const int y0 = r0 % ny, z0 = r0 / ny, dy = dr % ny, dz = dr / ny;
    for (int it = 0; it < count; ++it)
        for (int colour = 0; colour < 2; ++colour) {
            int j = j0, y = y0, z = z0;
            for (int t = threadIdx.x; t < nh; t += step) {
                const int x = 2 * j + ((colour + y + z) & 1);
                if (x < nx) {
                    const int i = (z * ny + y) * nx + x;
                    float dg;
                    const float fl = flux_xyz(L, i, x, y, z, dg);
                    L.p[i] = gs_update(L.p[i], fl, dg, L.b[i], w);
                }
                j += dj;
                int cy = 0;
                if (j >= hx) { j -= hx; cy = 1; }
                y += dy + cy;
                int cz = 0;
                if (y >= ny) { y -= ny; cz = 1; }
                z += dz + cz;
            }
            __syncthreads();
        }
}

// The same sweeps on a level of at most blockDim.x cells, one cell per thread: the
// cell's neighbour indices, face coefficients, diagonal and right-hand side stay in
// registers across the sweeps, so a half-sweep is six shared loads and one store.
// Same operands and operation order as sweeps(): bit-identical results.
__device__ void sweeps_small(const LevelView& L, int count, float w)
{
    const int i = threadIdx.x;
    const bool on = i < L.n;
    int nb[6] = {0, 0, 0, 0, 0, 0};
    float cf[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float bi = 0.f, dg = 0.f;
    int colour = -1;
    if (on) {
        int x, y, z;
        decode(L, i, x, y, z);
        colour = (x + y + z) & 1;
        for (int d = 0; d < 3; ++d) {
            const int lo = nbr(L.g, x, y, z, d, -1), up = nbr(L.g, x, y, z, d, +1);
            const float* f = d == 0 ? L.x : (d == 1 ? L.y : L.z);
            nb[2 * d] = lo < 0 ? i : lo;            // a missing neighbour contributes p - p = 0
            nb[2 * d + 1] = up < 0 ? i : up;
            cf[2 * d] = f[i];
            cf[2 * d + 1] = up < 0 ? 0.f : f[up];
        }
        dg = diag_sum(cf[0], cf[1], cf[2], cf[3], cf[4], cf[5]);
        bi = L.b[i];
    }
    for (int it = 0; it < count; ++it)
        for (int c = 0; c < 2; ++c) {
            if (colour == c) {
                const float p0 = L.p[i];
                const float fl = face_flux(cf[0], L.p[nb[0]], cf[1], L.p[nb[1]], cf[2], L.p[nb[2]], cf[3],
                                           L.p[nb[3]], cf[4], L.p[nb[4]], cf[5], L.p[nb[5]], p0);
                L.p[i] = gs_update(p0, fl, dg, bi, w);
            }
            __syncthreads();
        }
}

// block-reduction and dense-solve scratch of the one-CTA levels
struct BottomScratch {
    double red[kBottomThreads / 32];
    double red2[kBottomThreads / 32];
    double mean;
    float gemv[kBottomThreads];   // dense coarse solve: partial sums of the groups
};

__device__ __forceinline__ LevelView level_view(const BottomLevel& B, float* sm)
{
    LevelView L;
    L.g = B.g;
    L.n = L.g.n[0] * L.g.n[1] * L.g.n[2];
    L.inv_nx = B.inv_nx;
    L.inv_nxy = B.inv_nxy;
    float* base = sm + B.off;
    L.p = base;
    L.b = base + L.n;
    L.x = base + 2 * L.n;
    L.y = base + 3 * L.n;
    L.z = base + 4 * L.n;
    return L;
}

// Face coefficients of levels first .. nlev-1 (lower faces, walls zeroed) into
// their blocks, and level first's right-hand side from b when b is given.
template <class TP>
__device__ void load_levels(const BottomTask<TP>& T, float* sm, int first, const float* b)
{
    for (int l = first; l < T.nlev; ++l) {
        const LevelView L = level_view(T.lev[l], sm);
        const BottomLevel& B = T.lev[l];
        const bool rhs = l == first && b;
        if (B.walls_zeroed) {                      // straight copies: independent loads in flight
            for (int i = threadIdx.x; i < L.n; i += blockDim.x) {
                L.x[i] = __ldg(B.bx + i);
                L.y[i] = __ldg(B.by + i);
                L.z[i] = __ldg(B.bz + i);
                if (rhs) L.b[i] = b[i];
            }
            continue;
        }
        for (CellWalk c(L, threadIdx.x, blockDim.x); c.i < L.n; c.next(L.g, blockDim.x)) {
            const int i = c.i, x = c.x, y = c.y, z = c.z;
            L.x[i] = face_lo(B.bx, L.g, 0, x, y, z);
            L.y[i] = face_lo(B.by, L.g, 1, x, y, z);
            L.z[i] = face_lo(B.bz, L.g, 2, x, y, z);
            if (rhs) L.b[i] = b[i];
        }
    }
}

// The lower V-cycle over levels first .. nlev-1 in this CTA, from level first's
// right-hand side in its block to its iterate in its block (block barriers only).
template <class TP>
__device__ void local_vcycle(const BottomTask<TP>& T, float* sm, int first, float w, BottomScratch& S)
{
    const int nlev = T.nlev;
    auto view = [&](int l) { return level_view(T.lev[l], sm); };

    // descent
    for (int l = first; l + 1 < nlev; ++l) {
        const LevelView L = view(l);
        const LevelView C = view(l + 1);
        for (int i = threadIdx.x; i < L.n; i += blockDim.x) L.p[i] = 0.f;
        __syncthreads();
        if (L.n <= (int)blockDim.x) sweeps_small(L, T.nu1, w);
        else sweeps(L, T.nu1, w);
        const int c0 = T.lev[l].cf[0], c1 = T.lev[l].cf[1], c2 = T.lev[l].cf[2];
        for (CellWalk cw(C, threadIdx.x, blockDim.x); cw.i < C.n; cw.next(C.g, blockDim.x)) {
            const int j = cw.i, X = cw.x, Y = cw.y, Z = cw.z;
            float s = 0.f;
            for (int dz = 0; dz < c2; ++dz)
                for (int dy = 0; dy < c1; ++dy)
                    for (int dx = 0; dx < c0; ++dx) {
                        const int x = X * c0 + dx, y = Y * c1 + dy, z = Z * c2 + dz;
                        const int i = (z * L.g.n[1] + y) * L.g.n[0] + x;
                        float dg;
                        s += L.b[i] - flux_xyz(L, i, x, y, z, dg);
                    }
            C.b[j] = s;
        }
        __syncthreads();
    }

    // coarsest: zero-mean projection over active cells, then nu_c sweeps from zero
    {
        const LevelView C = view(nlev - 1);
        double s = 0.0, cnt = 0.0;
        for (int i = threadIdx.x; i < C.n; i += blockDim.x) {
            C.p[i] = 0.f;
            if (diag_at(C, i) > 0.f) {
                s += (double)C.b[i];
                cnt += 1.0;
            }
        }
        // both sums in one block reduction (the per-warp and cross-warp order of
        // block_sum) over the warps that hold cells: FP64 issues at a small fraction
        // of the FP32 rate here, and the other warps' partials are zeros, which
        // leave the sums unchanged
        const int nw = min((C.n + 31) >> 5, (int)(blockDim.x >> 5));
        if ((int)(threadIdx.x >> 5) < nw) {
            s = warp_sum(s);
            cnt = warp_sum(cnt);
            if ((threadIdx.x & 31) == 0) {
                S.red[threadIdx.x >> 5] = s;
                S.red2[threadIdx.x >> 5] = cnt;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double ts = 0.0, tc = 0.0;
            for (int k = 0; k < nw; ++k) {
                ts += S.red[k];
                tc += S.red2[k];
            }
            S.mean = tc > 0.0 ? ts / tc : 0.0;
        }
        __syncthreads();
        const double mean = S.mean;
        for (int i = threadIdx.x; i < C.n; i += blockDim.x)
            C.b[i] = diag_at(C, i) > 0.f ? (float)((double)C.b[i] - mean) : 0.f;
        __syncthreads();
        if (T.pinv) {
            // dense coarse solve p = A^+ b (A^+ symmetric: column j is row j, so the
            // threads of a group read consecutive entries); the n threads of each of
            // the G groups sum every G-th column, then the G partials are added in
            // group order
            const int n = C.n, G = (int)blockDim.x / n;
            const int i = threadIdx.x % n, grp = threadIdx.x / n;
            float acc = 0.f;
            if (grp < G)
                for (int j = grp; j < n; j += G) acc = fmaf(__ldg(T.pinv + (int64_t)j * n + i), C.b[j], acc);
            S.gemv[threadIdx.x] = acc;
            __syncthreads();
            if (threadIdx.x < n) {
                float sum = 0.f;
                for (int q = 0; q < G; ++q) sum += S.gemv[q * n + threadIdx.x];
                C.p[threadIdx.x] = sum;
            }
            __syncthreads();
        } else if (C.n <= (int)blockDim.x) {
            sweeps_small(C, T.nu_c, w);
        } else {
            sweeps(C, T.nu_c, w);
        }
    }

    // ascent
    for (int l = nlev - 2; l >= first; --l) {
        const LevelView L = view(l);
        const LevelView C = view(l + 1);
        const int c0 = T.lev[l].cf[0], c1 = T.lev[l].cf[1], c2 = T.lev[l].cf[2];
        for (CellWalk c(L, threadIdx.x, blockDim.x); c.i < L.n; c.next(L.g, blockDim.x))
            L.p[c.i] += C.p[((c.z >> (c2 - 1)) * C.g.n[1] + (c.y >> (c1 - 1))) * C.g.n[0] + (c.x >> (c0 - 1))];
        __syncthreads();
        if (L.n <= (int)blockDim.x) sweeps_small(L, T.nu2, w);
        else sweeps(L, T.nu2, w);
    }
}

// the task of block `t` into shared memory, word by word
template <class TP>
__device__ __forceinline__ void load_task(BottomTask<TP>& T, const BottomTask<TP>* tasks, int t)
{
    static_assert(sizeof(BottomTask<TP>) % 4 == 0, "task copied in words");
    const uint32_t* src = reinterpret_cast<const uint32_t*>(tasks + t);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&T);
    for (int k = threadIdx.x; k < (int)(sizeof(BottomTask<TP>) / 4); k += blockDim.x) dst[k] = __ldg(src + k);
    __syncthreads();
}

template <class TP>
__global__ void __launch_bounds__(kBottomThreads) k_bottom(const BottomTask<TP>* __restrict__ tasks)
{
    extern __shared__ __align__(16) float sm[];
    __shared__ BottomScratch S;
    // the task (level geometries, offsets, sweep counts) in shared memory: the level
    // views are rebuilt before every phase
    __shared__ __align__(16) BottomTask<TP> T;
    load_task(T, tasks, blockIdx.x);          // task lists and face coefficients are written before the cycle
    pdl_wait();
    if (T.ctl && T.ctl->done) return;
    const float w = T.ctl ? (float)T.ctl->omega : 1.0f;
    load_levels(T, sm, 0, T.b);
    __syncthreads();
    local_vcycle(T, sm, 0, w, S);
    const LevelView L = level_view(T.lev[0], sm);
    for (int i = threadIdx.x; i < L.n; i += blockDim.x) stv(T.out, (int64_t)i, L.p[i]);
}

// ------------------------------------------------------------------ cluster form
//
// The same lower V-cycle in one thread-block cluster of K CTAs.  A level of more
// than kBottomThreads cells is distributed: rank r of the cluster owns its cells
// [r cpr, (r + 1) cpr) in x-fastest order (cpr a whole number of rows), and keeps
// for them in its shared memory the iterate, right-hand side, residual, the six
// face coefficients and the diagonal (kDistArrays arrays of cpr floats).  x-
// neighbours are in the same row, so local; y- and z-neighbours may be owned by
// another rank and are read through distributed shared memory.  Each colour
// phase, residual, restriction and prolongation is followed by a cluster
// barrier (release/acquire at cluster scope).  The levels below, of at most
// kBottomThreads cells, run in rank 0 exactly as in the one-CTA form while the
// other ranks wait at the next cluster barrier.  Each distributed phase
// evaluates the same operands in the same order as the one-CTA form, so both
// forms give the same bits.

enum { kAP = 0, kAB, kAR, kAXL, kAXU, kAYL, kAYU, kAZL, kAZU, kADG };

struct DistLevel {
    Geo g;
    int nx, ny, nxy, n;
    int cpr, lo, cnt, r0;   // cells per rank; own cells [lo, lo + cnt) = own rows from r0
    int hx;                 // cells of one colour per row, rounded up
    float inv_cpr, inv_nx, inv_ny, inv_nxy, inv_hx;
    float* a;               // own block: array k at a + k * cpr
};

__device__ __forceinline__ DistLevel dist_view(const BottomLevel& B, float* sm, int rank)
{
    DistLevel D;
    D.g = B.g;
    D.nx = B.g.n[0];
    D.ny = B.g.n[1];
    D.nxy = D.nx * D.ny;
    D.n = D.nxy * B.g.n[2];
    D.cpr = B.cpr;
    D.lo = min(rank * D.cpr, D.n);
    D.cnt = min(D.cpr, D.n - D.lo);
    D.r0 = D.lo / D.nx;
    D.hx = (D.nx + 1) >> 1;
    D.inv_cpr = B.inv_cpr;
    D.inv_nx = B.inv_nx;
    D.inv_ny = 1.0f / (float)D.ny;
    D.inv_nxy = B.inv_nxy;
    D.inv_hx = 1.0f / (float)D.hx;
    D.a = sm + B.off;
    return D;
}

// address of array k of cell j (index within the level) in the rank that owns it
__device__ __forceinline__ const float* dist_at(const DistLevel& D, const cg::cluster_group& cl, int rank, int k, int j)
{
    const int o = quot(j, D.cpr, D.inv_cpr);
    const float* p = D.a + k * D.cpr + (j - o * D.cpr);
    return o == rank ? p : cl.map_shared_rank(p, (unsigned)o);
}

// (A p) at own cell c = (x, y, z) of a distributed level, same operands and order as flux_xyz
__device__ __forceinline__ float dist_flux(const DistLevel& D, const cg::cluster_group& cl, int rank, int c, int x,
                                           int y, int z, float p0)
{
    const float* P = D.a;
    const int nx = D.nx, i = D.lo + c;
    const float pxl = x > 0 ? P[c - 1] : (D.g.per[0] ? P[c + nx - 1] : p0);
    const float pxu = x < nx - 1 ? P[c + 1] : (D.g.per[0] ? P[c - nx + 1] : p0);
    const int jyl = y > 0 ? i - nx : (D.g.per[1] ? i + (D.ny - 1) * nx : -1);
    const int jyu = y < D.ny - 1 ? i + nx : (D.g.per[1] ? i - (D.ny - 1) * nx : -1);
    const int nz = D.g.n[2];
    const int jzl = z > 0 ? i - D.nxy : (D.g.per[2] ? i + (nz - 1) * D.nxy : -1);
    const int jzu = z < nz - 1 ? i + D.nxy : (D.g.per[2] ? i - (nz - 1) * D.nxy : -1);
    const float pyl = jyl < 0 ? p0 : *dist_at(D, cl, rank, kAP, jyl);
    const float pyu = jyu < 0 ? p0 : *dist_at(D, cl, rank, kAP, jyu);
    const float pzl = jzl < 0 ? p0 : *dist_at(D, cl, rank, kAP, jzl);
    const float pzu = jzu < 0 ? p0 : *dist_at(D, cl, rank, kAP, jzu);
    const float* A = D.a;
    const int s = D.cpr;
    return face_flux(A[kAXL * s + c], pxl, A[kAXU * s + c], pxu, A[kAYL * s + c], pyl, A[kAYU * s + c], pyu,
                     A[kAZL * s + c], pzl, A[kAZU * s + c], pzu, p0);
}

// own cell c -> (x, y, z)
__device__ __forceinline__ void dist_decode(const DistLevel& D, int c, int& x, int& y, int& z)
{
    const int r = quot(c, D.nx, D.inv_nx);
    x = c - r * D.nx;
    const int row = D.r0 + r;
    z = quot(row, D.ny, D.inv_ny);
    y = row - z * D.ny;
}

// Updated value of the colour's cell t (index among the own cells of that colour)
// in c, or c = -1 when t names no cell
__device__ __forceinline__ float dist_red_black(const DistLevel& D, const cg::cluster_group& cl, int rank, int t,
                                                int nt, int colour, float w, int& c)
{
    c = -1;
    if (t >= nt) return 0.f;
    const int r = quot(t, D.hx, D.inv_hx);
    const int j = t - r * D.hx;
    const int row = D.r0 + r;
    const int z = quot(row, D.ny, D.inv_ny);
    const int y = row - z * D.ny;
    const int x = 2 * j + ((colour + y + z) & 1);
    if (x >= D.nx) return 0.f;
    c = r * D.nx + x;
    const float p0 = D.a[c];
    const float fl = dist_flux(D, cl, rank, c, x, y, z, p0);
    return gs_update(p0, fl, D.a[kADG * D.cpr + c], D.a[kAB * D.cpr + c], w);
}

// nu red-black sweeps of a distributed level; a cluster barrier ends each colour.
// Each thread takes two cells per round and stores both after computing both
// (cells of one colour read only cells of the other), so their neighbour loads,
// several of them from other CTAs, are in flight together.
__device__ void dist_sweeps(const DistLevel& D, const cg::cluster_group& cl, int rank, int count, float w)
{
    const int nt = (D.cnt / D.nx) * D.hx;
    const int bd = blockDim.x;
    float* P = D.a;
    for (int it = 0; it < count; ++it)
        for (int colour = 0; colour < 2; ++colour) {
            for (int t = threadIdx.x; t < nt; t += 2 * bd) {
                int c0, c1;
                const float v0 = dist_red_black(D, cl, rank, t, nt, colour, w, c0);
                const float v1 = dist_red_black(D, cl, rank, t + bd, nt, colour, w, c1);
                if (c0 >= 0) P[c0] = v0;
                if (c1 >= 0) P[c1] = v1;
            }
            cl.sync();
        }
}

// coarse right-hand side of cell (X, Y, Z): the children's residuals summed in the
// one-CTA form's order (z, then y, then x innermost)
__device__ __forceinline__ float dist_child_sum(const DistLevel& F, const cg::cluster_group& cl, int rank,
                                                const int cf[3], int X, int Y, int Z)
{
    float s = 0.f;
    for (int dz = 0; dz < cf[2]; ++dz)
        for (int dy = 0; dy < cf[1]; ++dy)
            for (int dx = 0; dx < cf[0]; ++dx) {
                const int i = ((Z * cf[2] + dz) * F.ny + Y * cf[1] + dy) * F.nx + X * cf[0] + dx;
                s += *dist_at(F, cl, rank, kAR, i);
            }
    return s;
}

template <class TP>
__global__ void __launch_bounds__(kBottomThreads) k_bottom_cluster(const BottomTask<TP>* __restrict__ tasks)
{
    extern __shared__ __align__(16) float sm[];
    __shared__ BottomScratch S;
    __shared__ __align__(16) BottomTask<TP> T;
    const cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    load_task(T, tasks, (int)(blockIdx.x / cl.num_blocks()));
    const int nd = T.nd;

    // own cells of the distributed levels: faces (upper ones from the neighbour's
    // lower face, 0 on walls), diagonal, zero iterate; level 0's right-hand side
    for (int k = 0; k < nd; ++k) {
        const DistLevel D = dist_view(T.lev[k], sm, rank);
        const BottomLevel& B = T.lev[k];
        struct Faces { float xl, xu, yl, yu, zl, zu; };
        auto load = [&](int c) {
            Faces f;
            int x, y, z;
            dist_decode(D, c, x, y, z);
            const int i = D.lo + c;
            f.xl = __ldg(B.bx + i);
            f.yl = __ldg(B.by + i);
            f.zl = __ldg(B.bz + i);
            f.xu = x < D.nx - 1 ? __ldg(B.bx + i + 1) : (D.g.per[0] ? __ldg(B.bx + i - (D.nx - 1)) : 0.f);
            f.yu = y < D.ny - 1 ? __ldg(B.by + i + D.nx) : (D.g.per[1] ? __ldg(B.by + i - (D.ny - 1) * D.nx) : 0.f);
            f.zu = z < D.g.n[2] - 1 ? __ldg(B.bz + i + D.nxy)
                                    : (D.g.per[2] ? __ldg(B.bz + i - (D.g.n[2] - 1) * D.nxy) : 0.f);
            return f;
        };
        auto store = [&](int c, const Faces& f) {
            float* A = D.a;
            const int s = D.cpr;
            A[kAP * s + c] = 0.f;
            A[kAB * s + c] = 0.f;
            A[kAR * s + c] = 0.f;
            A[kAXL * s + c] = f.xl;
            A[kAXU * s + c] = f.xu;
            A[kAYL * s + c] = f.yl;
            A[kAYU * s + c] = f.yu;
            A[kAZL * s + c] = f.zl;
            A[kAZU * s + c] = f.zu;
            A[kADG * s + c] = diag_sum(f.xl, f.xu, f.yl, f.yu, f.zl, f.zu);
        };
        for (int c = threadIdx.x; c < D.cnt; c += 2 * blockDim.x) {   // two cells' loads in flight
            const int c1 = c + blockDim.x;
            const Faces f0 = load(c);
            Faces f1{};
            if (c1 < D.cnt) f1 = load(c1);
            store(c, f0);
            if (c1 < D.cnt) store(c1, f1);
        }
    }
    if (rank == 0) load_levels(T, sm, nd, nullptr);
    // the task lists and face coefficients are written before the cycle; the
    // control state and level 0's right-hand side come from the kernels before
    pdl_wait();
    if (T.ctl && T.ctl->done) return;              // the same flag in every rank of the cluster
    const float w = T.ctl ? (float)T.ctl->omega : 1.0f;
    {
        const DistLevel D = dist_view(T.lev[0], sm, rank);
        for (int c = threadIdx.x; c < D.cnt; c += blockDim.x) D.a[kAB * D.cpr + c] = T.b[D.lo + c];
    }
    cl.sync();

    // descent over the distributed levels: nu1 sweeps from zero, residual, restriction
    for (int k = 0; k < nd; ++k) {
        const DistLevel F = dist_view(T.lev[k], sm, rank);
        dist_sweeps(F, cl, rank, T.nu1, w);
        for (int c = threadIdx.x; c < F.cnt; c += 2 * blockDim.x) {   // two cells per round, as in the sweeps
            const int c1 = c + blockDim.x;
            int x, y, z;
            dist_decode(F, c, x, y, z);
            const float r0 = F.a[kAB * F.cpr + c] - dist_flux(F, cl, rank, c, x, y, z, F.a[kAP * F.cpr + c]);
            float r1 = 0.f;
            if (c1 < F.cnt) {
                dist_decode(F, c1, x, y, z);
                r1 = F.a[kAB * F.cpr + c1] - dist_flux(F, cl, rank, c1, x, y, z, F.a[kAP * F.cpr + c1]);
            }
            F.a[kAR * F.cpr + c] = r0;
            if (c1 < F.cnt) F.a[kAR * F.cpr + c1] = r1;
        }
        cl.sync();
        if (k + 1 < nd) {
            const DistLevel C = dist_view(T.lev[k + 1], sm, rank);
            for (int c = threadIdx.x; c < C.cnt; c += blockDim.x) {
                int X, Y, Z;
                dist_decode(C, c, X, Y, Z);
                C.a[kAB * C.cpr + c] = dist_child_sum(F, cl, rank, T.lev[k].cf, X, Y, Z);
                C.a[kAP * C.cpr + c] = 0.f;
            }
        } else if (rank == 0) {
            const LevelView C = level_view(T.lev[nd], sm);
            for (CellWalk cw(C, threadIdx.x, blockDim.x); cw.i < C.n; cw.next(C.g, blockDim.x))
                C.b[cw.i] = dist_child_sum(F, cl, rank, T.lev[k].cf, cw.x, cw.y, cw.z);
        }
        cl.sync();
    }

    // the levels below in rank 0
    if (rank == 0) local_vcycle(T, sm, nd, w, S);
    cl.sync();

    // ascent over the distributed levels: prolongation, nu2 sweeps
    for (int k = nd - 1; k >= 0; --k) {
        const DistLevel F = dist_view(T.lev[k], sm, rank);
        const int c0 = T.lev[k].cf[0], c1 = T.lev[k].cf[1], c2 = T.lev[k].cf[2];
        const Geo& Cg = T.lev[k + 1].g;
        const bool dist_coarse = k + 1 < nd;
        const DistLevel C = dist_view(T.lev[dist_coarse ? k + 1 : k], sm, rank);   // used when distributed
        auto parent = [&](int c) {
            int x, y, z;
            dist_decode(F, c, x, y, z);
            const int J = ((z >> (c2 - 1)) * Cg.n[1] + (y >> (c1 - 1))) * Cg.n[0] + (x >> (c0 - 1));
            if (dist_coarse) return *dist_at(C, cl, rank, kAP, J);
            const float* p = sm + T.lev[nd].off + J;   // rank 0's iterate of the first local level
            return rank == 0 ? *p : *cl.map_shared_rank(p, 0u);
        };
        for (int c = threadIdx.x; c < F.cnt; c += 2 * blockDim.x) {   // two cells' loads in flight
            const int c1 = c + blockDim.x;
            const float e0 = parent(c);
            const float e1 = c1 < F.cnt ? parent(c1) : 0.f;
            F.a[kAP * F.cpr + c] += e0;
            if (c1 < F.cnt) F.a[kAP * F.cpr + c1] += e1;
        }
        cl.sync();
        dist_sweeps(F, cl, rank, T.nu2, w);
    }

    // level 0's result; no rank reads another's shared memory after the last barrier
    const DistLevel F = dist_view(T.lev[0], sm, rank);
    for (int c = threadIdx.x; c < F.cnt; c += blockDim.x) stv(T.out, (int64_t)(F.lo + c), F.a[kAP * F.cpr + c]);
}

}  // namespace

template <class TP>
cudaError_t launch_bottom(const BottomTask<TP>* tasks, int ntasks, size_t smem, cudaStream_t s)
{
    if (ntasks <= 0) return cudaSuccess;
    static size_t opted = 0;   // dynamic shared memory opted in so far
    if (smem > opted) {
        cudaError_t e = cudaFuncSetAttribute(k_bottom<TP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        opted = smem;
    }
    return launch_pdl(k_bottom<TP>, ntasks, kBottomThreads, smem, s, 1, tasks);
}
template cudaError_t launch_bottom<float>(const BottomTask<float>*, int, size_t, cudaStream_t);
template cudaError_t launch_bottom<bf16>(const BottomTask<bf16>*, int, size_t, cudaStream_t);

template <class TP>
cudaError_t launch_bottom_cluster(const BottomTask<TP>* tasks, int ntasks, int ranks, size_t smem, cudaStream_t s)
{
    if (ntasks <= 0) return cudaSuccess;
    if (ranks < 2 || ranks > kClusterMaxRanks || smem > sizeof(float) * (size_t)kClusterMaxFloats)
        return cudaErrorInvalidValue;
    return launch_pdl(k_bottom_cluster<TP>, dim3((unsigned)(ntasks * ranks)), dim3(kBottomThreads), smem, s, ranks,
                      tasks);
}
template cudaError_t launch_bottom_cluster<float>(const BottomTask<float>*, int, int, size_t, cudaStream_t);
template cudaError_t launch_bottom_cluster<bf16>(const BottomTask<bf16>*, int, int, size_t, cudaStream_t);

// Per device, once: opt both instantiations in to 16-CTA clusters and the full
// shared-memory budget, then ask the occupancy calculator whether one cluster of
// 16 (else 8) such CTAs can be resident.
static std::atomic<int> g_cluster_cap{kClusterMaxRanks};   // test hook: largest cluster size used

void set_cluster_cap(int ranks) { g_cluster_cap.store(ranks); }

static int device_cluster_ranks();

int bottom_cluster_ranks()
{
    const int dev = device_cluster_ranks();
    const int cap = g_cluster_cap.load();
    if (dev >= 16 && cap >= 16) return 16;
    return dev >= 8 && cap >= 8 ? 8 : 0;   // a device that co-schedules 16 CTAs co-schedules 8
}

static int device_cluster_ranks()
{
    static std::mutex m;
    static std::map<int, int> known;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(m);
    auto it = known.find(dev);
    if (it != known.end()) return it->second;
    const int smem = (int)(sizeof(float) * (size_t)kClusterMaxFloats);
    int ranks = 0;
    bool ok = cudaFuncSetAttribute(k_bottom_cluster<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                  cudaSuccess &&
              cudaFuncSetAttribute(k_bottom_cluster<bf16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                  cudaSuccess &&
              cudaFuncSetAttribute(k_bottom_cluster<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
                  cudaSuccess &&
              cudaFuncSetAttribute(k_bottom_cluster<bf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
                  cudaSuccess;
    for (int k : {16, 8}) {
        if (!ok) break;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)k);
        cfg.blockDim = dim3(kBottomThreads);
        cfg.dynamicSmemBytes = (size_t)smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)k;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_bottom_cluster<float>, &cfg) == cudaSuccess && n >= 1) {
            ranks = k;
            break;
        }
    }
    cudaGetLastError();   // a refused query leaves no sticky error
    known[dev] = ranks;
    return ranks;
}

}  // namespace gmg
