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
#include "gmg_internal.h"
#include "gmg_device.cuh"

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

__device__ __forceinline__ float flux_at(const LevelView& L, int i, float& dg)
{
    int x, y, z;
    decode(L, i, x, y, z);
    return flux_xyz(L, i, x, y, z, dg);
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

template <class TP>
__global__ void __launch_bounds__(kBottomThreads) k_bottom(const BottomTask<TP>* __restrict__ tasks)
{
    extern __shared__ __align__(16) float sm[];
    __shared__ double red[kBottomThreads / 32];
    __shared__ double red2[kBottomThreads / 32];
    __shared__ double s_mean;
    __shared__ float s_gemv[kBottomThreads];   // dense coarse solve: partial sums of the groups
    // the task (level geometries, offsets, sweep counts) in shared memory: the level
    // views are rebuilt before every phase
    __shared__ __align__(16) BottomTask<TP> T;
    static_assert(sizeof(BottomTask<TP>) % 4 == 0, "task copied in words");
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(tasks + blockIdx.x);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&T);
        for (int k = threadIdx.x; k < (int)(sizeof(BottomTask<TP>) / 4); k += blockDim.x) dst[k] = __ldg(src + k);
        __syncthreads();
    }
    if (T.ctl && T.ctl->done) return;
    const int nlev = T.nlev;
    const float w = T.ctl ? (float)T.ctl->omega : 1.0f;

    auto view = [&](int l) {
        LevelView L;
        L.g = T.lev[l].g;
        L.n = L.g.n[0] * L.g.n[1] * L.g.n[2];
        L.inv_nx = T.lev[l].inv_nx;
        L.inv_nxy = T.lev[l].inv_nxy;
        float* base = sm + T.lev[l].off;
        L.p = base;
        L.b = base + L.n;
        L.x = base + 2 * L.n;
        L.y = base + 3 * L.n;
        L.z = base + 4 * L.n;
        return L;
    };

    // coefficients of every level (lower faces, walls zeroed) and the top right-hand side
    for (int l = 0; l < nlev; ++l) {
        const LevelView L = view(l);
        const BottomLevel& B = T.lev[l];
        if (B.walls_zeroed) {                      // straight copies: independent loads in flight
            for (int i = threadIdx.x; i < L.n; i += blockDim.x) {
                L.x[i] = __ldg(B.bx + i);
                L.y[i] = __ldg(B.by + i);
                L.z[i] = __ldg(B.bz + i);
                if (l == 0) L.b[i] = T.b[i];
            }
            continue;
        }
        for (CellWalk c(L, threadIdx.x, blockDim.x); c.i < L.n; c.next(L.g, blockDim.x)) {
            const int i = c.i, x = c.x, y = c.y, z = c.z;
            L.x[i] = face_lo(B.bx, L.g, 0, x, y, z);
            L.y[i] = face_lo(B.by, L.g, 1, x, y, z);
            L.z[i] = face_lo(B.bz, L.g, 2, x, y, z);
            if (l == 0) L.b[i] = T.b[i];
        }
    }
    __syncthreads();

    // descent
    for (int l = 0; l + 1 < nlev; ++l) {
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
        // both sums in one block reduction (the same per-warp and cross-warp order as block_sum)
        s = warp_sum(s);
        cnt = warp_sum(cnt);
        if ((threadIdx.x & 31) == 0) {
            red[threadIdx.x >> 5] = s;
            red2[threadIdx.x >> 5] = cnt;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double ts = 0.0, tc = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
                ts += red[k];
                tc += red2[k];
            }
            s_mean = tc > 0.0 ? ts / tc : 0.0;
        }
        __syncthreads();
        const double mean = s_mean;
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
            s_gemv[threadIdx.x] = acc;
            __syncthreads();
            if (threadIdx.x < n) {
                float sum = 0.f;
                for (int q = 0; q < G; ++q) sum += s_gemv[q * n + threadIdx.x];
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
    for (int l = nlev - 2; l >= 0; --l) {
        const LevelView L = view(l);
        const LevelView C = view(l + 1);
        const int c0 = T.lev[l].cf[0], c1 = T.lev[l].cf[1], c2 = T.lev[l].cf[2];
        for (CellWalk c(L, threadIdx.x, blockDim.x); c.i < L.n; c.next(L.g, blockDim.x))
            L.p[c.i] += C.p[((c.z >> (c2 - 1)) * C.g.n[1] + (c.y >> (c1 - 1))) * C.g.n[0] + (c.x >> (c0 - 1))];
        __syncthreads();
        if (L.n <= (int)blockDim.x) sweeps_small(L, T.nu2, w);
        else sweeps(L, T.nu2, w);
    }

    const LevelView L = view(0);
    for (int i = threadIdx.x; i < L.n; i += blockDim.x) stv(T.out, (int64_t)i, L.p[i]);
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
    k_bottom<TP><<<ntasks, kBottomThreads, smem, s>>>(tasks);
    return cudaGetLastError();
}
template cudaError_t launch_bottom<float>(const BottomTask<float>*, int, size_t, cudaStream_t);
template cudaError_t launch_bottom<bf16>(const BottomTask<bf16>*, int, size_t, cudaStream_t);

}  // namespace gmg
