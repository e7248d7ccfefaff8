// gmg_kernels.cu -- sm_103a kernels of the geometric-multigrid Poisson solver.
//
// The operator (the variable-coefficient Poisson equation the paper's Sec. 3.1
// targets) in grid units: (A p)_I = sum_f beta_f (p_nb(f) - p_I).  Kernels:
//
//   k_sweep       one full red-black Gauss-Seidel sweep, under-relaxed by
//                 omega (Sec. 3.1), in ONE launch: each CTA owns a TX x TY
//                 column of a z-chunk, stages halo-2 planes of the input in
//                 shared memory while marching in z, recomputes the red cells
//                 of a one-cell ring around its tile, and writes red and black
//                 cells to a separate output buffer (ping-pong), so no CTA
//                 ever reads a value another CTA writes in the same launch and
//                 no grid barrier is needed.  The coarse correction of the
//                 V-cycle (Sec. 3: piecewise-constant prolongation) and the
//                 zero initial guess of coarse levels are folded into its loads.
//   k_residual    r = b - A p, summed over the children of each coarse cell
//                 (restriction, Sec. 3) and/or squared and summed in FP64.
//   k_coarse      the coarsest level in one CTA: zero-mean projection of b
//                 over active cells, then nu_c sweeps in shared memory.
//   k_coarsen     coarse face coefficients (finite-volume rediscretisation on
//                 the iso- or anisotropically coarsened grid, Sec. 3.2).
//   k_control_*   the adaptive relaxation rule (Sec. 3.1) and convergence
//                 test, one block per problem.
//   k_ir_*        FP64 residual and update of the outer refinement loop.
//   k_project_*, k_gauge_*  right-hand-side projection, exit gauge.
//
// Reductions are deterministic: per-tile partials in FP64, summed in a fixed
// order by one block per problem.  Residual norms of the FP32 levels sum r^2 in
// FP32 over a few cells per thread (or a warp) before the FP64 partial, because
// FP64 arithmetic runs at 1/64 of the FP32 rate on this part.
#include "gmg_internal.h"
#include "gmg_device.cuh"

#include <cmath>
#include <type_traits>

namespace gmg {
namespace {

using namespace dev;

// ---------------------------------------------------------------- K1: fused sweep

template <class TP, class TC>
__global__ void __launch_bounds__(kThreads) k_sweep(const __grid_constant__ TaskList<SweepTask<TP, TC>> tl)
{
    constexpr int TX = kSweepTX, TY = kSweepTY, SW = TX + 4, SH = TY + 4, PL = SW * SH;
    constexpr int EW = TX + 2, EH = TY + 2;
    // ring buffers of z-planes over the tile plus a halo of 2 (the E2 region)
    __shared__ float sP[2][PL];    // input p (+ correction), planes kr, kr+1
    __shared__ float sM[3][PL];    // merged plane: red updated, black = input; kr-2..kr
    __shared__ float sB[2][PL];    // right-hand side, planes kr-1, kr
    __shared__ float sBX[2][PL];   // lower x-face coefficients, planes kr-1, kr
    __shared__ float sBY[2][PL];   // lower y-face coefficients, planes kr-1, kr
    __shared__ float sBZ[3][PL];   // lower z-face coefficients, planes kr-1..kr+1
    const int tid = threadIdx.x;
    pdl_wait();

    for (int tile = blockIdx.x; tile < tl.total; tile += gridDim.x) {
        int local;
        const SweepTask<TP, TC>* tp = task_of(tl, tile, local);
        const Ctl* ctl = tp->ctl;
        if (ctl && ctl->done) continue;                       // uniform in the block
        const Geo g = tp->g;
        const int cx = local % tp->tiles_x;
        const int rest = local / tp->tiles_x;
        const int cy = rest % tp->tiles_y;
        const int cz = rest / tp->tiles_y;
        const int x0 = cx * TX, y0 = cy * TY;
        const int z0 = cz * tp->zchunk;
        const int z1 = min(g.n[2], z0 + tp->zchunk);
        const int rot = tp->rot ? *tp->rot : 0;
        const TP* pin = tp->in_role < 0 ? nullptr : tp->buf[(tp->in_role + rot) % 3];
        TP* pout = tp->buf[(tp->out_role + rot) % 3];
        const TC* corr = tp->corr;
        const int cf0 = tp->cf[0], cf1 = tp->cf[1], cf2 = tp->cf[2];
        Geo gc = g;
        gc.n[0] = g.n[0] / cf0; gc.n[1] = g.n[1] / cf1; gc.n[2] = g.n[2] / cf2;
        const float w = ctl ? (float)ctl->omega : tp->omega;
        const float* bxa = tp->bx;
        const float* bya = tp->by;
        const float* bza = tp->bz;
        const float* ba = tp->b;

        auto load_p = [&](float* dst, int z) {
            int zw = z;
            const bool zok = wrapc(zw, g.n[2], g.per[2]);
            for (int i = tid; i < PL; i += kThreads) {
                const int sy = i / SW, sx = i - sy * SW;
                int x = x0 - 2 + sx, y = y0 - 2 + sy;
                float v = 0.f;
                if (zok && wrapc(x, g.n[0], g.per[0]) && wrapc(y, g.n[1], g.per[1])) {
                    if (pin) v = ldv(pin, lin(g, x, y, zw));
                    if (corr) v += ldv(corr, lin(gc, x / cf0, y / cf1, zw / cf2));
                }
                dst[i] = v;
            }
        };
        auto load_b = [&](float* dst, int z) {
            int zw = z;
            const bool zok = wrapc(zw, g.n[2], g.per[2]);
            for (int i = tid; i < PL; i += kThreads) {
                const int sy = i / SW, sx = i - sy * SW;
                int x = x0 - 2 + sx, y = y0 - 2 + sy;
                float v = 0.f;
                if (zok && wrapc(x, g.n[0], g.per[0]) && wrapc(y, g.n[1], g.per[1]))
                    v = __ldg(ba + lin(g, x, y, zw));
                dst[i] = v;
            }
        };
        auto load_face = [&](float* dst, const float* a, int d, int z) {
            for (int i = tid; i < PL; i += kThreads) {
                const int sy = i / SW, sx = i - sy * SW;
                dst[i] = face_lo(a, g, d, x0 - 2 + sx, y0 - 2 + sy, z);
            }
        };

        const int nsteps = (z1 - z0) + 2;   // red planes z0-1 .. z1
        for (int u = 0; u < nsteps; ++u) {
            const int kr = z0 - 1 + u;
            __syncthreads();                 // ring slots about to be overwritten are free
            if (u == 0) {
                load_p(sP[0], kr);
                load_p(sM[2], kr - 1);       // black cells of plane kr-1 = input values
                load_face(sBZ[0], bza, 2, kr);
            }
            load_p(sP[(u + 1) & 1], kr + 1);
            load_b(sB[u & 1], kr);
            load_face(sBX[u & 1], bxa, 0, kr);
            load_face(sBY[u & 1], bya, 1, kr);
            load_face(sBZ[(u + 1) % 3], bza, 2, kr + 1);
            __syncthreads();

            // red cells of plane kr on the tile and its one-cell ring
            {
                int zk = kr;
                const bool zok = wrapc(zk, g.n[2], g.per[2]);
                const float* P0 = sP[u & 1];
                const float* P1 = sP[(u + 1) & 1];
                const float* Mlo = sM[(u + 2) % 3];
                float* M0 = sM[u % 3];
                const float* B0 = sB[u & 1];
                const float* X0 = sBX[u & 1];
                const float* Y0 = sBY[u & 1];
                const float* Z0 = sBZ[u % 3];
                const float* Z1 = sBZ[(u + 1) % 3];
                for (int i = tid; i < EW * EH; i += kThreads) {
                    const int ey = i / EW, ex = i - ey * EW;
                    const int s = (ey + 1) * SW + (ex + 1);
                    int x = x0 - 1 + ex, y = y0 - 1 + ey;
                    float v = 0.f;
                    if (zok && wrapc(x, g.n[0], g.per[0]) && wrapc(y, g.n[1], g.per[1])) {
                        v = P0[s];
                        if (((x + y + zk) & 1) == 0) {
                            const float fl = face_flux(X0[s], P0[s - 1], X0[s + 1], P0[s + 1], Y0[s],
                                                       P0[s - SW], Y0[s + SW], P0[s + SW], Z0[s], Mlo[s],
                                                       Z1[s], P1[s], v);
                            const float dg = diag_sum(X0[s], X0[s + 1], Y0[s], Y0[s + SW], Z0[s], Z1[s]);
                            v = gs_update(v, fl, dg, B0[s], w);
                        }
                    }
                    M0[s] = v;
                }
            }
            __syncthreads();

            // black cells of plane kr-1 on the tile, from the new red values
            if (u >= 2) {
                const int k = kr - 1;
                const float* Mk = sM[(u + 2) % 3];
                const float* Mlo = sM[(u + 1) % 3];
                const float* Mhi = sM[u % 3];
                const float* Bk = sB[(u + 1) & 1];
                const float* Xk = sBX[(u + 1) & 1];
                const float* Yk = sBY[(u + 1) & 1];
                const float* Zk = sBZ[(u + 2) % 3];
                const float* Zk1 = sBZ[u % 3];
                for (int i = tid; i < TX * TY; i += kThreads) {
                    const int ty = i / TX, tx = i - ty * TX;
                    const int x = x0 + tx, y = y0 + ty;
                    if (x >= g.n[0] || y >= g.n[1]) continue;
                    const int s = (ty + 2) * SW + (tx + 2);
                    float v = Mk[s];
                    if (((x + y + k) & 1) == 1) {
                        const float fl = face_flux(Xk[s], Mk[s - 1], Xk[s + 1], Mk[s + 1], Yk[s], Mk[s - SW],
                                                   Yk[s + SW], Mk[s + SW], Zk[s], Mlo[s], Zk1[s], Mhi[s], v);
                        const float dg = diag_sum(Xk[s], Xk[s + 1], Yk[s], Yk[s + SW], Zk[s], Zk1[s]);
                        v = gs_update(v, fl, dg, Bk[s], w);
                    }
                    stv(pout, lin(g, x, y, k), v);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- K1: pipelined sweep, per-thread copies
//
// The same sweep as k_sweep (same arithmetic, bit-identical results) with the
// z-planes staged by asynchronous global->shared copies of every thread.  It
// serves FP32 levels whose rows are not 16-byte chunks (VEC = 1: single-float
// copies); levels with rows of a multiple of 4 cells run k_sweep_ws below.
// Ring buffers of R planes over the tile plus halo (x: 4 columns each side so
// rows split into 16-byte chunks; y: 2 rows each side) for p, b, the x/y/z
// faces and the merged plane M (red new, black old).  Group G(v) holds what
// step v + LA reads first; step u waits for G(u - LA), then issues G(u); the
// coarse correction of a p plane is added one step before the plane is read.

__device__ __forceinline__ void cp_async16(float* sdst, const float* gsrc, bool ok)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc), "r"(ok ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc, bool ok)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gsrc), "r"(ok ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Whole-plane copies by the tensor memory accelerator: one thread issues a box
// copy per plane (tensor map with a (TX + 8) x (TY + 4) box, zeros outside the
// grid) that completes on an mbarrier of the ring step; every wait is bounded.
constexpr uint32_t kPlaneBytes = sizeof(float) * (kSweepTX + 8) * (kSweepTY + 4);
constexpr int kWaitTries = 1 << 22;

__device__ int g_wait_fault = 0;
// poll limit of the ring-slot waits (set_ring_wait_tries); the waits for copies in
// flight always use kWaitTries
__device__ int g_ring_tries = kWaitTries;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count = 1)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One round of waiting: the thread may stay suspended (issuing nothing) until the
// phase completes or about kSuspendNs have passed.
constexpr uint32_t kSuspendNs = 500;

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, %3;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "n"(kSuspendNs)
        : "memory");
    return done != 0;
}

// false once kWaitTries rounds of try_wait (each may suspend the thread for up to
// kSuspendNs: about two seconds in all) have passed
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    for (int i = 0; i < kWaitTries; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

__device__ __forceinline__ void tma_plane(float* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

template <int VEC, bool CORR, class TC>
__global__ void __launch_bounds__(kThreads, 3) k_sweep_async(const __grid_constant__ TaskList<SweepTask<float, TC>> tl)
{
    constexpr int TX = kSweepTX, TY = kSweepTY;
    constexpr int XO = 4, SW = TX + 8, SH = TY + 4, PL = SW * SH;   // 40 x 12 positions per plane
    constexpr int R = 6;                        // planes per ring, every array (the step sequence is unrolled by 6)
    static_assert(R <= kSweepRing, "the shared memory the launcher reserves holds kSweepRing slots");
    constexpr int LA = CORR ? 2 : 3;            // copy lookahead in z-steps
    constexpr int PA = CORR ? 1 : 0;            // p planes arrive PA further ahead (correction)
    static_assert(3 + LA + PA <= R && 3 + LA <= R, "ring depth vs lookahead");
    constexpr int CPR = SW / 4;                 // 16-byte chunks per row
    constexpr int NCH = PL / 4;                 // chunks per plane (120)
    constexpr int RPR = (TX + 2) / 2;           // red cells per ring row
    constexpr int NRED = RPR * (TY + 2);
    constexpr int BPR = TX / 2;                 // black cells per tile row
    constexpr int NBLK = BPR * TY;
    static_assert(NCH <= kThreads / 2 && NRED <= kThreads && PL <= 2 * kThreads, "thread budget");
    // rings: 0 = p, 1 = b, 2 = lower x faces, 3 = lower y faces, 4 = lower z faces, 5 = merged red plane
    extern __shared__ __align__(128) float smem[];
    const int tid = threadIdx.x;
    const int half = tid / (kThreads / 2);      // copy duty: 0 -> p, b, x faces; 1 -> y, z faces
    const int chunk = tid % (kThreads / 2);
    pdl_wait();

    for (int tile = blockIdx.x; tile < tl.total; tile += gridDim.x) {
        int local;
        const SweepTask<float, TC>* tp = task_of(tl, tile, local);
        const Ctl* ctl = tp->ctl;
        if (ctl && ctl->done) continue;                       // uniform in the block
        const Geo g = tp->g;
        const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
        const int px = g.per[0], py = g.per[1], pz = g.per[2];
        const int cx = local % tp->tiles_x;
        const int rest = local / tp->tiles_x;
        const int cy = rest % tp->tiles_y;
        const int cz = rest / tp->tiles_y;
        const int x0 = cx * TX, y0 = cy * TY;
        const int z0 = cz * tp->zchunk;
        const int z1 = min(nz, z0 + tp->zchunk);
        const int rot = tp->rot ? *tp->rot : 0;
        const float* pin = tp->in_role < 0 ? nullptr : tp->buf[(tp->in_role + rot) % 3];
        float* pout = tp->buf[(tp->out_role + rot) % 3];
        const float w = ctl ? (float)ctl->omega : tp->omega;
        const float* const ba = tp->b;
        // the two arrays this thread's half copies besides p (half 0) or with z faces (half 1)
        const float* const srcA = half == 0 ? pin : tp->by;
        const float* const srcB = half == 0 ? tp->b : tp->bz;
        const float* const srcC = tp->bx;   // half 0 only

        // ---- per-thread geometry, fixed for the tile
        int coff = 0;
        bool cok = false;
        if (VEC == 4 && chunk < NCH) {
            const int sy = chunk / CPR, ch = chunk - sy * CPR;
            int x = x0 - XO + 4 * ch, y = y0 - 2 + sy;
            cok = wrapc(x, nx, px) && wrapc(y, ny, py);
            coff = cok ? y * nx + x : 0;
        }
        const int ey = tid / RPR, jr = tid - ey * RPR;
        int yr = y0 - 1 + ey;
        const bool yr_ok = tid < NRED && wrapc(yr, ny, py);
        const bool yr_wall = yr == 0 && !py;
        const int sred = (ey + 1) * SW + XO - 1 + 2 * jr;
        int xr0 = x0 - 1 + 2 * jr, xr1 = xr0 + 1;
        const bool xr_wall0 = xr0 == 0 && !px, xr_wall1 = xr1 == 0 && !px;
        const bool xr_ok0 = wrapc(xr0, nx, px), xr_ok1 = wrapc(xr1, nx, px);
        const int red_par = (1 + (y0 - 1 + ey)) & 1;          // red member: (red_par + kr) & 1
        const int tyb = tid / BPR, jb = tid - tyb * BPR;
        const int yb = y0 + tyb, xb = x0 + 2 * jb;
        const bool blk_on = tid < NBLK && yb < ny && xb < nx;
        const int sblk = (tyb + 2) * SW + XO + 2 * jb;
        const bool yb_wall = yb == 0 && !py;
        const bool xb_wall = xb == 0 && !px;
        float* const out_col = pout + ((int64_t)yb * nx + xb);
        const int64_t plane = (int64_t)nx * ny;

        auto zinfo = [&](int z, bool zface, int64_t& zoff) -> bool {
            int zw = z;
            bool ok = wrapc(zw, nz, pz);
            if (zface && ok && zw == 0 && !pz) ok = false;   // lower z faces of a wall plane
            zoff = (int64_t)zw * plane;
            return ok;
        };
        // whole plane of array a into dst, every thread helping (prologue; VEC == 1)
        auto copy_plane = [&](float* dst, const float* a, int z, bool zface) {
            int64_t zoff;
            const bool zok = a != nullptr && zinfo(z, zface, zoff);
            if (VEC == 4) {
                for (int c = tid; c < NCH; c += kThreads) {
                    const int sy = c / CPR, ch = c - sy * CPR;
                    int x = x0 - XO + 4 * ch, y = y0 - 2 + sy;
                    const bool ok = zok && wrapc(x, nx, px) && wrapc(y, ny, py);
                    cp_async16(dst + 4 * c, ok ? a + zoff + (int64_t)y * nx + x : ba, ok);
                }
            } else {
                for (int e = tid; e < PL; e += kThreads) {
                    const int sy = e / SW, sx = e - sy * SW;
                    int x = x0 - XO + sx, y = y0 - 2 + sy;
                    const bool ok = zok && wrapc(x, nx, px) && wrapc(y, ny, py);
                    cp_async4(dst + e, ok ? a + zoff + (int64_t)y * nx + x : ba, ok);
                }
            }
        };
        auto ring = [&](int r, int slot) -> float* { return smem + (r * R + slot) * PL; };

        // coarse correction of a p plane: gathered into registers one step ahead
        const TC* corr = tp->corr;
        const int cf0 = tp->cf[0], cf1 = tp->cf[1], cf2 = tp->cf[2];
        const int gcx = nx / cf0, gcy = ny / cf1;
        int crr0 = 0, crr1 = 0;
        bool crok0 = false, crok1 = false;
        if (CORR) {
            for (int r = 0; r < 2; ++r) {
                const int e = tid + r * kThreads;
                if (e < PL) {
                    const int sy = e / SW, sx = e - sy * SW;
                    int x = x0 - XO + sx, y = y0 - 2 + sy;
                    const bool ok = wrapc(x, nx, px) && wrapc(y, ny, py);
                    const int off = ok ? (y / cf1) * gcx + x / cf0 : 0;
                    if (r == 0) { crok0 = ok; crr0 = off; } else { crok1 = ok; crr1 = off; }
                }
            }
        }
        auto corr_load = [&](int z, float& c0, float& c1) {
            c0 = c1 = 0.f;
            if (!CORR) return;
            int zw = z;
            if (!wrapc(zw, nz, pz)) return;
            const int64_t zoff = (int64_t)(zw / cf2) * gcx * gcy;
            if (crok0) c0 = ldv(corr, zoff + crr0);
            if (crok1) c1 = ldv(corr, zoff + crr1);
        };
        auto corr_add = [&](float* dst, float c0, float c1) {
            if (!CORR) return;
            dst[tid] += c0;
            if (tid + kThreads < PL) dst[tid + kThreads] += c1;
        };

        // ---- copy groups.  Group G(v) holds b / x / y faces of plane kr0+v+LA, z faces of
        // kr0+v+1+LA and p of kr0+v+1+LA+PA: everything step v+LA reads for the first time
        // (p one step earlier when PA = 1, so its coarse correction can be added a step
        // before the plane is read).  Step u waits for G(u-LA), then issues G(u) after its
        // first barrier; the prologue issues G0 (p planes kr0-1 .. kr0+PA, z faces of kr0)
        // and G(-LA) .. G(-1).  Plane z lives in slot (z - kr0 + 1) mod R.
        const int kr0 = z0 - 1;
        const int nsteps = (z1 - z0) + 2;   // red planes z0-1 .. z1
        auto issue_group = [&](int v) {
            const int kb = kr0 + v + LA;
            const int sb = (v + LA + 1 + R * 4) % R, sz = (v + LA + 2 + R * 4) % R, sp = (v + LA + PA + 2 + R * 4) % R;
            copy_plane(ring(1, sb), ba, kb, false);
            copy_plane(ring(2, sb), tp->bx, kb, false);
            copy_plane(ring(3, sb), tp->by, kb, false);
            copy_plane(ring(4, sz), tp->bz, kb + 1, true);
            copy_plane(ring(0, sp), pin, kb + 1 + PA, false);
        };
        for (int z = kr0 - 1; z <= kr0 + PA; ++z) copy_plane(ring(0, (z - kr0 + 1 + R) % R), pin, z, false);
        copy_plane(ring(4, 1), tp->bz, kr0, true);
        cp_commit();
        for (int v = -LA; v < 0; ++v) {
            issue_group(v);
            cp_commit();
        }
        float cur0 = 0.f, cur1 = 0.f, nxt0 = 0.f, nxt1 = 0.f;
        if (CORR) {
            float c[3][2];
            for (int j = 0; j < 3; ++j) corr_load(kr0 - 1 + j, c[j][0], c[j][1]);
            corr_load(kr0 + 2, cur0, cur1);
            cp_wait<LA>();
            __syncthreads();
            for (int j = 0; j < 3; ++j) corr_add(ring(0, j), c[j][0], c[j][1]);
        }

        // one z-step; J = (u mod R) is a compile-time constant, so is every slot
        auto step = [&](int u, auto Jc) {
            constexpr int J = decltype(Jc)::value;
            constexpr int S0 = (J + 1) % R;                       // slot of plane kr
            constexpr int Sm1 = (J + R) % R, Sm2 = (J + R - 1) % R;
            constexpr int Sp1 = (J + 2) % R, Sp2 = (J + 3) % R;
            constexpr int SB = (J + 1 + LA) % R, SZ = (J + 2 + LA) % R, SP = (J + 2 + LA + PA) % R;
            const int kr = kr0 + u;
            cp_wait<LA - 1>();
            __syncthreads();                               // S1: G(u-LA) visible, step u-1 done everywhere
            // G(u): written slots hold planes every thread finished with in step u-1
            if (u + LA < nsteps) {
                if (VEC == 4) {
                    if (chunk < NCH) {
                        int64_t zo1, zo2;
                        if (half == 0) {
                            int64_t zo3;
                            const bool ok3 = pin != nullptr && zinfo(kr + 1 + LA + PA, false, zo3) && cok;
                            const bool ok1 = zinfo(kr + LA, false, zo1) && cok;
                            cp_async16(ring(0, SP) + 4 * chunk, ok3 ? srcA + zo3 + coff : ba, ok3);
                            cp_async16(ring(1, SB) + 4 * chunk, ok1 ? srcB + zo1 + coff : ba, ok1);
                            cp_async16(ring(2, SB) + 4 * chunk, ok1 ? srcC + zo1 + coff : ba, ok1);
                        } else {
                            const bool ok1 = zinfo(kr + LA, false, zo1) && cok;
                            const bool ok2 = zinfo(kr + 1 + LA, true, zo2) && cok;
                            cp_async16(ring(3, SB) + 4 * chunk, ok1 ? srcA + zo1 + coff : ba, ok1);
                            cp_async16(ring(4, SZ) + 4 * chunk, ok2 ? srcB + zo2 + coff : ba, ok2);
                        }
                    }
                } else {
                    issue_group(u);
                }
                corr_load(kr + 3, nxt0, nxt1);
            }
            cp_commit();
            if (CORR) {
                corr_add(ring(0, Sp2), cur0, cur1);        // p(kr+2): landed in G(u-LA-1), first read at step u+1
                cur0 = nxt0;
                cur1 = nxt1;
            }

            // red cells of plane kr on the tile and its one-cell ring
            if (tid < NRED) {
                int zk = kr;
                const bool zok = wrapc(zk, nz, pz);
                const int o = (red_par + kr) & 1;
                const int s = sred + o;
                float v = 0.f;
                if (zok && yr_ok && (o ? xr_ok1 : xr_ok0)) {
                    const float* P0 = ring(0, S0);
                    const float* X0 = ring(2, S0);
                    const float* Y0 = ring(3, S0);
                    const float* Z0 = ring(4, S0);
                    const float* Z1 = ring(4, Sp1);
                    v = P0[s];
                    const float xl = (o ? xr_wall1 : xr_wall0) ? 0.f : X0[s];
                    const float yl = yr_wall ? 0.f : Y0[s];
                    const float zl = (kr == 0 && !pz) ? 0.f : Z0[s];
                    const float fl = face_flux(xl, P0[s - 1], X0[s + 1], P0[s + 1], yl, P0[s - SW], Y0[s + SW],
                                               P0[s + SW], zl, ring(0, Sm1)[s], Z1[s], ring(0, Sp1)[s], v);
                    const float dg = diag_sum(xl, X0[s + 1], yl, Y0[s + SW], zl, Z1[s]);
                    v = gs_update(v, fl, dg, ring(1, S0)[s], w);
                }
                ring(5, S0)[s] = v;
            }
            __syncthreads();                               // S2: red cells of kr are merged

            // black cells of plane kr-1 on the tile; the pair's red cell comes from M
            if (u >= 2 && blk_on) {
                const int k = kr - 1;
                const int hb = ((xb + yb + k) & 1) ? 0 : 1;   // black member of the pair
                const int s = sblk + hb;
                const float* Mk = ring(5, Sm1);
                const float* Xk = ring(2, Sm1);
                const float* Yk = ring(3, Sm1);
                const float* Zk = ring(4, Sm1);
                const float* Zk1 = ring(4, S0);
                float v = ring(0, Sm1)[s];
                const float xl = (hb == 0 && xb_wall) ? 0.f : Xk[s];
                const float yl = yb_wall ? 0.f : Yk[s];
                const float zl = (k == 0 && !pz) ? 0.f : Zk[s];
                const float fl = face_flux(xl, Mk[s - 1], Xk[s + 1], Mk[s + 1], yl, Mk[s - SW], Yk[s + SW],
                                           Mk[s + SW], zl, ring(5, Sm2)[s], Zk1[s], ring(5, S0)[s], v);
                const float dg = diag_sum(xl, Xk[s + 1], yl, Yk[s + SW], zl, Zk1[s]);
                v = gs_update(v, fl, dg, ring(1, Sm1)[s], w);
                const float r = Mk[sblk + (1 - hb)];
                const float o0 = hb ? r : v, o1 = hb ? v : r;
                float* dst = out_col + (int64_t)k * plane;
                if (VEC == 4) {
                    *reinterpret_cast<float2*>(dst) = make_float2(o0, o1);
                } else {
                    dst[0] = o0;
                    if (xb + 1 < nx) dst[1] = o1;
                }
            }
        };
        static_assert(R == 6, "the unrolled step sequence below assumes six slots");
        for (int u = 0; u < nsteps; u += R) {
            step(u, std::integral_constant<int, 0>());
            if (u + 1 < nsteps) step(u + 1, std::integral_constant<int, 1>());
            if (u + 2 < nsteps) step(u + 2, std::integral_constant<int, 2>());
            if (u + 3 < nsteps) step(u + 3, std::integral_constant<int, 3>());
            if (u + 4 < nsteps) step(u + 4, std::integral_constant<int, 4>());
            if (u + 5 < nsteps) step(u + 5, std::integral_constant<int, 5>());
        }
        cp_wait<0>();
        __syncthreads();                                   // the next tile reuses the rings
    }
}

// ---------------------------------------------------------------- K2: pipelined residual
//
// r = b - A p on a TX x TY column marching through a z-chunk, restricted to the
// next level and summed in squares (FP64, one partial per tile).  Warp-
// specialised: warps 0-3 (consumers) each own two tile rows, one x-pair of
// cells per thread; warps 4-5 (producers) stream whole planes of p, b and the
// three face arrays into a ring of R = kResRing plane slots (4 blocks per SM).
// Group H(g) (the g-th plane this block streams, over all its tiles) lands in
// slot g mod R and completes on full[g mod R]: by TMA (one box per array, zeros
// outside the grid) when the box needs no periodic wrap in x or y, else by
// 16-byte asynchronous copies of the producers' lanes.  The consumers release a slot on empty[] once no later
// step reads it; the producer waits for that release before refilling the
// slot.  Restriction: x-pairs in the thread, y-pairs with the lane 16 apart,
// z-pairs across two steps, so coarse cells are written without atomics.
constexpr int kProducers = 64;                  // producer warps of the warp-specialised kernels: two
constexpr int kResConsumers = 128;
constexpr int kResBlock = kResConsumers + kProducers;

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// arrive-on triggered by the completion of this thread's earlier cp.async copies
__device__ __forceinline__ void cp_async_mbar_arrive(uint64_t* bar)
{
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// bounded wait on a ring slot that also gives up once another warp of the block
// recorded a fault
__device__ __forceinline__ bool mbar_wait_live(uint64_t* bar, uint32_t parity, const volatile int* dead, int tries)
{
    for (int i = 0; i < tries; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 63 && *dead) return false;
    }
    return false;
}

__device__ __forceinline__ int wrap_plane(int z, int nz, int pz)
{
    if (pz) z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
    return z;
}

// Producer warps of the warp-specialised sweeps: stream the planes z0 - 2 .. z1 + 1
// of every tile of this block (p, b and the three face arrays) into the ring of
// R plane slots.  Group g, the g-th plane streamed, lands in slot g mod R and
// completes on full[g mod R] (TMA boxes with zero fill when the tile's box needs
// no periodic wrap in x or y, else 16-byte asynchronous copies of the producers'
// lanes), once the consumers have released the slot's previous group on empty[].
// pt: producer thread 0 .. kProducers - 1.
template <class TC>
__device__ __forceinline__ void sweep_produce(const TaskList<SweepTask<float, TC>>& tl, float* smem, uint64_t* full,
                                              uint64_t* empty, volatile int* dead, int pt, int tries)
{
    constexpr int TX = kSweepTX, TY = kSweepTY;
    constexpr int XO = 4, SW = TX + 8, PL = SW * (TY + 4);
    constexpr int R = kSweepRing;
    constexpr int CPR = SW / 4, NCH = PL / 4;
    const int lane = pt & 31;
    auto ring = [&](int a, uint32_t g) -> float* { return smem + (a * R + (int)(g % R)) * PL; };
    uint32_t g = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < tl.total && ok; tile += gridDim.x) {
        int local;
        const SweepTask<float, TC>* tp = task_of(tl, tile, local);
        if (tp->ctl && tp->ctl->done) continue;
        const int nx = tp->g.n[0], ny = tp->g.n[1], nz = tp->g.n[2];
        const int px = tp->g.per[0], py = tp->g.per[1], pz = tp->g.per[2];
        const int cx = local % tp->tiles_x, rest = local / tp->tiles_x;
        const int x0 = cx * TX, y0 = (rest % tp->tiles_y) * TY, z0 = (rest / tp->tiles_y) * tp->zchunk;
        const int z1 = min(nz, z0 + tp->zchunk);
        const int rot = tp->rot ? *tp->rot : 0;
        const int pidx = tp->in_role < 0 ? 0 : (tp->in_role + rot) % 3;
        const float* pin = tp->in_role < 0 ? nullptr : tp->buf[pidx];
        const TmaPlanes* tm = tp->tma;
        const bool use_tma = tm != nullptr && pin != nullptr && !(px && (x0 - XO < 0 || x0 + TX + XO > nx)) &&
                             !(py && (y0 - 2 < 0 || y0 + TY + 2 > ny));
        const float* src[5] = {pin, tp->b, tp->bx, tp->by, tp->bz};
        const int64_t plane = (int64_t)nx * ny;
        constexpr int CPL = (NCH + kProducers - 1) / kProducers;
        int coff[CPL];
        bool cok[CPL];
        if (!use_tma) {
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int c = pt + kProducers * i;
                const int sy = c / CPR, ch = c - sy * CPR;
                int x = x0 - XO + 4 * ch, y = y0 - 2 + sy;
                cok[i] = c < NCH && wrapc(x, nx, px) && wrapc(y, ny, py);
                coff[i] = cok[i] ? y * nx + x : 0;
            }
        }
        const int nh = (z1 - z0) + 4;                      // planes z0-2 .. z1+1
        for (int m = 0; m < nh; ++m, ++g) {
            if (g >= (uint32_t)R && !mbar_wait_live(&empty[g % R], ((g / R) - 1) & 1u, dead, tries)) {
                ok = false;
                break;
            }
            uint64_t* bar = &full[g % R];
            const int z = z0 - 2 + m;
            if (use_tma) {
                if (pt == 32) mbar_arrive(bar);            // the second producer warp's arrival
                if (pt == 0) {
                    const int zw = wrap_plane(z, nz, pz);
                    mbar_expect_tx(bar, 5 * kPlaneBytes);
                    tma_plane(ring(0, g), &tm->p[pidx], x0 - XO, y0 - 2, zw, bar);
                    tma_plane(ring(1, g), &tm->b, x0 - XO, y0 - 2, zw, bar);
                    tma_plane(ring(2, g), &tm->x, x0 - XO, y0 - 2, zw, bar);
                    tma_plane(ring(3, g), &tm->y, x0 - XO, y0 - 2, zw, bar);
                    tma_plane(ring(4, g), &tm->z, x0 - XO, y0 - 2, zw, bar);
                }
            } else {
                int zw = z;
                const bool zok = wrapc(zw, nz, pz);
                const int64_t zoff = (int64_t)zw * plane;
#pragma unroll
                for (int i = 0; i < CPL; ++i) {
                    const int c = pt + kProducers * i;
                    if (c < NCH) {
#pragma unroll
                        for (int a = 0; a < 5; ++a) {
                            const bool okc = zok && cok[i] && src[a] != nullptr;
                            cp_async16(ring(a, g) + 4 * c, okc ? src[a] + zoff + coff[i] : tp->b, okc);
                        }
                    }
                }
                cp_async_mbar_arrive(bar);
                __syncwarp();
                if (lane == 0) mbar_arrive(bar);
            }
        }
    }
    if (!ok && lane == 0) {
        atomicExch(&g_wait_fault, 1);
        *dead = 1;
    }
    // no copy may be in flight when the block exits (the consumers may have given
    // up): wait, bounded, for the last R groups issued
    for (uint32_t q = g > (uint32_t)R ? g - R : 0; q < g; ++q) mbar_wait(&full[q % R], (q / R) & 1u);
}

// ---------------------------------------------------------------- K1: warp-specialised sweep
//
// The pipelined sweep (same arithmetic as k_sweep_async, bit-identical) with two
// producer warps streaming the planes of p, b and the three face arrays into a
// ring of R plane slots while 8 consumer warps compute.  Group H(g), the g-th
// plane this block streams over all its tiles, lands in slot g mod R and
// completes on full[g mod R] (TMA boxes with zero fill when the tile's box
// needs no periodic wrap in x or y, else 16-byte asynchronous copies of the
// producer's lanes); the consumers release it on empty[] when no later step
// reads it.  Step u of a tile (red cells of plane kr = z0 - 1 + u on the tile
// and its one-cell ring, then black cells of plane kr - 1 on the tile) reads
// H(u) .. H(u + 2) = planes kr - 1 .. kr + 1; with a coarse correction it also
// waits for H(u + 3) and adds the correction to that p plane, which the next
// step reads first.  The red results go to a consumer-only ring (M); one named
// barrier per step separates the red and black phases.
constexpr int kSweepConsumers = 256;
constexpr int kSweepBlock = kSweepConsumers + kProducers;

template <bool CORR, class TC>
__global__ void __launch_bounds__(kSweepBlock, 3) k_sweep_ws(const __grid_constant__ TaskList<SweepTask<float, TC>> tl)
{
    constexpr int TX = kSweepTX, TY = kSweepTY;
    constexpr int XO = 4, SW = TX + 8, PL = SW * (TY + 4);
    constexpr int R = kSweepRing;
    constexpr int RPR = (TX + 2) / 2, NRED = RPR * (TY + 2);   // red cells of the tile and its ring
    constexpr int BPR = TX / 2, NBLK = BPR * TY;               // black cells of the tile (x-pairs)
    constexpr int BLK0 = kSweepConsumers - NBLK;               // black duty: the last NBLK consumers
    constexpr int AHEAD = CORR ? 3 : 2;                        // a step waits for H(u + AHEAD)
    static_assert(NRED <= kSweepConsumers && BLK0 >= 0 && AHEAD + 2 <= R && PL <= 2 * kSweepConsumers,
                  "thread and ring budget");
    extern __shared__ __align__(128) float smem[];             // rings 0 p, 1 b, 2-4 faces, 5 merged red (M)
    __shared__ __align__(8) uint64_t full[R];
    __shared__ __align__(8) uint64_t empty[R];
    __shared__ int s_dead;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    if (tid == 0) {
        for (int j = 0; j < R; ++j) {
            mbar_init(&full[j], kProducers / 32);   // one arrival per producer warp
            mbar_init(&empty[j], kSweepConsumers / 32);
        }
        s_dead = 0;
        fence_mbar_init();
    }
    __syncthreads();
    pdl_wait();
    volatile int* dead = &s_dead;
    const int tries = g_ring_tries;
    auto ring = [&](int a, uint32_t g) -> float* { return smem + (a * R + (int)(g % R)) * PL; };

    if (tid >= kSweepConsumers) {
        sweep_produce<TC>(tl, smem, full, empty, dead, tid - kSweepConsumers, tries);
        return;
    }

    // ---------------------------------------------------- consumer warps
    uint32_t g = 0;                             // first group of the current tile
    for (int tile = blockIdx.x; tile < tl.total; tile += gridDim.x) {
        int local;
        const SweepTask<float, TC>* tp = task_of(tl, tile, local);
        const Ctl* ctl = tp->ctl;
        if (ctl && ctl->done) continue;
        const int nx = tp->g.n[0], ny = tp->g.n[1], nz = tp->g.n[2];
        const int px = tp->g.per[0], py = tp->g.per[1], pz = tp->g.per[2];
        const int cx = local % tp->tiles_x, rest = local / tp->tiles_x;
        const int x0 = cx * TX, y0 = (rest % tp->tiles_y) * TY, z0 = (rest / tp->tiles_y) * tp->zchunk;
        const int z1 = min(nz, z0 + tp->zchunk);
        const int rot = tp->rot ? *tp->rot : 0;
        float* pout = tp->buf[(tp->out_role + rot) % 3];
        const float w = ctl ? (float)ctl->omega : tp->omega;

        // red duty: one red cell of the tile or its ring per thread (tid < NRED)
        const int ey = tid / RPR, jr = tid - ey * RPR;
        int yr = y0 - 1 + ey;
        const bool yr_ok = tid < NRED && wrapc(yr, ny, py);
        const bool yr_wall = yr == 0 && !py;
        const int sred = (ey + 1) * SW + XO - 1 + 2 * jr;
        int xr0 = x0 - 1 + 2 * jr, xr1 = xr0 + 1;
        const bool xr_wall0 = xr0 == 0 && !px, xr_wall1 = xr1 == 0 && !px;
        const bool xr_ok0 = wrapc(xr0, nx, px), xr_ok1 = wrapc(xr1, nx, px);
        const int red_par = (1 + (y0 - 1 + ey)) & 1;          // red member: (red_par + kr) & 1
        // black duty: one x-pair of a tile row (tid >= BLK0)
        const int bi = tid - BLK0;
        const int tyb = bi / BPR, jb = bi - tyb * BPR;
        const int yb = y0 + tyb, xb = x0 + 2 * jb;
        const bool blk_on = bi >= 0 && yb < ny && xb < nx;
        const int sblk = (tyb + 2) * SW + XO + 2 * jb;
        const bool yb_wall = yb == 0 && !py;
        const bool xb_wall = xb == 0 && !px;
        float* const out_col = pout + ((int64_t)(blk_on ? yb : 0) * nx + (blk_on ? xb : 0));
        const int64_t plane = (int64_t)nx * ny;

        // coarse correction of p planes: gathered into registers one step ahead
        const TC* corr = tp->corr;
        const int cf0 = tp->cf[0], cf1 = tp->cf[1], cf2 = tp->cf[2];
        const int gcx = nx / cf0, gcy = ny / cf1;
        int crr0 = 0, crr1 = 0;
        bool crok0 = false, crok1 = false;
        if (CORR) {
            for (int r = 0; r < 2; ++r) {
                const int e = tid + r * kSweepConsumers;
                if (e < PL) {
                    const int sy = e / SW, sx = e - sy * SW;
                    int x = x0 - XO + sx, y = y0 - 2 + sy;
                    const bool okp = wrapc(x, nx, px) && wrapc(y, ny, py);
                    const int off = okp ? (y / cf1) * gcx + x / cf0 : 0;
                    if (r == 0) { crok0 = okp; crr0 = off; } else { crok1 = okp; crr1 = off; }
                }
            }
        }
        auto corr_load = [&](int z, float& c0, float& c1) {
            c0 = c1 = 0.f;
            if (!CORR) return;
            int zw = z;
            if (!wrapc(zw, nz, pz)) return;
            const int64_t zoff = (int64_t)(zw / cf2) * gcx * gcy;
            if (crok0) c0 = ldv(corr, zoff + crr0);
            if (crok1) c1 = ldv(corr, zoff + crr1);
        };
        auto corr_add = [&](float* dst, float c0, float c1) {
            if (!CORR) return;
            dst[tid] += c0;
            if (tid + kSweepConsumers < PL) dst[tid + kSweepConsumers] += c1;
        };

        const int kr0 = z0 - 1;
        const int nsteps = (z1 - z0) + 2;                      // red planes z0-1 .. z1
        const int nh = nsteps + 2;                             // H(m): plane kr0 - 1 + m
        bool live = true;
        for (int m = 0; m < AHEAD && live; ++m)
            live = mbar_wait_live(&full[(g + m) % R], ((g + m) / R) & 1u, dead, tries);
        float cur0 = 0.f, cur1 = 0.f;
        if (CORR) {
            if (live) {
                for (int m = 0; m < 3; ++m) {
                    float c0, c1;
                    corr_load(kr0 - 1 + m, c0, c1);
                    corr_add(ring(0, g + m), c0, c1);
                }
                corr_load(kr0 + 2, cur0, cur1);
            }
        }
        // every consumer warp agrees that the tile's first planes arrived (and were corrected)
        {
            int any;
            asm volatile("{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.s32 %0, 1, 0, q;\n}\n"
                         : "=r"(any) : "r"((int)!live), "n"(kSweepConsumers) : "memory");
            live = !any;
        }
        // ring slots advance by one per step: sl holds H(u) (plane kr-1); sw and pw are the
        // slot and phase parity of H(u + AHEAD), the group this step waits for
        auto rs = [&](int arr, uint32_t slot) -> float* { return smem + (arr * R + (int)slot) * PL; };
        uint32_t sl = g % R, sw = (g + AHEAD) % R, pw = ((g + AHEAD) / R) & 1u;
        for (int u = 0; u < nsteps && live; ++u) {
            const uint32_t s0 = sl + 1 == R ? 0 : sl + 1, su = s0 + 1 == R ? 0 : s0 + 1;   // kr, kr+1
            const uint32_t sm = sl == 0 ? R - 1 : sl - 1;                                 // kr-2
            const int kr = kr0 + u;
            bool ok = true;
            if (u + AHEAD <= nh - 1) ok = mbar_wait_live(&full[sw], pw, dead, tries);
            if (CORR && ok && u + 3 <= nh - 1) {
                float nxt0, nxt1;
                corr_load(kr + 3, nxt0, nxt1);
                corr_add(rs(0, su + 1 == R ? 0 : su + 1), cur0, cur1);   // p(kr+2), first read in step u+1
                cur0 = nxt0;
                cur1 = nxt1;
            }
            // red cells of plane kr
            if (ok && tid < NRED) {
                int zk = kr;
                const bool zok = wrapc(zk, nz, pz);
                const int o = (red_par + kr) & 1;
                const int s = sred + o;
                float v = 0.f;
                if (zok && yr_ok && (o ? xr_ok1 : xr_ok0)) {
                    const float* P0 = rs(0, s0);
                    const float* X0 = rs(2, s0);
                    const float* Y0 = rs(3, s0);
                    const float* Z0 = rs(4, s0);
                    const float* Z1 = rs(4, su);
                    v = P0[s];
                    const float xl = (o ? xr_wall1 : xr_wall0) ? 0.f : X0[s];
                    const float yl = yr_wall ? 0.f : Y0[s];
                    const float zl = (kr == 0 && !pz) ? 0.f : Z0[s];
                    const float fl = face_flux(xl, P0[s - 1], X0[s + 1], P0[s + 1], yl, P0[s - SW], Y0[s + SW],
                                               P0[s + SW], zl, rs(0, sl)[s], Z1[s], rs(0, su)[s], v);
                    const float dg = diag_sum(xl, X0[s + 1], yl, Y0[s + SW], zl, Z1[s]);
                    v = gs_update(v, fl, dg, rs(1, s0)[s], w);
                }
                rs(5, s0)[s] = v;
            }
            // S2: red cells of kr merged (and corrections visible), faults agreed
            {
                int any;
                asm volatile("{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.s32 %0, 1, 0, q;\n}\n"
                             : "=r"(any) : "r"((int)!ok), "n"(kSweepConsumers) : "memory");
                if (any) {
                    live = false;
                    break;
                }
            }
            // black cells of plane kr-1; the pair's red cell comes from M
            if (u >= 2 && blk_on) {
                const int k = kr - 1;
                const int hb = ((xb + yb + k) & 1) ? 0 : 1;   // black member of the pair
                const int s = sblk + hb;
                const float* Mk = rs(5, sl);
                const float* Xk = rs(2, sl);
                const float* Yk = rs(3, sl);
                const float* Zk = rs(4, sl);
                const float* Zk1 = rs(4, s0);
                float v = rs(0, sl)[s];
                const float xl = (hb == 0 && xb_wall) ? 0.f : Xk[s];
                const float yl = yb_wall ? 0.f : Yk[s];
                const float zl = (k == 0 && !pz) ? 0.f : Zk[s];
                const float fl = face_flux(xl, Mk[s - 1], Xk[s + 1], Mk[s + 1], yl, Mk[s - SW], Yk[s + SW],
                                           Mk[s + SW], zl, rs(5, sm)[s], Zk1[s], rs(5, s0)[s], v);
                const float dg = diag_sum(xl, Xk[s + 1], yl, Yk[s + SW], zl, Zk1[s]);
                v = gs_update(v, fl, dg, rs(1, sl)[s], w);
                const float r = Mk[sblk + (1 - hb)];
                const float o0 = hb ? r : v, o1 = hb ? v : r;
                *reinterpret_cast<float2*>(out_col + (int64_t)k * plane) = make_float2(o0, o1);
            }
            // plane kr-1 (H(u)) is no longer read by this tile's later steps
            if (CORR) fence_proxy_async();                 // corrected p planes: generic writes before refills
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[sl]);
            sl = s0;
            if (++sw == R) {
                sw = 0;
                pw ^= 1u;
            }
        }
        if (!live) {
            if (tid == 0) {
                atomicExch(&g_wait_fault, 1);
                s_dead = 1;
            }
            return;
        }
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(&empty[(g + nsteps) % R]);
            mbar_arrive(&empty[(g + nsteps + 1) % R]);
        }
        g += nh;
    }
}

struct ResTile {
    const ResTask<float>* tp;
    int local, x0, y0, z0, z1;
    int pidx;                                   // buffer holding the iterate
    const float* pin;
};

__device__ __forceinline__ bool res_tile(const TaskList<ResTask<float>>& tl, int tile, ResTile& t)
{
    t.tp = task_of(tl, tile, t.local);
    if (t.tp->ctl && t.tp->ctl->done) return false;
    const int cx = t.local % t.tp->tiles_x;
    const int rest = t.local / t.tp->tiles_x;
    const int cy = rest % t.tp->tiles_y;
    const int cz = rest / t.tp->tiles_y;
    t.x0 = cx * kSweepTX;
    t.y0 = cy * kSweepTY;
    t.z0 = cz * t.tp->zchunk;
    t.z1 = min(t.tp->g.n[2], t.z0 + t.tp->zchunk);
    const int rot = t.tp->rot ? *t.tp->rot : 0;
    t.pidx = t.tp->role < 0 ? 0 : (t.tp->role + rot) % 3;
    t.pin = t.tp->role < 0 ? nullptr : t.tp->buf[t.pidx];
    return true;
}

__device__ void control_rule(Ctl& C, double rr);

// Sum of part[0 .. n) by the kResConsumers consumer threads in exactly the order of
// sum_range over kThreads threads (each consumer stands for threads tid and tid +
// kResConsumers of that block), so the folded control rule sees the same bits as
// k_control_cycle.  Result valid in consumer 0.
__device__ double consumer_sum(const double* part, int n, double* red)
{
    static_assert(kThreads == 2 * kResConsumers, "two virtual threads per consumer");
    const int tid = threadIdx.x, lane = tid & 31;
    double a = 0.0, b = 0.0;
    for (int i = tid; i < n; i += kThreads) a += __ldcg(part + i);
    for (int i = tid + kResConsumers; i < n; i += kThreads) b += __ldcg(part + i);
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
        red[tid >> 5] = a;
        red[(tid + kResConsumers) >> 5] = b;
    }
    asm volatile("bar.sync 1, %0;\n" ::"n"(kResConsumers) : "memory");
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    asm volatile("bar.sync 1, %0;\n" ::"n"(kResConsumers) : "memory");
    return s;
}

__global__ void __launch_bounds__(kResBlock, 4) k_residual_ws(const __grid_constant__ TaskList<ResTask<float>> tl)
{
    constexpr int TX = kSweepTX, TY = kSweepTY;
    constexpr int XO = 4, SW = TX + 8, PL = SW * (TY + 4);
    constexpr int R = kResRing;
    constexpr int CPR = SW / 4, NCH = PL / 4;
    constexpr int BPR = TX / 2;
    static_assert(BPR * TY == kResConsumers && BPR == 16, "one x-pair per consumer thread, two rows per warp");
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t full[R];
    __shared__ __align__(8) uint64_t empty[R];
    __shared__ double red[kResConsumers / 32];
    __shared__ int s_dead;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    if (tid == 0) {
        for (int j = 0; j < R; ++j) {
            mbar_init(&full[j], kProducers / 32);   // one arrival per producer warp
            mbar_init(&empty[j], kResConsumers / 32);
        }
        s_dead = 0;
        fence_mbar_init();
    }
    __syncthreads();
    pdl_wait();
    volatile int* dead = &s_dead;
    const int tries = g_ring_tries;
    auto ring = [&](int a, uint32_t g) -> float* { return smem + (a * R + (int)(g % R)) * PL; };

    if (tid >= kResConsumers) {
        // ------------------------------------------------ producer warps
        const int pt = tid - kResConsumers;                 // producer thread 0 .. kProducers-1
        uint32_t g = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < tl.total && ok; tile += gridDim.x) {
            ResTile t;
            if (!res_tile(tl, tile, t)) continue;
            const ResTask<float>* tp = t.tp;
            const int nx = tp->g.n[0], ny = tp->g.n[1], nz = tp->g.n[2];
            const int px = tp->g.per[0], py = tp->g.per[1], pz = tp->g.per[2];
            const TmaPlanes* tm = tp->tma;
            const bool use_tma = tm != nullptr && t.pin != nullptr &&
                                 !(px && (t.x0 - XO < 0 || t.x0 + TX + XO > nx)) &&
                                 !(py && (t.y0 - 2 < 0 || t.y0 + TY + 2 > ny));
            const CUtensorMap* pmap = use_tma ? &tm->p[t.pidx] : nullptr;
            const float* src[5] = {t.pin, tp->b, tp->bx, tp->by, tp->bz};
            const int64_t plane = (int64_t)nx * ny;
            const int nh = (t.z1 - t.z0) + 2;                  // planes z0-1 .. z1
            // per-thread copies: this lane's 16-byte chunks (c = lane + 32 i) of a plane, fixed for the tile
            constexpr int CPL = (NCH + kProducers - 1) / kProducers;
            int coff[CPL];
            bool cok[CPL];
            if (!use_tma) {
#pragma unroll
                for (int i = 0; i < CPL; ++i) {
                    const int c = pt + kProducers * i;
                    const int sy = c / CPR, ch = c - sy * CPR;
                    int x = t.x0 - XO + 4 * ch, y = t.y0 - 2 + sy;
                    cok[i] = c < NCH && wrapc(x, nx, px) && wrapc(y, ny, py);
                    coff[i] = cok[i] ? y * nx + x : 0;
                }
            }
            for (int m = 0; m < nh; ++m, ++g) {
                if (g >= (uint32_t)R && !mbar_wait_live(&empty[g % R], ((g / R) - 1) & 1u, dead, tries)) {
                    ok = false;
                    break;
                }
                uint64_t* bar = &full[g % R];
                const int z = t.z0 - 1 + m;
                if (use_tma) {
                    if (pt == 32) mbar_arrive(bar);            // the second producer warp's arrival
                    if (pt == 0) {
                        const int zw = wrap_plane(z, nz, pz);
                        mbar_expect_tx(bar, 5 * kPlaneBytes);
                        tma_plane(ring(0, g), pmap, t.x0 - XO, t.y0 - 2, zw, bar);
                        tma_plane(ring(1, g), &tm->b, t.x0 - XO, t.y0 - 2, zw, bar);
                        tma_plane(ring(2, g), &tm->x, t.x0 - XO, t.y0 - 2, zw, bar);
                        tma_plane(ring(3, g), &tm->y, t.x0 - XO, t.y0 - 2, zw, bar);
                        tma_plane(ring(4, g), &tm->z, t.x0 - XO, t.y0 - 2, zw, bar);
                    }
                } else {
                    int zw = z;
                    const bool zok = wrapc(zw, nz, pz);
                    const int64_t zoff = (int64_t)zw * plane;
#pragma unroll
                    for (int i = 0; i < CPL; ++i) {
                        const int c = pt + kProducers * i;
                        if (c < NCH) {
#pragma unroll
                            for (int a = 0; a < 5; ++a) {
                                const bool okc = zok && cok[i] && src[a] != nullptr;
                                cp_async16(ring(a, g) + 4 * c, okc ? src[a] + zoff + coff[i] : tp->b, okc);
                            }
                        }
                    }
                    cp_async_mbar_arrive(bar);
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar);
                }
            }
        }
        if (!ok && lane == 0) {
            atomicExch(&g_wait_fault, 1);
            s_dead = 1;
        }
        // no copy may be in flight when the block exits (the consumers may have
        // given up): wait, bounded, for the last R groups issued
        for (uint32_t q = g > (uint32_t)R ? g - R : 0; q < g; ++q) mbar_wait(&full[q % R], (q / R) & 1u);
        return;
    }

    // ---------------------------------------------------- consumer warps
    const int tyb = tid / BPR, jb = tid - tyb * BPR;
    uint32_t g = 0;                             // first group of the current tile
    for (int tile = blockIdx.x; tile < tl.total; tile += gridDim.x) {
        ResTile t;
        if (!res_tile(tl, tile, t)) continue;
        const ResTask<float>* tp = t.tp;
        const int nx = tp->g.n[0], ny = tp->g.n[1];
        const int px = tp->g.per[0], py = tp->g.per[1], pz = tp->g.per[2];
        float* const bc = tp->bc;
        const int c0 = tp->cf[0], c1 = tp->cf[1], c2 = tp->cf[2];
        const int yb = t.y0 + tyb, xb = t.x0 + 2 * jb;
        const bool pair_on = yb < ny && xb < nx;
        const int sp = (tyb + 2) * SW + XO + 2 * jb;
        const bool yb_wall = yb == 0 && !py;
        const bool xb_wall = xb == 0 && !px;
        const int gcx = nx / c0, gcy = ny / c1;
        const bool writer = pair_on && (c1 == 1 || (tyb & 1) == 0);
        const int64_t cplane = (int64_t)gcx * gcy;
        const int64_t crow = (int64_t)(yb / c1) * gcx + xb / c0;
        const int nsteps = t.z1 - t.z0;
        // r^2 is summed in FP32 over at most kNormFold planes (2 * kNormFold terms), then
        // added into an FP64 total: FP64 arithmetic runs at 1/64 of the FP32 rate here, and
        // one FP64 add per 2 * kNormFold cells keeps it off the critical path.  The FP32
        // partial's relative error is below 2 * kNormFold * 2^-24 (< 1e-6).
        constexpr int kNormFold = 8;
        double rr = 0.0;
        float rr32 = 0.f;
        int fold = kNormFold;
        float acc0 = 0.f, acc1 = 0.f;
        bool live = mbar_wait_live(&full[g % R], (g / R) & 1u, dead, tries) &&
                    mbar_wait_live(&full[(g + 1) % R], ((g + 1) / R) & 1u, dead, tries);
        auto rs = [&](int arr, uint32_t slot) -> float* { return smem + (arr * R + (int)slot) * PL; };
        uint32_t sl = g % R, sw = (g + 2) % R, pw = ((g + 2) / R) & 1u;   // H(u); H(u+2) and its parity
        for (int u = 0; u < nsteps && live; ++u) {
            const uint32_t s0 = sl + 1 == R ? 0 : sl + 1, su = sw;      // planes k, k+1
            if (!mbar_wait_live(&full[sw], pw, dead, tries)) {
                live = false;
                break;
            }
            const int k = t.z0 + u;
            float r0 = 0.f, r1 = 0.f;
            if (pair_on) {
                const float* P0 = rs(0, s0);
                const float* Pl = rs(0, sl);
                const float* Pu = rs(0, su);
                const float* B0 = rs(1, s0);
                const float* X0 = rs(2, s0);
                const float* Y0 = rs(3, s0);
                const float* Z0 = rs(4, s0);
                const float* Z1 = rs(4, su);
                for (int h = 0; h < 2; ++h) {
                    const int s = sp + h;
                    const float p0 = P0[s];
                    const float xl = (h == 0 && xb_wall) ? 0.f : X0[s];
                    const float yl = yb_wall ? 0.f : Y0[s];
                    const float zl = (k == 0 && !pz) ? 0.f : Z0[s];
                    const float fl = face_flux(xl, P0[s - 1], X0[s + 1], P0[s + 1], yl, P0[s - SW], Y0[s + SW],
                                               P0[s + SW], zl, Pl[s], Z1[s], Pu[s], p0);
                    const float r = B0[s] - fl;
                    if (h == 0) r0 = r; else r1 = (xb + 1 < nx) ? r : 0.f;
                }
                rr32 = fmaf(r1, r1, fmaf(r0, r0, rr32));
                if (--fold == 0) {
                    rr += (double)rr32;
                    rr32 = 0.f;
                    fold = kNormFold;
                }
            }
            // plane k-1 is no longer read
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[sl]);
            sl = s0;
            if (++sw == R) {
                sw = 0;
                pw ^= 1u;
            }
            if (bc) {
                float v0 = c0 == 2 ? r0 + r1 : r0;
                float v1 = c0 == 2 ? 0.f : r1;
                if (c1 == 2) {
                    v0 += __shfl_xor_sync(0xffffffffu, v0, 16);
                    v1 += __shfl_xor_sync(0xffffffffu, v1, 16);
                }
                acc0 += v0;
                acc1 += v1;
                if (c2 == 1 || (k & 1) == 1) {
                    if (writer) {
                        float* dst = bc + (int64_t)(k / c2) * cplane + crow;
                        dst[0] = acc0;
                        if (c0 == 1 && xb + 1 < nx) dst[1] = acc1;
                    }
                    acc0 = acc1 = 0.f;
                }
            }
        }
        if (live) {
            // planes z1-1 and z1 (the last two groups of the tile) are released too
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&empty[(g + nsteps) % R]);
                mbar_arrive(&empty[(g + nsteps + 1) % R]);
            }
        }
        g += nsteps + 2;
        // all consumer warps agree on faults before the tile's norm partial
        int any_dead;
        asm volatile("{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.s32 %0, 1, 0, q;\n}\n"
                     : "=r"(any_dead)
                     : "r"((int)!live), "n"(kResConsumers)
                     : "memory");
        if (any_dead) {
            if (tid == 0) {
                atomicExch(&g_wait_fault, 1);
                s_dead = 1;
            }
            break;   // still counted below, so that a folded control rule is not left waiting
        }
        if (tp->partials) {
            const double q = warp_sum(rr + (double)rr32);
            if (lane == 0) red[tid >> 5] = q;
            asm volatile("bar.sync 1, %0;\n" ::"n"(kResConsumers) : "memory");
            if (tid == 0) {
                double s = 0.0;
                for (int i = 0; i < kResConsumers / 32; ++i) s += red[i];
                tp->partials[t.local] = s;
            }
            asm volatile("bar.sync 1, %0;\n" ::"n"(kResConsumers) : "memory");
        }
    }

    // control rule folded into the fine-level norm (Sec. 3.1): the last block to
    // finish sums every task's partials and updates its control state
    if (tl.ctl_tasks) {
        __shared__ int s_last;
        __shared__ double red_ctl[kThreads / 32];
        if (tid == 0) {
            __threadfence();                       // this block's partials before its arrival
            s_last = atomicAdd(tl.arrivals, 1u) == gridDim.x - 1;
        }
        asm volatile("bar.sync 1, %0;\n" ::"n"(kResConsumers) : "memory");
        if (s_last) {
            __threadfence();
            for (int k = 0; k < tl.nctl; ++k) {
                const CtlTask& ct = tl.ctl_tasks[k];
                if (*(volatile const int*)&ct.ctl->done) continue;   // the same value in every thread
                const double rr = consumer_sum(ct.partials, ct.nparts, red_ctl);
                if (tid == 0) control_rule(*ct.ctl, rr);
            }
            if (tid == 0) *tl.arrivals = 0u;     // ready for the next launch
        }
    }
}

// reference sweep: one colour per launch, in place, one thread per cell
__global__ void k_sweep_colour(Geo g, const float* __restrict__ bx, const float* __restrict__ by,
                               const float* __restrict__ bz, const float* __restrict__ b, float* p,
                               float w, int colour)
{
    const int64_t N = (int64_t)g.n[0] * g.n[1] * g.n[2];
    for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < N;
         I += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(I % g.n[0]);
        const int y = (int)((I / g.n[0]) % g.n[1]);
        const int z = (int)(I / ((int64_t)g.n[0] * g.n[1]));
        if (((x + y + z) & 1) != colour) continue;
        auto pv = [&](int xx, int yy, int zz) -> float {
            if (!wrapc(xx, g.n[0], g.per[0]) || !wrapc(yy, g.n[1], g.per[1]) ||
                !wrapc(zz, g.n[2], g.per[2]))
                return 0.f;
            return p[lin(g, xx, yy, zz)];
        };
        const float fxl = face_lo(bx, g, 0, x, y, z), fxu = face_lo(bx, g, 0, x + 1, y, z);
        const float fyl = face_lo(by, g, 1, x, y, z), fyu = face_lo(by, g, 1, x, y + 1, z);
        const float fzl = face_lo(bz, g, 2, x, y, z), fzu = face_lo(bz, g, 2, x, y, z + 1);
        const float p0 = p[I];
        const float fl = face_flux(fxl, pv(x - 1, y, z), fxu, pv(x + 1, y, z), fyl, pv(x, y - 1, z), fyu,
                                   pv(x, y + 1, z), fzl, pv(x, y, z - 1), fzu, pv(x, y, z + 1), p0);
        const float dg = diag_sum(fxl, fxu, fyl, fyu, fzl, fzu);
        p[I] = gs_update(p0, fl, dg, __ldg(b + I), w);
    }
}

// ---------------------------------------------------------------- K2: residual

template <class TP>
__global__ void __launch_bounds__(kThreads) k_residual(const __grid_constant__ TaskList<ResTask<TP>> tl)
{
    __shared__ float sr[kResTZ][kResTY][kResTX];
    __shared__ double red[kThreads / 32];
    pdl_wait();
    const int tx = threadIdx.x % kResTX;
    const int ty = (threadIdx.x / kResTX) % kResTY;
    const int tz = threadIdx.x / (kResTX * kResTY);

    for (int tile = blockIdx.x; tile < tl.total; tile += gridDim.x) {
        int local;
        const ResTask<TP>* tp = task_of(tl, tile, local);
        if (tp->ctl && tp->ctl->done) continue;
        const Geo g = tp->g;
        const int cx = local % tp->tiles_x;
        const int rest = local / tp->tiles_x;
        const int cy = rest % tp->tiles_y;
        const int cz = rest / tp->tiles_y;
        const int x = cx * kResTX + tx, y = cy * kResTY + ty, z = cz * kResTZ + tz;
        const int rot = tp->rot ? *tp->rot : 0;
        const TP* p = tp->role < 0 ? nullptr : tp->buf[(tp->role + rot) % 3];
        const bool in = x < g.n[0] && y < g.n[1] && z < g.n[2];
        float r = 0.f;
        if (in) {
            auto pv = [&](int xx, int yy, int zz) -> float {
                if (!p) return 0.f;
                if (!wrapc(xx, g.n[0], g.per[0]) || !wrapc(yy, g.n[1], g.per[1]) ||
                    !wrapc(zz, g.n[2], g.per[2]))
                    return 0.f;
                return ldv(p, lin(g, xx, yy, zz));
            };
            const float fxl = face_lo(tp->bx, g, 0, x, y, z), fxu = face_lo(tp->bx, g, 0, x + 1, y, z);
            const float fyl = face_lo(tp->by, g, 1, x, y, z), fyu = face_lo(tp->by, g, 1, x, y + 1, z);
            const float fzl = face_lo(tp->bz, g, 2, x, y, z), fzu = face_lo(tp->bz, g, 2, x, y, z + 1);
            const float Ap = face_flux(fxl, pv(x - 1, y, z), fxu, pv(x + 1, y, z), fyl, pv(x, y - 1, z),
                                       fyu, pv(x, y + 1, z), fzl, pv(x, y, z - 1), fzu, pv(x, y, z + 1),
                                       pv(x, y, z));
            r = __ldg(tp->b + lin(g, x, y, z)) - Ap;
        }
        if (tp->bc) {
            float v = r;
            if (tp->cf[0] == 2) v += __shfl_xor_sync(0xffffffffu, v, 1);
            sr[tz][ty][tx] = v;
            __syncthreads();
            if (in && (tx % tp->cf[0]) == 0 && (ty % tp->cf[1]) == 0 && (tz % tp->cf[2]) == 0) {
                float s = 0.f;
                for (int dz = 0; dz < tp->cf[2]; ++dz)
                    for (int dy = 0; dy < tp->cf[1]; ++dy) s += sr[tz + dz][ty + dy][tx];
                Geo gc = g;
                gc.n[0] /= tp->cf[0]; gc.n[1] /= tp->cf[1]; gc.n[2] /= tp->cf[2];
                tp->bc[lin(gc, x / tp->cf[0], y / tp->cf[1], z / tp->cf[2])] = s;
            }
            __syncthreads();
        }
        if (tp->partials) {
            const double q = block_sum_sq(r, red);
            if (threadIdx.x == 0) tp->partials[local] = q;
        }
    }
}

// one block per task: b <- b - mean over active cells (0 on inactive cells)
__global__ void __launch_bounds__(kThreads) k_project_level(const LevelProjTask* __restrict__ tasks)
{
    __shared__ double red[kThreads / 32];
    __shared__ double s_mean;
    const LevelProjTask& T = tasks[blockIdx.x];
    if (T.ctl && T.ctl->done) return;
    const Geo g = T.g;
    const int64_t N = (int64_t)g.n[0] * g.n[1] * g.n[2];
    auto active = [&](int64_t i) -> bool {
        const int x = (int)(i % g.n[0]);
        const int y = (int)((i / g.n[0]) % g.n[1]);
        const int z = (int)(i / ((int64_t)g.n[0] * g.n[1]));
        const float dg = diag_sum(face_lo(T.bx, g, 0, x, y, z), face_lo(T.bx, g, 0, x + 1, y, z),
                                  face_lo(T.by, g, 1, x, y, z), face_lo(T.by, g, 1, x, y + 1, z),
                                  face_lo(T.bz, g, 2, x, y, z), face_lo(T.bz, g, 2, x, y, z + 1));
        return dg > 0.f;
    };
    double s = 0.0, cnt = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += kThreads)
        if (active(i)) {
            s += (double)T.b[i];
            cnt += 1.0;
        }
    s = block_sum(s, red);
    cnt = block_sum(cnt, red);
    if (threadIdx.x == 0) s_mean = cnt > 0.0 ? s / cnt : 0.0;
    __syncthreads();
    const double mean = s_mean;
    for (int64_t i = threadIdx.x; i < N; i += kThreads)
        T.b[i] = active(i) ? (float)((double)T.b[i] - mean) : 0.f;
}

// ---------------------------------------------------------------- K7 and transfers

// C4: coarse face = (1/c_d) sum of the fine faces it covers (finite volume), or
// the sum itself (galerkin: the faces of R A P, piecewise-constant P)
__global__ void k_coarsen(Geo f, int c0, int c1, int c2, const float* __restrict__ bx,
                          const float* __restrict__ by, const float* __restrict__ bz, float* cbx,
                          float* cby, float* cbz, int galerkin)
{
    Geo cg = f;
    cg.n[0] = f.n[0] / c0; cg.n[1] = f.n[1] / c1; cg.n[2] = f.n[2] / c2;
    const int cfac[3] = {c0, c1, c2};
    const float* fa[3] = {bx, by, bz};
    float* ca[3] = {cbx, cby, cbz};
    const int64_t N = (int64_t)cg.n[0] * cg.n[1] * cg.n[2];
    for (int64_t J = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; J < N;
         J += (int64_t)gridDim.x * blockDim.x) {
        const int X = (int)(J % cg.n[0]);
        const int Y = (int)((J / cg.n[0]) % cg.n[1]);
        const int Z = (int)(J / ((int64_t)cg.n[0] * cg.n[1]));
        const int Jc[3] = {X, Y, Z};
        for (int d = 0; d < 3; ++d) {
            int lo[3], hi[3];
            for (int e = 0; e < 3; ++e) {
                lo[e] = cfac[e] * Jc[e];
                hi[e] = e == d ? lo[e] + 1 : lo[e] + cfac[e];
            }
            float s = 0.f;
            for (int z = lo[2]; z < hi[2]; ++z)
                for (int y = lo[1]; y < hi[1]; ++y)
                    for (int x = lo[0]; x < hi[0]; ++x) s += face_lo(fa[d], f, d, x, y, z);
            ca[d][J] = galerkin ? s : s / (float)cfac[d];
        }
    }
}

__global__ void k_prolong_add(Geo f, int c0, int c1, int c2, const float* __restrict__ e, float* p)
{
    Geo cg = f;
    cg.n[0] = f.n[0] / c0; cg.n[1] = f.n[1] / c1; cg.n[2] = f.n[2] / c2;
    const int64_t N = (int64_t)f.n[0] * f.n[1] * f.n[2];
    for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < N;
         I += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(I % f.n[0]);
        const int y = (int)((I / f.n[0]) % f.n[1]);
        const int z = (int)(I / ((int64_t)f.n[0] * f.n[1]));
        p[I] += __ldg(e + lin(cg, x / c0, y / c1, z / c2));
    }
}

// buf[role] += e[I / c] by 16-byte chunks of 4 cells of a row (fine rows of a
// multiple of 4 cells); the same FP32 addition as the correction folded into a
// sweep's plane loads, so both give the same iterate bit for bit.
__global__ void __launch_bounds__(kThreads) k_prolong_rows(const __grid_constant__ ProlongTask t)
{
    pdl_wait();
    const int nx = t.g.n[0], ny = t.g.n[1], nz = t.g.n[2];
    const int cpr = nx / 4;                                  // chunks per row
    const int gcx = nx / t.cf[0], gcy = ny / t.cf[1];
    const int sy = t.cf[1] - 1, sz = t.cf[2] - 1;             // shifts: factor 2 -> 1, 1 -> 0
    const int rot = t.rot ? *t.rot : 0;
    float* p = t.buf[(t.role + rot) % 3];
    const int64_t total = (int64_t)cpr * ny * nz;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = k / cpr;
        const int c = (int)(k - row * cpr);
        const int y = (int)(row % ny), z = (int)(row / ny);
        const int64_t crow = ((int64_t)(z >> sz) * gcy + (y >> sy)) * gcx;
        float4 v = *reinterpret_cast<float4*>(p + 4 * k);
        if (t.cf[0] == 2) {
            const float2 e2 = __ldg(reinterpret_cast<const float2*>(t.e + crow + 2 * c));
            v.x += e2.x;
            v.y += e2.x;
            v.z += e2.y;
            v.w += e2.y;
        } else {
            const float4 e4 = __ldg(reinterpret_cast<const float4*>(t.e + crow + 4 * c));
            v.x += e4.x;
            v.y += e4.y;
            v.z += e4.z;
            v.w += e4.w;
        }
        *reinterpret_cast<float4*>(p + 4 * k) = v;
    }
}

__global__ void k_active_mask(Geo g, const float* __restrict__ bx, const float* __restrict__ by,
                              const float* __restrict__ bz, uint8_t* mask)
{
    const int64_t N = (int64_t)g.n[0] * g.n[1] * g.n[2];
    for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < N;
         I += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(I % g.n[0]);
        const int y = (int)((I / g.n[0]) % g.n[1]);
        const int z = (int)(I / ((int64_t)g.n[0] * g.n[1]));
        const float dg = diag_sum(face_lo(bx, g, 0, x, y, z), face_lo(bx, g, 0, x + 1, y, z),
                                  face_lo(by, g, 1, x, y, z), face_lo(by, g, 1, x, y + 1, z),
                                  face_lo(bz, g, 2, x, y, z), face_lo(bz, g, 2, x, y, z + 1));
        mask[I] = dg > 0.f ? 1 : 0;
    }
}

__global__ void k_check_coeffs(int64_t n, const float* __restrict__ bx, const float* __restrict__ by,
                               const float* __restrict__ bz, int* bad)
{
    int local = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float a = bx[i], b = by[i], c = bz[i];
        if (!(a >= 0.f && a <= 3.0e38f) || !(b >= 0.f && b <= 3.0e38f) || !(c >= 0.f && c <= 3.0e38f))
            local = 1;
    }
    if (__any_sync(0xffffffffu, local) && (threadIdx.x & 31) == 0) atomicAdd(bad, 1);
}

__global__ void k_sum_partials(const double* __restrict__ part, int n, double* out)
{
    __shared__ double red[kThreads / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *out = s;
}

// ---------------------------------------------------------------- projection and gauge

template <class TS>
__global__ void __launch_bounds__(kThreads) k_project_sum(const __grid_constant__ TaskList<ProjTask<TS>> tl)
{
    __shared__ double red[kThreads / 32];
    for (int tile = blockIdx.x; tile < tl.total; tile += gridDim.x) {
        int local;
        const ProjTask<TS>* t = task_of(tl, tile, local);
        const int64_t beg = (int64_t)local * kElemTile;
        const int64_t end = min(t->n, beg + kElemTile);
        // the sum in FP64 (the mean must be exact to the solve's tolerance); the
        // counts, at most kElemTile / kThreads per thread, in FP32 (exact)
        double s = 0.0;
        float c32 = 0.f, bad32 = 0.f;
        for (int64_t i = beg + threadIdx.x; i < end; i += kThreads) {
            const double v = (double)t->sigma[i];
            if (!isfinite(v)) bad32 += 1.f;
            if (t->mask[i]) {
                s += v;
                c32 += 1.f;
            }
        }
        s = block_sum(s, red);
        const double c = block_sum((double)c32, red);
        const double bad = block_sum((double)bad32, red);
        if (threadIdx.x == 0) {
            t->partials[3 * local + 0] = s;
            t->partials[3 * local + 1] = c;
            t->partials[3 * local + 2] = bad;
        }
    }
}

template <class TS>
__global__ void __launch_bounds__(kThreads) k_project_apply(const __grid_constant__ TaskList<ProjTask<TS>> tl)
{
    __shared__ double red[kThreads / 32];
    for (int tile = blockIdx.x; tile < tl.total; tile += gridDim.x) {
        int local;
        const ProjTask<TS>* t = task_of(tl, tile, local);
        const double mean = t->ctl->mean;
        const int64_t beg = (int64_t)local * kElemTile;
        const int64_t end = min(t->n, beg + kElemTile);
        // |b|^2: for an FP32 right-hand side, FP32 squares over the kElemTile / kThreads
        // cells of a thread, then FP64 (relative error below 2^-20); FP64 squares for
        // an FP64 one (no range limit)
        float q32 = 0.f;
        double q64 = 0.0;
        for (int64_t i = beg + threadIdx.x; i < end; i += kThreads) {
            const bool act = t->mask[i] != 0;
            const double bv = act ? (double)t->sigma[i] - mean : 0.0;
            if (t->b32) {
                const float f = (float)bv;
                t->b32[i] = f;
                q32 = fmaf(f, f, q32);
            } else {
                t->b64[i] = bv;
                q64 = fma(bv, bv, q64);
            }
            const double pv = (act && t->p_in) ? (double)t->p_in[i] : 0.0;
            if (t->p32) t->p32[i] = (float)pv;
            if (t->p64) t->p64[i] = pv;
        }
        const double q = block_sum((double)q32 + q64, red);
        if (threadIdx.x == 0) t->bpartials[local] = q;
    }
}

template <class TP, class TD>
__global__ void __launch_bounds__(kThreads) k_gauge_sum(const __grid_constant__ TaskList<GaugeTask<TP, TD>> tl)
{
    __shared__ double red[kThreads / 32];
    for (int tile = blockIdx.x; tile < tl.total; tile += gridDim.x) {
        int local;
        const GaugeTask<TP, TD>* t = task_of(tl, tile, local);
        const int rot = t->rot ? *t->rot : 0;
        const TP* p = t->buf[rot % 3];
        const int64_t beg = (int64_t)local * kElemTile;
        const int64_t end = min(t->n, beg + kElemTile);
        double s = 0.0;
        for (int64_t i = beg + threadIdx.x; i < end; i += kThreads)
            if (t->mask[i]) s += (double)p[i];
        s = block_sum(s, red);
        if (threadIdx.x == 0) t->partials[local] = s;
    }
}

template <class TP, class TD>
__global__ void __launch_bounds__(kThreads) k_gauge_apply(const __grid_constant__ TaskList<GaugeTask<TP, TD>> tl)
{
    for (int tile = blockIdx.x; tile < tl.total; tile += gridDim.x) {
        int local;
        const GaugeTask<TP, TD>* t = task_of(tl, tile, local);
        const int rot = t->rot ? *t->rot : 0;
        const TP* p = t->buf[rot % 3];
        if (t->ctl->status == kNonFinite) continue;   // the caller's p stays untouched
        const double mean = t->ctl->mean;
        const bool zero = t->ctl->zero_out != 0;
        const int64_t beg = (int64_t)local * kElemTile;
        const int64_t end = min(t->n, beg + kElemTile);
        for (int64_t i = beg + threadIdx.x; i < end; i += kThreads) {
            const double v = (!zero && t->mask[i]) ? (double)p[i] - mean : 0.0;
            t->dst[i] = (TD)v;
        }
    }
}

// one block per problem: sums in a fixed order
__device__ double sum_range(const double* part, int n, int stride, int off, double* red)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[(int64_t)i * stride + off];
    return block_sum(s, red);
}

__global__ void k_project_finalize(const CtlTask* __restrict__ tasks)
{
    __shared__ double red[kThreads / 32];
    const CtlTask& t = tasks[blockIdx.x];
    const double s = sum_range(t.ppartials, t.npparts, 3, 0, red);
    const double c = sum_range(t.ppartials, t.npparts, 3, 1, red);
    const double bad = sum_range(t.ppartials, t.npparts, 3, 2, red);
    if (threadIdx.x == 0) {
        Ctl& C = *t.ctl;
        C.stat_cnt = c;
        C.mean = c > 0.0 ? s / c : 0.0;
        C.nonfinite = bad > 0.0 ? 1 : 0;
    }
}

__global__ void k_gauge_finalize(const CtlTask* __restrict__ tasks)
{
    __shared__ double red[kThreads / 32];
    const CtlTask& t = tasks[blockIdx.x];
    const double s = sum_range(t.ppartials, t.npparts, 1, 0, red);
    if (threadIdx.x == 0) {
        Ctl& C = *t.ctl;
        C.mean = C.stat_cnt > 0.0 ? s / C.stat_cnt : 0.0;
    }
}

// ---------------------------------------------------------------- K6: control

__global__ void k_control_init(const CtlTask* __restrict__ tasks)
{
    __shared__ double red[kThreads / 32];
    const CtlTask& t = tasks[blockIdx.x];
    const double bb = sum_range(t.bpartials, t.nbparts, 1, 0, red);
    const double rr = t.partials ? sum_range(t.partials, t.nparts, 1, 0, red) : bb;
    if (threadIdx.x == 0) {
        Ctl& C = *t.ctl;
        C.bnorm = sqrt(bb);
        C.cycles = 0;
        C.total_cycles = 0;
        C.rot = 0;
        C.zero_out = 0;
        C.hist_scale = C.bnorm > 0.0 ? 1.0 / C.bnorm : 0.0;
        if (C.nonfinite) {
            C.status = kNonFinite;
            C.done = 1;
        } else if (C.bnorm == 0.0) {
            C.status = kOk;
            C.zero_out = 1;
            C.done = 1;
            if (C.hist_cap >= 0) C.hist_res[0] = 0.0;
        } else {
            C.r_prev = sqrt(rr);
            C.hist_res[0] = C.r_prev * C.hist_scale;   // the same rounding as every later entry
            if (C.r_prev / C.bnorm <= C.tol) {
                C.status = kOk;
                C.done = 1;
            } else {
                C.status = kRunning;
                C.done = 0;
            }
        }
    }
}

// the adaptive relaxation rule after one V-cycle (Sec. 3.1), from the fine
// residual's squared norm rr; one thread
__device__ void control_rule(Ctl& C, double rr)
{
    const double rk = sqrt(rr);
    const double w = C.omega;
    // a relaxation factor that is not a positive finite number means the control
    // state is corrupt: the solve stops as diverged with the accepted iterate
    const bool w_ok = isfinite(w) && w > 0.0;
    const bool acc = w_ok && rk < C.r_prev;     // NaN rejects
    C.r_last = rk;
    C.cycles += 1;
    C.total_cycles += 1;
    if (!w_ok) {
        C.status = kDiverged;
    } else if (acc) {
        C.rot = (C.rot + C.res_role) % 3;
        C.r_prev = rk;
        C.omega = fmin(1.0, C.grow * w);
    } else if (w <= C.omega_min) {
        C.status = kDiverged;
    } else {
        C.omega = fmax(C.omega_min, C.shrink * w);
    }
    const int k = C.total_cycles;
    if (k <= C.hist_cap) {
        C.hist_res[k] = C.r_prev * C.hist_scale;
        C.hist_omega[k - 1] = w;
        C.hist_acc[k - 1] = acc ? 1 : 0;
    }
    if (C.status != kDiverged && C.r_prev / C.bnorm <= C.tol) C.status = kOk;
    else if (C.status == kRunning && C.cycles >= C.max_cycles) C.status = kNotConverged;
    if (C.status != kRunning) C.done = 1;
}

__global__ void k_control_cycle(const CtlTask* __restrict__ tasks)
{
    __shared__ double red[kThreads / 32];
    pdl_wait();
    const CtlTask& t = tasks[blockIdx.x];
    if (t.ctl->done) return;   // uniform in the block
    const double rr = sum_range(t.partials, t.nparts, 1, 0, red);
    if (threadIdx.x == 0) control_rule(*t.ctl, rr);
}

// ---------------------------------------------------------------- K9: FP64 refinement

// ---------------------------------------------------------------- double-length FP32 arithmetic
//
// A value held as an unevaluated sum hi + lo of two FP32 numbers (Dekker,
// "A floating-point technique for extending the available precision", 1971):
// error-free sums (Knuth's two-sum; Dekker's fast two-sum when |a| >= |b|) and
// the error-free product with a fused multiply-add give about 44 significant
// bits on the FP32 pipe, which on this part runs 64 times the FP64 rate.
// Every rounding is spelled out, so no compiled contraction changes them.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ DF fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    DF s = two_sum(a.hi, b.hi);
    const DF t = two_sum(a.lo, b.lo);
    s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

// a * b for an FP32 b
__device__ __forceinline__ DF df_mul(DF a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    const float e = __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p));
    return fast_two_sum(p, e);
}

// x (FP64) as hi + lo without FP64 arithmetic: hi takes the leading 24 bits of
// the significand (truncated, exact), lo the 29 bits below them rounded to 24,
// so |x - hi - lo| <= 2^-47 |x|.  false when x lies outside the range this
// covers (|x| >= 2^128, non-finite, or |x| < 2^-74, where lo would underflow;
// zero is covered exactly).
__device__ __forceinline__ bool split64(double x, DF& out)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    if ((u << 1) == 0) {
        out = {0.f, 0.f};
        return true;
    }
    const int ef = (int)((u >> 52) & 0x7ff) - 1023 + 127;   // FP32 biased exponent of hi
    if (ef < 53 || ef > 254) return false;
    const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
    const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
    const float hi = __uint_as_float(sign | ((unsigned)ef << 23) | (unsigned)(m >> 29));
    const float lo = __fmul_rn(__uint2float_rn((unsigned)(m & 0x1FFFFFFFu)), __uint_as_float((unsigned)(ef - 52) << 23));
    out = {hi, sign ? -lo : lo};
    return true;
}

// ---------------------------------------------------------------- K9: FP64 refinement residual
//
// r = b64 - A p64, the refinement's residual, written as the FP32 inner
// right-hand side, with the inner iterate's role-0 buffer cleared.  Cells whose
// six neighbours lie inside the grid take them at fixed offsets; the others wrap
// periodic axes and drop wall faces.
//
// DF = false is the definition, all in FP64 (about 23 FP64 operations a cell,
// which bound the kernel: FP64 runs at 1/64 of the FP32 rate on this part).
// DF = true, the one the solver runs: the six differences p_nb - p_I in FP64
// (so their rounding is relative to the difference, not to |p|), then every
// difference and b64 split into hi + lo and the products, sums and b - A p in
// double-length FP32; eight FP64 operations a cell.  A cell whose values leave
// the split's range is evaluated by the FP64 expression.  r64, when set,
// receives r in full (the single-step op; the solver writes only the FP32 r).
// Each thread sums r^2 in FP64 over all its tiles; each block writes one
// partial, partials[blockIdx.x].
template <bool DF_PATH>
__global__ void __launch_bounds__(kThreads) k_ir_residual(const __grid_constant__ IrTask t)
{
    __shared__ double red[kThreads / 32];
    const Geo g = t.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int64_t nxy = (int64_t)nx * ny;
    const int tx = threadIdx.x % kResTX;
    const int ty = (threadIdx.x / kResTX) % kResTY;
    const int tz = threadIdx.x / (kResTX * kResTY);
    const int total = t.tiles_x * t.tiles_y * t.tiles_z;
    double rr = 0.0;
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int cx = tile % t.tiles_x;
        const int rest = tile / t.tiles_x;
        const int cy = rest % t.tiles_y;
        const int cz = rest / t.tiles_y;
        const int x = cx * kResTX + tx, y = cy * kResTY + ty, z = cz * kResTZ + tz;
        if (x < nx && y < ny && z < nz) {
            const int64_t I = ((int64_t)z * ny + y) * nx + x;
            const double p0 = t.p64[I];
            double pxl, pxu, pyl, pyu, pzl, pzu;
            float fxl, fxu, fyl, fyu, fzl, fzu;
            if (x > 0 && x < nx - 1 && y > 0 && y < ny - 1 && z > 0 && z < nz - 1) {
                pxl = t.p64[I - 1];
                pxu = t.p64[I + 1];
                pyl = t.p64[I - nx];
                pyu = t.p64[I + nx];
                pzl = t.p64[I - nxy];
                pzu = t.p64[I + nxy];
                fxl = __ldg(t.bx + I);
                fxu = __ldg(t.bx + I + 1);
                fyl = __ldg(t.by + I);
                fyu = __ldg(t.by + I + nx);
                fzl = __ldg(t.bz + I);
                fzu = __ldg(t.bz + I + nxy);
            } else {
                auto pv = [&](int xx, int yy, int zz) -> double {
                    if (!wrapc(xx, nx, g.per[0]) || !wrapc(yy, ny, g.per[1]) || !wrapc(zz, nz, g.per[2]))
                        return 0.0;
                    return t.p64[lin(g, xx, yy, zz)];
                };
                pxl = pv(x - 1, y, z);
                pxu = pv(x + 1, y, z);
                pyl = pv(x, y - 1, z);
                pyu = pv(x, y + 1, z);
                pzl = pv(x, y, z - 1);
                pzu = pv(x, y, z + 1);
                fxl = face_lo(t.bx, g, 0, x, y, z);
                fxu = face_lo(t.bx, g, 0, x + 1, y, z);
                fyl = face_lo(t.by, g, 1, x, y, z);
                fyu = face_lo(t.by, g, 1, x, y + 1, z);
                fzl = face_lo(t.bz, g, 2, x, y, z);
                fzu = face_lo(t.bz, g, 2, x, y, z + 1);
            }
            const double b = t.b64[I];
            double r = 0.0;
            float r32 = 0.f;
            bool done = false;
            if (DF_PATH) {
                DF d[6], bb;
                const bool ok = split64(pxl - p0, d[0]) & split64(pxu - p0, d[1]) & split64(pyl - p0, d[2]) &
                                split64(pyu - p0, d[3]) & split64(pzl - p0, d[4]) & split64(pzu - p0, d[5]) &
                                split64(b, bb);
                if (ok) {
                    const DF ax = df_add(df_mul(d[0], fxl), df_mul(d[1], fxu));
                    const DF ay = df_add(df_mul(d[2], fyl), df_mul(d[3], fyu));
                    const DF az = df_add(df_mul(d[4], fzl), df_mul(d[5], fzu));
                    const DF ap = df_add(df_add(ax, ay), az);
                    const DF rd = df_add(bb, {-ap.hi, -ap.lo});
                    r32 = rd.hi;
                    if (t.r64) r = (double)rd.hi + (double)rd.lo;
                    done = true;
                }
            }
            if (!done) {
                const double Ap = (((double)fxl * (pxl - p0) + (double)fxu * (pxu - p0)) +
                                   ((double)fyl * (pyl - p0) + (double)fyu * (pyu - p0))) +
                                  ((double)fzl * (pzl - p0) + (double)fzu * (pzu - p0));
                r = b - Ap;
                r32 = (float)r;
            }
            if (t.r64) t.r64[I] = r;
            if (t.b32) t.b32[I] = r32;
            if (t.ebuf[0]) t.ebuf[0][I] = 0.f;
            const double rs = (double)r32;
            rr = fma(rs, rs, rr);
        }
    }
    const double q = block_sum(rr, red);
    if (threadIdx.x == 0) t.partials[blockIdx.x] = q;
}

__global__ void k_ir_begin_inner(Ctl* ctl, const double* __restrict__ part, int n, double tol,
                                 double inner_rtol, int max_cycles)
{
    __shared__ double red[kThreads / 32];
    const double rr = sum_range(part, n, 1, 0, red);
    if (threadIdx.x == 0) {
        Ctl& C = *ctl;
        const double rn = sqrt(rr);
        const double prev = C.outer_r;
        C.outer_r = rn;
        if (C.total_cycles == 0 && C.hist_cap >= 0)
            C.hist_res[0] = C.outer_bnorm > 0.0 ? rn * (1.0 / C.outer_bnorm) : 0.0;   // as hist_scale
        if (!(rn == rn)) {
            C.outer_status = kDiverged;
            C.done = 1;
        } else if (rn / C.outer_bnorm <= tol) {
            C.outer_status = kOk;
            C.done = 1;
        } else if (C.total_cycles >= max_cycles) {
            C.outer_status = kNotConverged;
            C.done = 1;
        } else if (C.total_cycles > 0 && !(rn < prev)) {
            C.outer_status = kNotConverged;   // refinement stopped improving
            C.done = 1;
        } else {
            C.outer_status = kRunning;
            C.bnorm = rn;                     // inner right-hand side = outer residual
            C.r_prev = rn;
            C.tol = fmax(tol * C.outer_bnorm / rn, inner_rtol);
            C.cycles = 0;
            C.max_cycles = max_cycles - C.total_cycles;
            C.rot = 0;
            C.status = kRunning;
            C.done = 0;
            C.hist_scale = 1.0 / C.outer_bnorm;
        }
    }
}

__global__ void k_ir_update(Geo g, double* p64, const float* e0, const float* e1, const float* e2,
                            const int* rot)
{
    const int64_t N = (int64_t)g.n[0] * g.n[1] * g.n[2];
    const int r = *rot % 3;
    const float* e = r == 0 ? e0 : (r == 1 ? e1 : e2);
    for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < N;
         I += (int64_t)gridDim.x * blockDim.x)
        p64[I] += (double)e[I];
}

int grid_for(int64_t n, int per_block = kThreads)
{
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    const int64_t cap = (int64_t)sm_count() * 32;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

// ---------------------------------------------------------------- launchers

template <class TP, class TC>
cudaError_t launch_sweep(const TaskList<SweepTask<TP, TC>>& tl, int grid, cudaStream_t s)
{
    if (tl.total <= 0) return cudaSuccess;
    if constexpr (std::is_same<TP, float>::value) {
        constexpr size_t smem = kSweepSmemBytes;
        static bool attr = false;   // opt in to > 48 KB of dynamic shared memory once
        if (!attr) {
            const int b = (int)smem;
            cudaError_t e = cudaFuncSetAttribute(k_sweep_ws<false, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep_async<1, false, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep_ws<true, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep_async<1, true, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        if (tl.corr) {
            if (tl.vec >= 4) return launch_pdl(k_sweep_ws<true, TC>, grid, kSweepBlock, smem, s, 1, tl);
            return launch_pdl(k_sweep_async<1, true, TC>, grid, kThreads, smem, s, 1, tl);
        }
        if (tl.vec >= 4) return launch_pdl(k_sweep_ws<false, TC>, grid, kSweepBlock, smem, s, 1, tl);
        return launch_pdl(k_sweep_async<1, false, TC>, grid, kThreads, smem, s, 1, tl);
    }
    return launch_pdl(k_sweep<TP, TC>, grid, kThreads, 0, s, 1, tl);
}
template cudaError_t launch_sweep<float, float>(const TaskList<SweepTask<float, float>>&, int, cudaStream_t);
template cudaError_t launch_sweep<float, bf16>(const TaskList<SweepTask<float, bf16>>&, int, cudaStream_t);
template cudaError_t launch_sweep<bf16, bf16>(const TaskList<SweepTask<bf16, bf16>>&, int, cudaStream_t);

template <class TP>
cudaError_t launch_residual(const TaskList<ResTask<TP>>& tl, int grid, cudaStream_t s)
{
    if (tl.total <= 0) return cudaSuccess;
    if constexpr (std::is_same<TP, float>::value) {
        if (tl.march) {
            constexpr size_t smem = kResidualSmemBytes;
            static bool attr = false;
            if (!attr) {
                cudaError_t e = cudaFuncSetAttribute(k_residual_ws, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem);
                if (e != cudaSuccess) return e;
                attr = true;
            }
            return launch_pdl(k_residual_ws, grid, kResBlock, smem, s, 1, tl);
        }
    }
    return launch_pdl(k_residual<TP>, grid, kThreads, 0, s, 1, tl);
}
template cudaError_t launch_residual<float>(const TaskList<ResTask<float>>&, int, cudaStream_t);
template cudaError_t launch_residual<bf16>(const TaskList<ResTask<bf16>>&, int, cudaStream_t);

cudaError_t launch_project_level(const LevelProjTask* tasks, int ntasks, cudaStream_t s)
{
    if (ntasks <= 0) return cudaSuccess;
    k_project_level<<<ntasks, kThreads, 0, s>>>(tasks);
    return cudaGetLastError();
}

cudaError_t launch_sweep_two_pass(Geo g, const float* bx, const float* by, const float* bz,
                                  const float* b, float* p, float omega, cudaStream_t s)
{
    const int64_t N = (int64_t)g.n[0] * g.n[1] * g.n[2];
    for (int c = 0; c < 2; ++c) k_sweep_colour<<<grid_for(N), kThreads, 0, s>>>(g, bx, by, bz, b, p, omega, c);
    return cudaGetLastError();
}

cudaError_t launch_coarsen_coeffs(Geo fine, const int cf[3], const float* bx, const float* by,
                                  const float* bz, float* cbx, float* cby, float* cbz, int galerkin,
                                  cudaStream_t s)
{
    const int64_t N = (int64_t)(fine.n[0] / cf[0]) * (fine.n[1] / cf[1]) * (fine.n[2] / cf[2]);
    k_coarsen<<<grid_for(N), kThreads, 0, s>>>(fine, cf[0], cf[1], cf[2], bx, by, bz, cbx, cby, cbz, galerkin);
    return cudaGetLastError();
}

cudaError_t launch_prolong_add(Geo fine, const int cf[3], const float* e, float* p, cudaStream_t s)
{
    const int64_t N = (int64_t)fine.n[0] * fine.n[1] * fine.n[2];
    k_prolong_add<<<grid_for(N), kThreads, 0, s>>>(fine, cf[0], cf[1], cf[2], e, p);
    return cudaGetLastError();
}

cudaError_t launch_prolong_rows(const ProlongTask& t, cudaStream_t s)
{
    const int64_t chunks = (int64_t)(t.g.n[0] / 4) * t.g.n[1] * t.g.n[2];
    return launch_pdl(k_prolong_rows, grid_for(chunks), kThreads, 0, s, 1, t);
}

cudaError_t launch_active_mask(Geo g, const float* bx, const float* by, const float* bz,
                               uint8_t* mask, cudaStream_t s)
{
    const int64_t N = (int64_t)g.n[0] * g.n[1] * g.n[2];
    k_active_mask<<<grid_for(N), kThreads, 0, s>>>(g, bx, by, bz, mask);
    return cudaGetLastError();
}

cudaError_t launch_check_coeffs(int64_t n, const float* bx, const float* by, const float* bz, int* bad,
                                cudaStream_t s)
{
    k_check_coeffs<<<grid_for(n), kThreads, 0, s>>>(n, bx, by, bz, bad);
    return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* partials, int n, double* out, cudaStream_t s)
{
    k_sum_partials<<<1, kThreads, 0, s>>>(partials, n, out);
    return cudaGetLastError();
}

template <class TS>
cudaError_t launch_project_sum(const TaskList<ProjTask<TS>>& tl, int grid, cudaStream_t s)
{
    k_project_sum<TS><<<grid, kThreads, 0, s>>>(tl);
    return cudaGetLastError();
}
template <class TS>
cudaError_t launch_project_apply(const TaskList<ProjTask<TS>>& tl, int grid, cudaStream_t s)
{
    k_project_apply<TS><<<grid, kThreads, 0, s>>>(tl);
    return cudaGetLastError();
}
template cudaError_t launch_project_sum<float>(const TaskList<ProjTask<float>>&, int, cudaStream_t);
template cudaError_t launch_project_sum<double>(const TaskList<ProjTask<double>>&, int, cudaStream_t);
template cudaError_t launch_project_apply<float>(const TaskList<ProjTask<float>>&, int, cudaStream_t);
template cudaError_t launch_project_apply<double>(const TaskList<ProjTask<double>>&, int, cudaStream_t);

cudaError_t launch_project_finalize(const CtlTask* t, int nprob, cudaStream_t s)
{
    k_project_finalize<<<nprob, kThreads, 0, s>>>(t);
    return cudaGetLastError();
}
cudaError_t launch_control_init(const CtlTask* t, int nprob, cudaStream_t s)
{
    k_control_init<<<nprob, kThreads, 0, s>>>(t);
    return cudaGetLastError();
}
cudaError_t launch_control_cycle(const CtlTask* t, int nprob, cudaStream_t s)
{
    return launch_pdl(k_control_cycle, nprob, kThreads, 0, s, 1, t);
}

template <class TP, class TD>
cudaError_t launch_gauge_sum(const TaskList<GaugeTask<TP, TD>>& tl, int grid, cudaStream_t s)
{
    k_gauge_sum<TP, TD><<<grid, kThreads, 0, s>>>(tl);
    return cudaGetLastError();
}
template <class TP, class TD>
cudaError_t launch_gauge_apply(const TaskList<GaugeTask<TP, TD>>& tl, int grid, cudaStream_t s)
{
    k_gauge_apply<TP, TD><<<grid, kThreads, 0, s>>>(tl);
    return cudaGetLastError();
}
template cudaError_t launch_gauge_sum<float, float>(const TaskList<GaugeTask<float, float>>&, int, cudaStream_t);
template cudaError_t launch_gauge_sum<double, double>(const TaskList<GaugeTask<double, double>>&, int, cudaStream_t);
template cudaError_t launch_gauge_apply<float, float>(const TaskList<GaugeTask<float, float>>&, int, cudaStream_t);
template cudaError_t launch_gauge_apply<double, double>(const TaskList<GaugeTask<double, double>>&, int, cudaStream_t);

cudaError_t launch_gauge_finalize(const CtlTask* t, int nprob, cudaStream_t s)
{
    k_gauge_finalize<<<nprob, kThreads, 0, s>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_ir_residual(const IrTask& t, int grid, cudaStream_t s, bool fp64_definition)
{
    if (fp64_definition) k_ir_residual<false><<<grid, kThreads, 0, s>>>(t);
    else k_ir_residual<true><<<grid, kThreads, 0, s>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_ir_begin_inner(const IrTask& t, int nparts, double tol, double inner_rtol,
                                  int max_cycles, cudaStream_t s)
{
    k_ir_begin_inner<<<1, kThreads, 0, s>>>(t.ctl, t.partials, nparts, tol, inner_rtol, max_cycles);
    return cudaGetLastError();
}

cudaError_t launch_ir_update(const IrTask& t, cudaStream_t s)
{
    const int64_t N = (int64_t)t.g.n[0] * t.g.n[1] * t.g.n[2];
    k_ir_update<<<grid_for(N), kThreads, 0, s>>>(t.g, t.p64, t.ebuf[0], t.ebuf[1], t.ebuf[2], t.rot);
    return cudaGetLastError();
}

cudaError_t set_ring_wait_tries(int tries)
{
    const int v = tries < 0 ? kWaitTries : tries;
    return cudaMemcpyToSymbol(g_ring_tries, &v, sizeof(int));
}

int* wait_fault_flag()
{
    int* p = nullptr;
    return cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_wait_fault) == cudaSuccess ? p : nullptr;
}

}  // namespace gmg
