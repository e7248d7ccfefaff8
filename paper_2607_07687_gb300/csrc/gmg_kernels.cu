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
// order by one block per problem.
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

// ---------------------------------------------------------------- K1: pipelined sweep
//
// The same sweep as k_sweep (same arithmetic, bit-identical results) with the
// z-planes staged by asynchronous global->shared copies.  Ring buffers of
// planes over the tile plus halo (x: 4 columns each side so rows split into
// 16-byte chunks; y: 2 rows each side):
//   P  input p (+ coarse correction)     planes kr .. kr+3   (4 slots)
//   B, X, Y  b and lower x/y faces       planes kr-1 .. kr+1 (4 slots)
//   Z  lower z faces                     planes kr-1 .. kr+2 (5 slots)
//   M  merged plane (red new, black old) planes kr-2 .. kr   (3 slots)
// At step u (red plane kr = z0 - 1 + u, black plane kr - 1) the copies for
// step u+1 are issued first, then the step waits for its own group.  The
// coarse correction of a P plane is added two steps before the plane is read,
// so it needs no extra barrier.  VEC = 4 copies 16-byte chunks (rows of a
// multiple of 4 cells, 16-byte aligned arrays), VEC = 1 copies single floats.

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

template <int VEC, bool CORR, class TC>
__global__ void __launch_bounds__(kThreads, 3) k_sweep_async(const __grid_constant__ TaskList<SweepTask<float, TC>> tl)
{
    constexpr int TX = kSweepTX, TY = kSweepTY;
    constexpr int XO = 4, SW = TX + 8, SH = TY + 4, PL = SW * SH;   // 40 x 12 positions per plane
    constexpr int R = kSweepRing;               // planes per ring, every array
    constexpr int CPR = SW / 4;                 // 16-byte chunks per row
    constexpr int NCH = PL / 4;                 // chunks per plane (120)
    constexpr int RPR = (TX + 2) / 2;           // red cells per ring row
    constexpr int NRED = RPR * (TY + 2);
    constexpr int BPR = TX / 2;                 // black cells per tile row
    constexpr int NBLK = BPR * TY;
    static_assert(NCH <= kThreads / 2 && NRED <= kThreads && PL <= 2 * kThreads, "thread budget");
    // rings: 0 = p, 1 = b, 2 = lower x faces, 3 = lower y faces, 4 = lower z faces, 5 = merged red plane
    extern __shared__ __align__(16) float smem[];
    const int tid = threadIdx.x;
    const int half = tid / (kThreads / 2);      // copy duty: 0 -> p, b, x faces; 1 -> y, z faces
    const int chunk = tid % (kThreads / 2);

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

        // ---- prologue: p planes kr0-1 .. kr0+1 and z faces of kr0, then step 0's group;
        // plane z lives in slot (z - kr0 + 1) mod R
        const int kr0 = z0 - 1;
        copy_plane(ring(0, 0), pin, kr0 - 1, false);
        copy_plane(ring(0, 1), pin, kr0, false);
        copy_plane(ring(0, 2), pin, kr0 + 1, false);
        copy_plane(ring(4, 1), tp->bz, kr0, true);
        cp_commit();
        float ca0, ca1, cb0, cb1, cc0, cc1, cur0, cur1, nxt0, nxt1;
        corr_load(kr0 - 1, ca0, ca1);
        corr_load(kr0, cb0, cb1);
        corr_load(kr0 + 1, cc0, cc1);
        copy_plane(ring(0, 3), pin, kr0 + 2, false);
        copy_plane(ring(1, 1), ba, kr0, false);
        copy_plane(ring(2, 1), tp->bx, kr0, false);
        copy_plane(ring(3, 1), tp->by, kr0, false);
        copy_plane(ring(4, 2), tp->bz, kr0 + 1, true);
        cp_commit();
        corr_load(kr0 + 2, cur0, cur1);
        cp_wait<1>();
        __syncthreads();
        corr_add(ring(0, 0), ca0, ca1);
        corr_add(ring(0, 1), cb0, cb1);
        corr_add(ring(0, 2), cc0, cc1);

        const int nsteps = (z1 - z0) + 2;   // red planes z0-1 .. z1

        // one z-step; J = (u mod R) is a compile-time constant, so is every slot
        auto step = [&](int u, auto Jc) {
            constexpr int J = decltype(Jc)::value;
            constexpr int S0 = (J + 1) % R;                       // slot of plane kr
            constexpr int Sm1 = (J + R) % R, Sm2 = (J + R - 1) % R;
            constexpr int Sp1 = (J + 2) % R, Sp2 = (J + 3) % R, Sp3 = (J + 4) % R;
            const int kr = kr0 + u;
            // copies for step u+1: p(kr+3), b / x / y faces (kr+1), z faces (kr+2)
            if (u + 1 < nsteps) {
                if (VEC == 4) {
                    if (chunk < NCH) {
                        int64_t zo1, zo2;
                        if (half == 0) {
                            int64_t zo3;
                            const bool ok3 = pin != nullptr && zinfo(kr + 3, false, zo3) && cok;
                            const bool ok1 = zinfo(kr + 1, false, zo1) && cok;
                            cp_async16(ring(0, Sp3) + 4 * chunk, ok3 ? srcA + zo3 + coff : ba, ok3);
                            cp_async16(ring(1, Sp1) + 4 * chunk, ok1 ? srcB + zo1 + coff : ba, ok1);
                            cp_async16(ring(2, Sp1) + 4 * chunk, ok1 ? srcC + zo1 + coff : ba, ok1);
                        } else {
                            const bool ok1 = zinfo(kr + 1, false, zo1) && cok;
                            const bool ok2 = zinfo(kr + 2, true, zo2) && cok;
                            cp_async16(ring(3, Sp1) + 4 * chunk, ok1 ? srcA + zo1 + coff : ba, ok1);
                            cp_async16(ring(4, Sp2) + 4 * chunk, ok2 ? srcB + zo2 + coff : ba, ok2);
                        }
                    }
                } else {
                    copy_plane(ring(0, Sp3), pin, kr + 3, false);
                    copy_plane(ring(1, Sp1), ba, kr + 1, false);
                    copy_plane(ring(2, Sp1), tp->bx, kr + 1, false);
                    copy_plane(ring(3, Sp1), tp->by, kr + 1, false);
                    copy_plane(ring(4, Sp2), tp->bz, kr + 2, true);
                }
                corr_load(kr + 3, nxt0, nxt1);
            }
            cp_commit();
            cp_wait<1>();
            __syncthreads();                               // S1: this step's planes are visible
            corr_add(ring(0, Sp2), cur0, cur1);            // p(kr+2), first read at step u+1
            cur0 = nxt0;
            cur1 = nxt1;

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
                    const float fl = face_flux(xl, P0[s - 1], X0[s + 1], P0[s + 1], yl, P0[s - SW], Y0[s + SW],
                                               P0[s + SW], Z0[s], ring(0, Sm1)[s], Z1[s], ring(0, Sp1)[s], v);
                    const float dg = diag_sum(xl, X0[s + 1], yl, Y0[s + SW], Z0[s], Z1[s]);
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
                const float fl = face_flux(xl, Mk[s - 1], Xk[s + 1], Mk[s + 1], yl, Mk[s - SW], Yk[s + SW],
                                           Mk[s + SW], Zk[s], ring(5, Sm2)[s], Zk1[s], ring(5, S0)[s], v);
                const float dg = diag_sum(xl, Xk[s + 1], yl, Yk[s + SW], Zk[s], Zk1[s]);
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
// r = b - A p on a TX x TY column marching through a z-chunk, with the planes
// of p, b and the faces staged by the same asynchronous copies as the sweep.
// Each of the first TX*TY/2 threads owns a pair of cells of a row; the
// restriction to the next level sums x-pairs in the thread, y-pairs with the
// lane 16 apart (rows 2w and 2w+1 share a warp) and z-pairs across two steps,
// so coarse cells are written without atomics.  Sum r^2 per tile in FP64.
template <int VEC>
__global__ void __launch_bounds__(kThreads, 3) k_residual_async(const __grid_constant__ TaskList<ResTask<float>> tl)
{
    constexpr int TX = kSweepTX, TY = kSweepTY;
    constexpr int XO = 4, SW = TX + 8, SH = TY + 4, PL = SW * SH;
    constexpr int R = kSweepRing;
    constexpr int CPR = SW / 4, NCH = PL / 4;
    constexpr int BPR = TX / 2, NPAIR = BPR * TY;
    static_assert(VEC == 4, "16-byte plane copies only");
    static_assert(NPAIR <= kThreads && BPR == 16, "pair layout: two rows per warp");
    extern __shared__ __align__(16) float smem[];
    __shared__ double red[kThreads / 32];
    const int tid = threadIdx.x;
    const int half = tid / (kThreads / 2);
    const int chunk = tid % (kThreads / 2);

    for (int tile = blockIdx.x; tile < tl.total; tile += gridDim.x) {
        int local;
        const ResTask<float>* tp = task_of(tl, tile, local);
        if (tp->ctl && tp->ctl->done) continue;               // uniform in the block
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
        const float* pin = tp->role < 0 ? nullptr : tp->buf[(tp->role + rot) % 3];
        const float* const ba = tp->b;
        const float* const srcA = half == 0 ? pin : tp->by;
        const float* const srcB = half == 0 ? tp->b : tp->bz;
        const float* const srcC = tp->bx;
        float* const bc = tp->bc;
        const int c0 = tp->cf[0], c1 = tp->cf[1], c2 = tp->cf[2];
        const int64_t plane = (int64_t)nx * ny;

        int coff = 0;
        bool cok = false;
        if (chunk < NCH) {
            const int sy = chunk / CPR, ch = chunk - sy * CPR;
            int x = x0 - XO + 4 * ch, y = y0 - 2 + sy;
            cok = wrapc(x, nx, px) && wrapc(y, ny, py);
            coff = cok ? y * nx + x : 0;
        }
        const int tyb = tid / BPR, jb = tid - tyb * BPR;
        const int yb = y0 + tyb, xb = x0 + 2 * jb;
        const bool pair_on = tid < NPAIR && yb < ny && xb < nx;
        const int sp = (tyb + 2) * SW + XO + 2 * jb;
        const bool yb_wall = yb == 0 && !py;
        const bool xb_wall = xb == 0 && !px;
        const int gcx = nx / c0, gcy = ny / c1;
        // coarse cell(s) this thread writes: one x-pair sum (c0 = 2) or two cells
        const bool writer = pair_on && (c1 == 1 || (tyb & 1) == 0);
        const int64_t cplane = (int64_t)gcx * gcy;
        const int64_t crow = (int64_t)(yb / c1) * gcx + xb / c0;

        auto zinfo = [&](int z, bool zface, int64_t& zoff) -> bool {
            int zw = z;
            bool ok = wrapc(zw, nz, pz);
            if (zface && ok && zw == 0 && !pz) ok = false;
            zoff = (int64_t)zw * plane;
            return ok;
        };
        auto copy_plane = [&](float* dst, const float* a, int z, bool zface) {
            int64_t zoff;
            const bool zok = a != nullptr && zinfo(z, zface, zoff);
            for (int c = tid; c < NCH; c += kThreads) {
                const int sy = c / CPR, ch = c - sy * CPR;
                int x = x0 - XO + 4 * ch, y = y0 - 2 + sy;
                const bool ok = zok && wrapc(x, nx, px) && wrapc(y, ny, py);
                cp_async16(dst + 4 * c, ok ? a + zoff + (int64_t)y * nx + x : ba, ok);
            }
        };
        auto ring = [&](int r, int slot) -> float* { return smem + (r * R + slot) * PL; };

        // plane z in slot (z - z0 + 1) mod R
        copy_plane(ring(0, 0), pin, z0 - 1, false);
        copy_plane(ring(0, 1), pin, z0, false);
        copy_plane(ring(0, 2), pin, z0 + 1, false);
        copy_plane(ring(4, 1), tp->bz, z0, true);
        copy_plane(ring(1, 1), ba, z0, false);
        copy_plane(ring(2, 1), tp->bx, z0, false);
        copy_plane(ring(3, 1), tp->by, z0, false);
        copy_plane(ring(4, 2), tp->bz, z0 + 1, true);
        cp_commit();

        const int nsteps = z1 - z0;
        double rr = 0.0;
        float acc0 = 0.f, acc1 = 0.f;
        auto step = [&](int u, auto Jc) {
            constexpr int J = decltype(Jc)::value;
            constexpr int S0 = (J + 1) % R, Sm1 = J % R, Sp1 = (J + 2) % R, Sp2 = (J + 3) % R;
            const int k = z0 + u;
            // copies for step u+1: p(k+2), b / x / y faces (k+1), z faces (k+2)
            if (u + 1 < nsteps && chunk < NCH) {
                int64_t zo1, zo2;
                if (half == 0) {
                    const bool ok2 = pin != nullptr && zinfo(k + 2, false, zo2) && cok;
                    const bool ok1 = zinfo(k + 1, false, zo1) && cok;
                    cp_async16(ring(0, Sp2) + 4 * chunk, ok2 ? srcA + zo2 + coff : ba, ok2);
                    cp_async16(ring(1, Sp1) + 4 * chunk, ok1 ? srcB + zo1 + coff : ba, ok1);
                    cp_async16(ring(2, Sp1) + 4 * chunk, ok1 ? srcC + zo1 + coff : ba, ok1);
                } else {
                    const bool ok1 = zinfo(k + 1, false, zo1) && cok;
                    const bool ok2 = zinfo(k + 2, true, zo2) && cok;
                    cp_async16(ring(3, Sp1) + 4 * chunk, ok1 ? srcA + zo1 + coff : ba, ok1);
                    cp_async16(ring(4, Sp2) + 4 * chunk, ok2 ? srcB + zo2 + coff : ba, ok2);
                }
            }
            cp_commit();
            cp_wait<1>();
            __syncthreads();
            float r0 = 0.f, r1 = 0.f;
            if (pair_on) {
                const float* P0 = ring(0, S0);
                const float* Pl = ring(0, Sm1);
                const float* Pu = ring(0, Sp1);
                const float* X0 = ring(2, S0);
                const float* Y0 = ring(3, S0);
                const float* Z0 = ring(4, S0);
                const float* Z1 = ring(4, Sp1);
                const float* B0 = ring(1, S0);
                for (int h = 0; h < 2; ++h) {
                    const int s = sp + h;
                    const float p0 = P0[s];
                    const float xl = (h == 0 && xb_wall) ? 0.f : X0[s];
                    const float yl = yb_wall ? 0.f : Y0[s];
                    const float fl = face_flux(xl, P0[s - 1], X0[s + 1], P0[s + 1], yl, P0[s - SW], Y0[s + SW],
                                               P0[s + SW], Z0[s], Pl[s], Z1[s], Pu[s], p0);
                    const float r = B0[s] - fl;
                    if (h == 0) r0 = r; else r1 = (xb + 1 < nx) ? r : 0.f;
                }
                rr += (double)r0 * (double)r0 + (double)r1 * (double)r1;
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
        if (tp->partials) {
            const double q = block_sum(rr, red);
            if (tid == 0) tp->partials[local] = q;
        } else {
            __syncthreads();
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
            const double q = block_sum((double)r * (double)r, red);
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

__global__ void k_coarsen(Geo f, int c0, int c1, int c2, const float* __restrict__ bx,
                          const float* __restrict__ by, const float* __restrict__ bz, float* cbx,
                          float* cby, float* cbz)
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
            ca[d][J] = s / (float)cfac[d];
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
        double s = 0.0, c = 0.0, bad = 0.0;
        for (int64_t i = beg + threadIdx.x; i < end; i += kThreads) {
            const double v = (double)t->sigma[i];
            if (!isfinite(v)) bad += 1.0;
            if (t->mask[i]) {
                s += v;
                c += 1.0;
            }
        }
        s = block_sum(s, red);
        c = block_sum(c, red);
        bad = block_sum(bad, red);
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
        double q = 0.0;
        for (int64_t i = beg + threadIdx.x; i < end; i += kThreads) {
            const bool act = t->mask[i] != 0;
            const double bv = act ? (double)t->sigma[i] - mean : 0.0;
            if (t->b32) {
                const float f = (float)bv;
                t->b32[i] = f;
                q += (double)f * (double)f;
            } else {
                t->b64[i] = bv;
                q += bv * bv;
            }
            const double pv = (act && t->p_in) ? (double)t->p_in[i] : 0.0;
            if (t->p32) t->p32[i] = (float)pv;
            if (t->p64) t->p64[i] = pv;
        }
        q = block_sum(q, red);
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
            C.hist_res[0] = C.r_prev / C.bnorm;
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

// the adaptive relaxation rule after one V-cycle (Sec. 3.1)
__global__ void k_control_cycle(const CtlTask* __restrict__ tasks)
{
    __shared__ double red[kThreads / 32];
    const CtlTask& t = tasks[blockIdx.x];
    if (t.ctl->done) return;   // uniform in the block
    const double rr = sum_range(t.partials, t.nparts, 1, 0, red);
    if (threadIdx.x == 0) {
        Ctl& C = *t.ctl;
        const double rk = sqrt(rr);
        const double w = C.omega;
        const bool acc = rk < C.r_prev;     // NaN rejects
        C.r_last = rk;
        C.cycles += 1;
        C.total_cycles += 1;
        if (acc) {
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
}

// ---------------------------------------------------------------- K9: FP64 refinement

__global__ void __launch_bounds__(kThreads) k_ir_residual(const __grid_constant__ IrTask t)
{
    __shared__ double red[kThreads / 32];
    const Geo g = t.g;
    const int tx = threadIdx.x % kResTX;
    const int ty = (threadIdx.x / kResTX) % kResTY;
    const int tz = threadIdx.x / (kResTX * kResTY);
    const int total = t.tiles_x * t.tiles_y * t.tiles_z;
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int cx = tile % t.tiles_x;
        const int rest = tile / t.tiles_x;
        const int cy = rest % t.tiles_y;
        const int cz = rest / t.tiles_y;
        const int x = cx * kResTX + tx, y = cy * kResTY + ty, z = cz * kResTZ + tz;
        double r = 0.0;
        if (x < g.n[0] && y < g.n[1] && z < g.n[2]) {
            auto pv = [&](int xx, int yy, int zz) -> double {
                if (!wrapc(xx, g.n[0], g.per[0]) || !wrapc(yy, g.n[1], g.per[1]) ||
                    !wrapc(zz, g.n[2], g.per[2]))
                    return 0.0;
                return t.p64[lin(g, xx, yy, zz)];
            };
            const double fxl = face_lo(t.bx, g, 0, x, y, z), fxu = face_lo(t.bx, g, 0, x + 1, y, z);
            const double fyl = face_lo(t.by, g, 1, x, y, z), fyu = face_lo(t.by, g, 1, x, y + 1, z);
            const double fzl = face_lo(t.bz, g, 2, x, y, z), fzu = face_lo(t.bz, g, 2, x, y, z + 1);
            const double p0 = pv(x, y, z);
            const double Ap = ((fxl * (pv(x - 1, y, z) - p0) + fxu * (pv(x + 1, y, z) - p0)) +
                               (fyl * (pv(x, y - 1, z) - p0) + fyu * (pv(x, y + 1, z) - p0))) +
                              (fzl * (pv(x, y, z - 1) - p0) + fzu * (pv(x, y, z + 1) - p0));
            const int64_t I = lin(g, x, y, z);
            r = t.b64[I] - Ap;
            t.b32[I] = (float)r;
            t.ebuf[0][I] = 0.f;
        }
        const double q = block_sum(r * r, red);
        if (threadIdx.x == 0) t.partials[tile] = q;
    }
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
            C.hist_res[0] = C.outer_bnorm > 0.0 ? rn / C.outer_bnorm : 0.0;
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
    if (b > 152 * 32) b = 152 * 32;
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
            cudaError_t e = cudaFuncSetAttribute(k_sweep_async<4, false, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep_async<1, false, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep_async<4, true, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep_async<1, true, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        if (tl.corr) {
            if (tl.vec >= 4) k_sweep_async<4, true, TC><<<grid, kThreads, smem, s>>>(tl);
            else k_sweep_async<1, true, TC><<<grid, kThreads, smem, s>>>(tl);
        } else {
            if (tl.vec >= 4) k_sweep_async<4, false, TC><<<grid, kThreads, smem, s>>>(tl);
            else k_sweep_async<1, false, TC><<<grid, kThreads, smem, s>>>(tl);
        }
    } else {
        k_sweep<TP, TC><<<grid, kThreads, 0, s>>>(tl);
    }
    return cudaGetLastError();
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
                cudaError_t e = cudaFuncSetAttribute(k_residual_async<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem);
                if (e != cudaSuccess) return e;
                attr = true;
            }
            k_residual_async<4><<<grid, kThreads, smem, s>>>(tl);
            return cudaGetLastError();
        }
    }
    k_residual<TP><<<grid, kThreads, 0, s>>>(tl);
    return cudaGetLastError();
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
                                  const float* bz, float* cbx, float* cby, float* cbz, cudaStream_t s)
{
    const int64_t N = (int64_t)(fine.n[0] / cf[0]) * (fine.n[1] / cf[1]) * (fine.n[2] / cf[2]);
    k_coarsen<<<grid_for(N), kThreads, 0, s>>>(fine, cf[0], cf[1], cf[2], bx, by, bz, cbx, cby, cbz);
    return cudaGetLastError();
}

cudaError_t launch_prolong_add(Geo fine, const int cf[3], const float* e, float* p, cudaStream_t s)
{
    const int64_t N = (int64_t)fine.n[0] * fine.n[1] * fine.n[2];
    k_prolong_add<<<grid_for(N), kThreads, 0, s>>>(fine, cf[0], cf[1], cf[2], e, p);
    return cudaGetLastError();
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
    k_control_cycle<<<nprob, kThreads, 0, s>>>(t);
    return cudaGetLastError();
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

cudaError_t launch_ir_residual(const IrTask& t, int grid, cudaStream_t s)
{
    k_ir_residual<<<grid, kThreads, 0, s>>>(t);
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

}  // namespace gmg
