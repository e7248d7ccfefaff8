// gmg_pcg.cu -- the Jacobi-preconditioned conjugate-gradient Poisson solve, the
// general-purpose solver the paper compares its multigrid against (Sec. 3: PCG
// applies to any grid but needs global inner products every iteration, and its
// iteration count grows with the problem size; Table 1).  The paper does not
// name the preconditioner; this is the diagonal (Jacobi) one.
//
// CG runs on the symmetric positive (semi-)definite form B = -A of the operator
// (A p = sum_f beta_f (p_nb - p)), with rho = A x - b = -(b - A x):
//   start   rho = A x - b, z = D^-1 rho, d = 0, beta = 0      (D = diag(B) = sum_f beta_f)
//   step    d <- z + beta d;  q = A d;  alpha = (rho.z) / -(d.q)
//           x += alpha d;  rho += alpha q;  z = D^-1 rho
//           beta = (rho.z)_new / (rho.z)_old
// Cells with D = 0 (no open face) keep D^-1 = 0, so they never move.  One
// iteration is two grid launches (k_pcg_dir_apply: the new direction and its
// image; k_pcg_update: iterate, residual, preconditioned residual) and two
// one-block control launches that turn the FP64 tile partials of the inner
// products into alpha, beta and the stopping decision on the device, so a
// CUDA graph of several iterations runs without the host.  Grids: 32 x 8
// threads per (x, y) tile, each thread marching a z-chunk; one FP64 partial
// per block and product (FP32 products summed in the thread and the warp).
#include "gmg_internal.h"
#include "gmg_device.cuh"

namespace gmg {
namespace {

using namespace dev;

constexpr int kPX = 32, kPY = 8;

// FP32 sum over the warp, FP64 over the block's warps; result in thread 0
__device__ __forceinline__ double block_sum_f(float v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int tid = threadIdx.y * kPX + threadIdx.x;
    if ((tid & 31) == 0) red[tid >> 5] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int i = 0; i < kPX * kPY / 32; ++i) s += red[i];
    __syncthreads();
    return s;
}

__device__ __forceinline__ int block_index() { return (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x; }

// value of v at (x, y, z), or 0 outside a wall (its face coefficient is 0 there)
__device__ __forceinline__ float at(const float* v, const Geo& g, int x, int y, int z)
{
    if (!wrapc(x, g.n[0], g.per[0]) || !wrapc(y, g.n[1], g.per[1]) || !wrapc(z, g.n[2], g.per[2])) return 0.f;
    return v[lin(g, x, y, z)];
}

__device__ __forceinline__ float apply_at(const PcgTask& t, const float* v, int x, int y, int z, float& dg)
{
    const Geo& g = t.g;
    const float fxl = face_lo(t.bx, g, 0, x, y, z), fxu = face_lo(t.bx, g, 0, x + 1, y, z);
    const float fyl = face_lo(t.by, g, 1, x, y, z), fyu = face_lo(t.by, g, 1, x, y + 1, z);
    const float fzl = face_lo(t.bz, g, 2, x, y, z), fzu = face_lo(t.bz, g, 2, x, y, z + 1);
    dg = diag_sum(fxl, fxu, fyl, fyu, fzl, fzu);
    const float c = v[lin(g, x, y, z)];
    return face_flux(fxl, at(v, g, x - 1, y, z), fxu, at(v, g, x + 1, y, z), fyl, at(v, g, x, y - 1, z), fyu,
                     at(v, g, x, y + 1, z), fzl, at(v, g, x, y, z - 1), fzu, at(v, g, x, y, z + 1), c);
}

// rho = A x - b, D^-1, z = D^-1 rho, d = 0 (into d_dst); partials (rho.z, rho.rho, b.b)
__global__ void __launch_bounds__(kPX * kPY) k_pcg_start(const __grid_constant__ PcgTask t)
{
    __shared__ double red[kPX * kPY / 32];
    if (t.ctl->done) return;
    const Geo g = t.g;
    const int x = blockIdx.x * kPX + threadIdx.x, y = blockIdx.y * kPY + threadIdx.y;
    const int z0 = blockIdx.z * t.zc, z1 = min(g.n[2], z0 + t.zc);
    float rz = 0.f, rr = 0.f, bb = 0.f;
    if (x < g.n[0] && y < g.n[1])
        for (int z = z0; z < z1; ++z) {
            const int64_t I = lin(g, x, y, z);
            float dg;
            const float rho = apply_at(t, t.x, x, y, z, dg) - t.b[I];
            const float inv = dg > 0.f ? 1.f / dg : 0.f;
            const float zz = inv * rho;
            t.inv_diag[I] = inv;
            t.r[I] = rho;
            t.z[I] = zz;
            t.d_dst[I] = 0.f;                   // read as the first iteration's d_src
            rz = fmaf(rho, zz, rz);
            rr = fmaf(rho, rho, rr);
            bb = fmaf(t.b[I], t.b[I], bb);
        }
    const int blk = block_index();
    const double s0 = block_sum_f(rz, red), s1 = block_sum_f(rr, red), s2 = block_sum_f(bb, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        t.part[3 * blk + 0] = s0;
        t.part[3 * blk + 1] = s1;
        t.part[3 * blk + 2] = s2;
    }
}

// d_dst = z + beta d_src (at the cell and, on the fly, at its neighbours), q = A d_dst;
// partial d.q
__global__ void __launch_bounds__(kPX * kPY) k_pcg_dir_apply(const __grid_constant__ PcgTask t)
{
    __shared__ double red[kPX * kPY / 32];
    if (t.ctl->done) return;
    const Geo g = t.g;
    const float beta = (float)t.scal->beta;
    const int x = blockIdx.x * kPX + threadIdx.x, y = blockIdx.y * kPY + threadIdx.y;
    const int z0 = blockIdx.z * t.zc, z1 = min(g.n[2], z0 + t.zc);
    auto dn = [&](int xx, int yy, int zz) -> float {
        if (!wrapc(xx, g.n[0], g.per[0]) || !wrapc(yy, g.n[1], g.per[1]) || !wrapc(zz, g.n[2], g.per[2]))
            return 0.f;
        const int64_t J = lin(g, xx, yy, zz);
        return fmaf(beta, t.d_src[J], t.z[J]);
    };
    float dq = 0.f;
    if (x < g.n[0] && y < g.n[1])
        for (int z = z0; z < z1; ++z) {
            const int64_t I = lin(g, x, y, z);
            const float fxl = face_lo(t.bx, g, 0, x, y, z), fxu = face_lo(t.bx, g, 0, x + 1, y, z);
            const float fyl = face_lo(t.by, g, 1, x, y, z), fyu = face_lo(t.by, g, 1, x, y + 1, z);
            const float fzl = face_lo(t.bz, g, 2, x, y, z), fzu = face_lo(t.bz, g, 2, x, y, z + 1);
            const float dI = dn(x, y, z);
            const float q = face_flux(fxl, dn(x - 1, y, z), fxu, dn(x + 1, y, z), fyl, dn(x, y - 1, z), fyu,
                                      dn(x, y + 1, z), fzl, dn(x, y, z - 1), fzu, dn(x, y, z + 1), dI);
            t.d_dst[I] = dI;
            t.q[I] = q;
            dq = fmaf(dI, q, dq);
        }
    const double s = block_sum_f(dq, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) t.part[3 * block_index()] = s;
}

// x += alpha d, rho += alpha q, z = D^-1 rho; partials (rho.z, rho.rho)
__global__ void __launch_bounds__(kPX * kPY) k_pcg_update(const __grid_constant__ PcgTask t)
{
    __shared__ double red[kPX * kPY / 32];
    if (t.ctl->done) return;
    const Geo g = t.g;
    const float alpha = (float)t.scal->alpha;
    const int x = blockIdx.x * kPX + threadIdx.x, y = blockIdx.y * kPY + threadIdx.y;
    const int z0 = blockIdx.z * t.zc, z1 = min(g.n[2], z0 + t.zc);
    float rz = 0.f, rr = 0.f;
    if (x < g.n[0] && y < g.n[1])
        for (int z = z0; z < z1; ++z) {
            const int64_t I = lin(g, x, y, z);
            t.x[I] = fmaf(alpha, t.d_dst[I], t.x[I]);
            const float rho = fmaf(alpha, t.q[I], t.r[I]);
            const float zz = t.inv_diag[I] * rho;
            t.r[I] = rho;
            t.z[I] = zz;
            rz = fmaf(rho, zz, rz);
            rr = fmaf(rho, rho, rr);
        }
    const int blk = block_index();
    const double s0 = block_sum_f(rz, red), s1 = block_sum_f(rr, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        t.part[3 * blk + 0] = s0;
        t.part[3 * blk + 1] = s1;
    }
}

__device__ double sum_part(const double* part, int n, int off, double* red)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[3 * i + off];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    __syncthreads();
    return t;
}

// phase 0: after k_pcg_start (3: the same after a restart, iterations kept);
// 1: alpha after k_pcg_dir_apply; 2: beta and the stop test after k_pcg_update.
// The recursively updated residual drifts from b - A x in FP32, so when it
// meets the tolerance the solve only pauses (done with status running): the
// host then restarts from the current iterate, and phase 3 decides on the
// true residual.
__global__ void k_pcg_control(const __grid_constant__ PcgTask t, int phase)
{
    __shared__ double red[kThreads / 32];
    Ctl& C = *t.ctl;
    if (C.done) return;
    const double a = sum_part(t.part, t.nparts, 0, red);
    const double b = phase == 1 ? 0.0 : sum_part(t.part, t.nparts, 1, red);
    const double c = (phase == 0 || phase == 3) ? sum_part(t.part, t.nparts, 2, red) : 0.0;
    if (threadIdx.x != 0) return;
    PcgScal& S = *t.scal;
    if (phase == 0 || phase == 3) {
        C.bnorm = S.smoother ? sqrt(b) : sqrt(c);   // a smoothing run measures against its start
        C.r_prev = sqrt(b);
        if (phase == 0) C.cycles = 0;
        S.rz = a;
        S.beta = 0.0;
        if (C.nonfinite) {
            C.status = kNonFinite;
            C.done = 1;
        } else if (C.bnorm == 0.0) {
            C.status = kOk;
            C.zero_out = 1;
            C.done = 1;
        } else if (C.r_prev / C.bnorm <= C.tol) {
            C.status = kOk;
            C.done = 1;
        } else {
            C.status = kRunning;
        }
    } else if (phase == 1) {
        // a = d.q = -(d.B d) < 0 for d != 0; otherwise CG has broken down
        if (!(a < 0.0)) {
            C.status = kDiverged;
            C.done = 1;
        } else {
            S.alpha = S.rz / -a;
        }
    } else {
        C.cycles += 1;
        C.r_prev = sqrt(b);
        if (!(C.r_prev == C.r_prev)) {
            C.status = kDiverged;
            C.done = 1;
        } else if (C.r_prev / C.bnorm <= C.tol) {
            C.done = 1;                   // pause: the true residual decides (phase 3)
        } else if (C.cycles >= C.max_cycles) {
            C.status = kNotConverged;
            C.done = 1;
        } else {
            S.beta = a / S.rz;
            S.rz = a;
        }
    }
}

__global__ void k_pcg_arm(Ctl* ctl, PcgScal* scal, int max_it, double tol, int smoother)
{
    Ctl& C = *ctl;
    C.done = 0;
    C.status = kRunning;
    C.cycles = 0;
    C.max_cycles = max_it;
    C.tol = tol;
    C.nonfinite = 0;
    C.zero_out = 0;
    scal->smoother = smoother;
}

dim3 pcg_grid(const PcgTask& t)
{
    return dim3((unsigned)((t.g.n[0] + kPX - 1) / kPX), (unsigned)((t.g.n[1] + kPY - 1) / kPY),
                (unsigned)((t.g.n[2] + t.zc - 1) / t.zc));
}

}  // namespace

int pcg_blocks(const Geo& g, int zc)
{
    return ((g.n[0] + kPX - 1) / kPX) * ((g.n[1] + kPY - 1) / kPY) * ((g.n[2] + zc - 1) / zc);
}

cudaError_t launch_pcg_start(const PcgTask& t, bool restart, cudaStream_t s)
{
    k_pcg_start<<<pcg_grid(t), dim3(kPX, kPY), 0, s>>>(t);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) k_pcg_control<<<1, kThreads, 0, s>>>(t, restart ? 3 : 0);
    return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t launch_pcg_iteration(const PcgTask& t, cudaStream_t s)
{
    k_pcg_dir_apply<<<pcg_grid(t), dim3(kPX, kPY), 0, s>>>(t);
    k_pcg_control<<<1, kThreads, 0, s>>>(t, 1);
    k_pcg_update<<<pcg_grid(t), dim3(kPX, kPY), 0, s>>>(t);
    k_pcg_control<<<1, kThreads, 0, s>>>(t, 2);
    return cudaGetLastError();
}

cudaError_t launch_pcg_arm(Ctl* ctl, PcgScal* scal, int max_it, double tol, int smoother, cudaStream_t s)
{
    k_pcg_arm<<<1, 1, 0, s>>>(ctl, scal, max_it, tol, smoother);
    return cudaGetLastError();
}

}  // namespace gmg
