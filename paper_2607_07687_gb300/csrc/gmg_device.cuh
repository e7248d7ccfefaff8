// gmg_device.cuh -- device helpers shared by the solver's kernel files.
#pragma once

#include "gmg_internal.h"

namespace gmg {
namespace dev {

// Map a (possibly out-of-range) index onto the grid: periodic axes wrap by
// any number of periods (tiles and halos can exceed a small periodic level),
// walled axes report "outside".
__device__ __forceinline__ bool wrapc(int& i, int n, int per)
{
    if (i >= 0 && i < n) return true;
    if (!per) return false;
    i %= n;
    if (i < 0) i += n;
    return true;
}

__device__ __forceinline__ int64_t lin(const Geo& g, int x, int y, int z)
{
    return ((int64_t)z * g.n[1] + y) * g.n[0] + x;
}

template <class T>
__device__ __forceinline__ float ldv(const T* p, int64_t i);
template <>
__device__ __forceinline__ float ldv<float>(const float* p, int64_t i) { return __ldg(p + i); }
template <>
__device__ __forceinline__ float ldv<bf16>(const bf16* p, int64_t i) { return __bfloat162float(p[i]); }

template <class T>
__device__ __forceinline__ void stv(T* p, int64_t i, float v);
template <>
__device__ __forceinline__ void stv<float>(float* p, int64_t i, float v) { p[i] = v; }
template <>
__device__ __forceinline__ void stv<bf16>(bf16* p, int64_t i, float v) { p[i] = __float2bfloat16_rn(v); }

// coefficient of the lower d-face of the cell at (unwrapped) c: 0 on walls and outside
__device__ __forceinline__ float face_lo(const float* a, const Geo& g, int d, int x, int y, int z)
{
    if (!wrapc(x, g.n[0], g.per[0]) || !wrapc(y, g.n[1], g.per[1]) || !wrapc(z, g.n[2], g.per[2]))
        return 0.f;
    const int c = d == 0 ? x : (d == 1 ? y : z);
    if (c == 0 && !g.per[d]) return 0.f;
    return __ldg(a + lin(g, x, y, z));
}

// (A p)_I = sum over the six faces of beta_f (p_nb - p_I), in one fixed order
// (lower/upper x, y, z).  Each difference of two nearby FP32 values is exact,
// so the rounding error scales with the local differences rather than with
// |p|; the form nb - diag * p would cancel and lose ~log2(|p| / |A p|) bits.
// The roundings are spelled out (one product and one fused multiply-add per
// axis, then two adds) so that no kernel's compiled contraction choices change
// them: every kernel that evaluates the operator rounds identically.
__device__ __forceinline__ float face_flux(float bxl, float pxl, float bxu, float pxu, float byl,
                                           float pyl, float byu, float pyu, float bzl, float pzl,
                                           float bzu, float pzu, float p)
{
    const float ax = __fmaf_rn(bxu, __fsub_rn(pxu, p), __fmul_rn(bxl, __fsub_rn(pxl, p)));
    const float ay = __fmaf_rn(byu, __fsub_rn(pyu, p), __fmul_rn(byl, __fsub_rn(pyl, p)));
    const float az = __fmaf_rn(bzu, __fsub_rn(pzu, p), __fmul_rn(bzl, __fsub_rn(pzl, p)));
    return __fadd_rn(__fadd_rn(ax, ay), az);
}

__device__ __forceinline__ float diag_sum(float bxl, float bxu, float byl, float byu, float bzl,
                                          float bzu)
{
    return ((bxl + bxu) + (byl + byu)) + (bzl + bzu);
}

// under-relaxed Gauss-Seidel update of one cell (Sec. 3.1) in correction form:
// (1 - w) p + w (sum beta p_nb - b) / diag = p + w ((A p)_I - b_I) / diag;
// isolated cells (diag = 0) keep p.  The quotient is the fast approximate one
// (2 ulp): a smoother step needs no correctly rounded division, and the
// residual that decides convergence is computed without it.
__device__ __forceinline__ float gs_update(float p, float flux, float dg, float b, float w)
{
    if (!(dg > 0.f)) return p;
    return __fmaf_rn(w, __fdividef(__fsub_rn(flux, b), dg), p);
}

template <class Task>
__device__ __forceinline__ const Task* task_of(const TaskList<Task>& tl, int tile, int& local)
{
    if (!tl.tasks) {
        local = tile;
        return &tl.single;
    }
    int lo = 0, hi = tl.ntasks - 1;
    while (lo < hi) {   // last t with tile_off[t] <= tile
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(tl.tile_off + mid) <= tile) lo = mid;
        else hi = mid - 1;
    }
    local = tile - __ldg(tl.tile_off + lo);
    return tl.tasks + lo;
}

// Programmatic dependent launch (kernels started by launch_pdl): wait until every
// grid this one depends on has completed with its memory visible.  No kernel
// signals its dependents early (griddepcontrol.launch_dependents): they are
// scheduled as its blocks exit, which measured faster on the V-cycle than both
// an early signal (blocks of the next kernel then hold SM resources while they
// wait) and plain stream order.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block, fixed order; result valid in thread 0.  `red` holds one
// double per warp.  Ends with a barrier so `red` may be reused at once.
__device__ __forceinline__ double block_sum(double v, double* red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    __syncthreads();
    return s;
}

// Sum of r * r over the block, result valid in thread 0: FP32 within each warp (a
// fixed five-level tree of 32 non-negative terms, relative error below 5 * 2^-24),
// FP64 across warps.  FP64 arithmetic runs at 1/64 of the FP32 rate on this part,
// so a per-cell FP64 reduction would bound a memory-bound kernel.
__device__ __forceinline__ double block_sum_sq(float r, double* red)
{
    float v = r * r;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    __syncthreads();
    return s;
}

}  // namespace dev
}  // namespace gmg
