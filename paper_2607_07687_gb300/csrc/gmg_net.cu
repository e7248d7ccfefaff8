// gmg_net.cu -- kernels of the learned warm-start network (see include/gmg_net.h).
//
// 3x3x3 convolutions are implicit GEMMs on the tensor cores (mma.sync
// m16n8k16, BF16 operands, FP32 accumulation): M = cells of a 4 x 32 tile of
// one z-plane, N = output channels, K = 27 taps x input channels, one
// 16-channel slice of K at a time staged in shared memory with the tile's
// 3 x 6 x 34 halo.  The input gradient is the same kernel on flipped,
// transposed weights; the weight gradient is a GEMM per (tap, 16-channel
// slice) with the cells as K, split over CTAs and summed with FP32 atomics.
#include "../../include/gmg_net.h"
#include "gmg_hw.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <initializer_list>

namespace gmgnet {
// tcgen05 convolution (gmg_net_tc.cu): 0 done, 1 shapes not supported, 2 CUDA error
int conv3_tc(int D, int H, int W, const void* x, int cx, int ci, const void* w, const float* bias, int co, int relu,
             void* y, int cy, int yoff, cudaStream_t s);
}

namespace {

using bf16 = __nv_bfloat16;

constexpr int TY = 4, TX = 32;              // conv tile: 4 rows of 32 cells
constexpr int HZ = 3, HY = TY + 2, HX = TX + 2, HALO = HZ * HY * HX;
constexpr int kConvThreads = 128;           // one warp per tile row

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct ConvArgs {
    int D, H, W;
    const bf16* x;
    int cx, ci;
    const bf16* w;      // [27][co][ci]
    const float* bias;  // or nullptr
    int relu;
    bf16* y;
    int cy, yoff;
};

// NT = co / 8 output-channel tiles of 8
template <int NT>
__global__ void __launch_bounds__(kConvThreads) k_conv3(const ConvArgs a)
{
    constexpr int CO = NT * 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16* sA = reinterpret_cast<bf16*>(smem_raw);   // [HALO][16]
    bf16* sW = sA + HALO * 16;                      // [27][CO][16]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z;
    const int D = a.D, H = a.H, W = a.W;
    float acc[2][NT][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.f;

    for (int ch = 0; ch < a.ci / 16; ++ch) {
        __syncthreads();   // the previous slice has been consumed
        for (int e = tid; e < HALO * 2; e += kConvThreads) {
            const int h = e >> 1, half = e & 1;
            const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
            const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (gx >= 0 && gx < W && gy >= 0 && gy < H && gz >= 0 && gz < D)
                v = *reinterpret_cast<const uint4*>(a.x + ((int64_t)(gz * H + gy) * W + gx) * a.cx + ch * 16 +
                                                    half * 8);
            *reinterpret_cast<uint4*>(sA + h * 16 + half * 8) = v;
        }
        for (int e = tid; e < 27 * CO * 2; e += kConvThreads) {
            const int r = e >> 1, half = e & 1;
            *reinterpret_cast<uint4*>(sW + r * 16 + half * 8) =
                *reinterpret_cast<const uint4*>(a.w + (int64_t)r * a.ci + ch * 16 + half * 8);
        }
        __syncthreads();
        for (int tap = 0; tap < 27; ++tap) {
            const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                // rows gid and gid + 8 of the m-th 16-cell run of this warp's tile row
                const int h0 = (dz * HY + warp + dy) * HX + 16 * m + gid + dx;
                const bf16* r0 = sA + h0 * 16 + 2 * tig;
                const bf16* r1 = r0 + 8 * 16;
                const uint32_t a0 = ld32(r0), a1 = ld32(r1), a2 = ld32(r0 + 8), a3 = ld32(r1 + 8);
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    const bf16* wb = sW + (tap * CO + n * 8 + gid) * 16 + 2 * tig;
                    mma_bf16(acc[m][n], a0, a1, a2, a3, ld32(wb), ld32(wb + 8));
                }
            }
        }
    }
    const int yy = y0 + warp;
    if (yy >= H) return;
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
            const int xx = x0 + 16 * m + gid + 8 * hf;
            if (xx >= W) continue;
            bf16* out = a.y + ((int64_t)(z0 * H + yy) * W + xx) * a.cy + a.yoff;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const int o = n * 8 + 2 * tig;
                float v0 = acc[m][n][2 * hf], v1 = acc[m][n][2 * hf + 1];
                if (a.bias) {
                    v0 += a.bias[o];
                    v1 += a.bias[o + 1];
                }
                if (a.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                *reinterpret_cast<__nv_bfloat162*>(out + o) = __floats2bfloat162_rn(v0, v1);
            }
        }
}

template <int NT>
cudaError_t launch_conv3(const ConvArgs& a, cudaStream_t s)
{
    const size_t smem = sizeof(bf16) * (HALO * 16 + 27 * NT * 8 * 16);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_conv3<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid((a.W + TX - 1) / TX, (a.H + TY - 1) / TY, a.D);
    k_conv3<NT><<<grid, kConvThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

namespace {

// ---------------------------------------------------------------- weight gradient
// CTA (tap, 16-channel slice of ci, split s) sums over its share of 128-cell
// runs: acc[o][c] += sum_cells g[cell][o] x[cell + offset(tap)][c].  The cell
// run is K: g^T (co x 128) is the A operand, the shifted x (128 x 16) is B.
constexpr int kWgThreads = 128;
constexpr int kWgRun = 128;

template <int MT>   // MT = co / 16
__global__ void __launch_bounds__(kWgThreads) k_conv3_wgrad(int D, int H, int W, const bf16* __restrict__ x, int cx,
                                                            int ci, const bf16* __restrict__ g, int cg,
                                                            float* __restrict__ dw)
{
    constexpr int CO = MT * 16;
    __shared__ __align__(16) bf16 sG[CO][kWgRun + 8];   // g^T of the run (+8: fewer bank conflicts)
    __shared__ __align__(16) bf16 sX[16][kWgRun + 8];   // shifted x^T of the run, one channel slice
    __shared__ float sRed[4][CO][16];
    const int tap = blockIdx.x, slice = blockIdx.y;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int64_t ncell = (int64_t)D * H * W;
    const int64_t nrun = (ncell + kWgRun - 1) / kWgRun;
    float acc[MT][2][4];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int n = 0; n < 2; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.f;

    for (int64_t run = blockIdx.z; run < nrun; run += gridDim.z) {
        const int64_t c0 = run * kWgRun;
        __syncthreads();
        // g^T: 8-channel vectors of each cell scattered into columns
        for (int e = tid; e < kWgRun * (CO / 8); e += kWgThreads) {
            const int p = e / (CO / 8), q = e - p * (CO / 8);
            const int64_t cell = c0 + p;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (cell < ncell) v = *reinterpret_cast<const uint4*>(g + cell * cg + q * 8);
            const bf16* vv = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) sG[q * 8 + j][p] = vv[j];
        }
        // x at cell + offset(tap), zero outside the grid
        for (int e = tid; e < kWgRun * 2; e += kWgThreads) {
            const int p = e >> 1, half = e & 1;
            const int64_t cell = c0 + p;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (cell < ncell) {
                const int xx = (int)(cell % W), yy = (int)((cell / W) % H), zz = (int)(cell / ((int64_t)W * H));
                const int sx = xx + dx, sy = yy + dy, sz = zz + dz;
                if (sx >= 0 && sx < W && sy >= 0 && sy < H && sz >= 0 && sz < D)
                    v = *reinterpret_cast<const uint4*>(x + ((int64_t)(sz * H + sy) * W + sx) * cx + slice * 16 +
                                                        half * 8);
            }
            const bf16* vv = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) sX[half * 8 + j][p] = vv[j];
        }
        __syncthreads();
        // each warp takes two of the eight k-steps of 16 cells
#pragma unroll
        for (int kk = warp * 2; kk < warp * 2 + 2; ++kk) {
            const int k0 = kk * 16 + 2 * tig;
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                const bf16* r0 = &sG[m * 16 + gid][k0];
                const bf16* r1 = &sG[m * 16 + gid + 8][k0];
                const uint32_t a0 = ld32(r0), a1 = ld32(r1), a2 = ld32(r0 + 8), a3 = ld32(r1 + 8);
#pragma unroll
                for (int n = 0; n < 2; ++n) {
                    const bf16* b = &sX[n * 8 + gid][k0];
                    mma_bf16(acc[m][n], a0, a1, a2, a3, ld32(b), ld32(b + 8));
                }
            }
        }
    }
    // sum the four warps' partial tiles, then one atomic per weight
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int n = 0; n < 2; ++n) {
            const int o = m * 16 + gid, c = n * 8 + 2 * tig;
            sRed[warp][o][c] = acc[m][n][0];
            sRed[warp][o][c + 1] = acc[m][n][1];
            sRed[warp][o + 8][c] = acc[m][n][2];
            sRed[warp][o + 8][c + 1] = acc[m][n][3];
        }
    __syncthreads();
    for (int e = tid; e < CO * 16; e += kWgThreads) {
        const int o = e / 16, c = e % 16;
        const float v = sRed[0][o][c] + sRed[1][o][c] + sRed[2][o][c] + sRed[3][o][c];
        atomicAdd(dw + ((int64_t)tap * CO + o) * ci + slice * 16 + c, v);
    }
}

__global__ void k_bias_grad(int64_t ncell, const bf16* __restrict__ g, int cg, int C, float* __restrict__ db)
{
    __shared__ float s[128];
    const int c = threadIdx.x % C, lanes = blockDim.x / C;   // blockDim.x multiple of C
    const int r = threadIdx.x / C;
    float acc = 0.f;
    if (r < lanes)
        for (int64_t cell = (int64_t)blockIdx.x * lanes + r; cell < ncell; cell += (int64_t)gridDim.x * lanes)
            acc += __bfloat162float(g[cell * cg + c]);
    s[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < C) {
        float t = 0.f;
        for (int q = 0; q < lanes; ++q) t += s[q * C + threadIdx.x];
        atomicAdd(db + threadIdx.x, t);
    }
}

// ---------------------------------------------------------------- elementwise

__global__ void k_relu_backward(int64_t ncell, bf16* g, int cg, const bf16* y, int cy, int C)
{
    const int64_t n = ncell * C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = e / C;
        const int c = (int)(e - cell * C);
        if (!(__bfloat162float(y[cell * cy + c]) > 0.f)) g[cell * cg + c] = __float2bfloat16_rn(0.f);
    }
}

// coarse dimensions d, h, w of the 2x pooled / upsampled pair
__global__ void k_pool2(int d, int h, int w, const bf16* x, int cx, int C, bf16* y, int cy, int yoff)
{
    const int64_t n = (int64_t)d * h * w * C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const int64_t cell = e / C;
        const int X = (int)(cell % w), Y = (int)((cell / w) % h), Z = (int)(cell / ((int64_t)w * h));
        float s = 0.f;
        for (int k = 0; k < 8; ++k) {
            const int fx = 2 * X + (k & 1), fy = 2 * Y + ((k >> 1) & 1), fz = 2 * Z + (k >> 2);
            s += __bfloat162float(x[((int64_t)(fz * 2 * h + fy) * 2 * w + fx) * cx + c]);
        }
        y[cell * cy + yoff + c] = __float2bfloat16_rn(0.125f * s);
    }
}

// fine dimensions D, H, W
__global__ void k_pool2_backward(int D, int H, int W, const bf16* gy, int cgy, int C, bf16* gx, int cgx,
                                 const bf16* add, int cadd, int addoff)
{
    const int64_t n = (int64_t)D * H * W * C;
    const int h = H / 2, w = W / 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const int64_t cell = e / C;
        const int xx = (int)(cell % W), yy = (int)((cell / W) % H), zz = (int)(cell / ((int64_t)W * H));
        float v = 0.125f * __bfloat162float(gy[((int64_t)((zz / 2) * h + yy / 2) * w + xx / 2) * cgy + c]);
        if (add) v += __bfloat162float(add[cell * cadd + addoff + c]);
        gx[cell * cgx + c] = __float2bfloat16_rn(v);
    }
}

// coarse dimensions d, h, w
__global__ void k_up2(int d, int h, int w, const bf16* x, int cx, int C, bf16* y, int cy, int yoff)
{
    const int64_t n = (int64_t)8 * d * h * w * C;
    const int H = 2 * h, W = 2 * w;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const int64_t cell = e / C;
        const int xx = (int)(cell % W), yy = (int)((cell / W) % H), zz = (int)(cell / ((int64_t)W * H));
        y[cell * cy + yoff + c] = x[((int64_t)((zz / 2) * h + yy / 2) * w + xx / 2) * cx + c];
    }
}

__global__ void k_up2_backward(int d, int h, int w, const bf16* gy, int cgy, int goff, int C, bf16* gx, int cgx)
{
    const int64_t n = (int64_t)d * h * w * C;
    const int H = 2 * h, W = 2 * w;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const int64_t cell = e / C;
        const int X = (int)(cell % w), Y = (int)((cell / w) % h), Z = (int)(cell / ((int64_t)w * h));
        float s = 0.f;
        for (int k = 0; k < 8; ++k) {
            const int fx = 2 * X + (k & 1), fy = 2 * Y + ((k >> 1) & 1), fz = 2 * Z + (k >> 2);
            s += __bfloat162float(gy[((int64_t)(fz * H + fy) * W + fx) * cgy + goff + c]);
        }
        gx[cell * cgx + c] = __float2bfloat16_rn(s);
    }
}

// ---- the same elementwise kernels on 8-channel chunks (16-byte loads and stores),
// for channel counts, strides and offsets that are multiples of 8; identical sums

__device__ __forceinline__ void unpack8(const uint4& v, float* f)
{
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 t = __bfloat1622float2(h[j]);
        f[2 * j] = t.x;
        f[2 * j + 1] = t.y;
    }
}

__device__ __forceinline__ uint4 pack8(const float* f)
{
    uint4 v;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
    return v;
}

__device__ __forceinline__ const uint4& ld8(const bf16* p) { return *reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ uint4& st8(bf16* p) { return *reinterpret_cast<uint4*>(p); }

__global__ void k_relu_backward_v(int64_t ncell, bf16* g, int cg, const bf16* y, int cy, int C)
{
    const int nq = C / 8;
    const int64_t n = ncell * nq;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = e / nq;
        const int q = (int)(e - cell * nq);
        float gv[8], yv[8];
        unpack8(ld8(g + cell * cg + 8 * q), gv);
        unpack8(ld8(y + cell * cy + 8 * q), yv);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (!(yv[j] > 0.f)) gv[j] = 0.f;
        st8(g + cell * cg + 8 * q) = pack8(gv);
    }
}

__global__ void k_pool2_v(int d, int h, int w, const bf16* x, int cx, int C, bf16* y, int cy, int yoff)
{
    const int nq = C / 8;
    const int64_t n = (int64_t)d * h * w * nq;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = e / nq;
        const int q = (int)(e - cell * nq);
        const int X = (int)(cell % w), Y = (int)((cell / w) % h), Z = (int)(cell / ((int64_t)w * h));
        float sum[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < 8; ++k) {
            const int fx = 2 * X + (k & 1), fy = 2 * Y + ((k >> 1) & 1), fz = 2 * Z + (k >> 2);
            float v[8];
            unpack8(ld8(x + ((int64_t)(fz * 2 * h + fy) * 2 * w + fx) * cx + 8 * q), v);
#pragma unroll
            for (int j = 0; j < 8; ++j) sum[j] += v[j];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) sum[j] *= 0.125f;
        st8(y + cell * cy + yoff + 8 * q) = pack8(sum);
    }
}

__global__ void k_pool2_backward_v(int D, int H, int W, const bf16* gy, int cgy, int C, bf16* gx, int cgx,
                                   const bf16* add, int cadd, int addoff)
{
    const int nq = C / 8;
    const int64_t n = (int64_t)D * H * W * nq;
    const int h = H / 2, w = W / 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = e / nq;
        const int q = (int)(e - cell * nq);
        const int xx = (int)(cell % W), yy = (int)((cell / W) % H), zz = (int)(cell / ((int64_t)W * H));
        float v[8];
        unpack8(ld8(gy + ((int64_t)((zz / 2) * h + yy / 2) * w + xx / 2) * cgy + 8 * q), v);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] *= 0.125f;
        if (add) {
            float a[8];
            unpack8(ld8(add + cell * cadd + addoff + 8 * q), a);
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] += a[j];
        }
        st8(gx + cell * cgx + 8 * q) = pack8(v);
    }
}

__global__ void k_up2_v(int d, int h, int w, const bf16* x, int cx, int C, bf16* y, int cy, int yoff)
{
    const int nq = C / 8;
    const int64_t n = (int64_t)8 * d * h * w * nq;
    const int H = 2 * h, W = 2 * w;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = e / nq;
        const int q = (int)(e - cell * nq);
        const int xx = (int)(cell % W), yy = (int)((cell / W) % H), zz = (int)(cell / ((int64_t)W * H));
        st8(y + cell * cy + yoff + 8 * q) = ld8(x + ((int64_t)((zz / 2) * h + yy / 2) * w + xx / 2) * cx + 8 * q);
    }
}

__global__ void k_up2_backward_v(int d, int h, int w, const bf16* gy, int cgy, int goff, int C, bf16* gx, int cgx)
{
    const int nq = C / 8;
    const int64_t n = (int64_t)d * h * w * nq;
    const int H = 2 * h, W = 2 * w;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = e / nq;
        const int q = (int)(e - cell * nq);
        const int X = (int)(cell % w), Y = (int)((cell / w) % h), Z = (int)(cell / ((int64_t)w * h));
        float sum[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < 8; ++k) {
            const int fx = 2 * X + (k & 1), fy = 2 * Y + ((k >> 1) & 1), fz = 2 * Z + (k >> 2);
            float v[8];
            unpack8(ld8(gy + ((int64_t)(fz * H + fy) * W + fx) * cgy + goff + 8 * q), v);
#pragma unroll
            for (int j = 0; j < 8; ++j) sum[j] += v[j];
        }
        st8(gx + cell * cgx + 8 * q) = pack8(sum);
    }
}

// 16-byte chunks apply: channel counts, strides and offsets multiples of 8, aligned pointers
bool chunked(std::initializer_list<long long> counts, std::initializer_list<const void*> ptrs)
{
    for (long long c : counts)
        if (c % 8) return false;
    for (const void* p : ptrs)
        if (p && ((uintptr_t)p & 15)) return false;
    return true;
}

int grid_of(int64_t n, int threads = 256)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    const int64_t cap = (int64_t)gmg::sm_count() * 16;
    if (b > cap) b = cap;
    return (int)b;
}

int status(cudaError_t e) { return e == cudaSuccess ? 0 : 2; }

}  // namespace

namespace {

// ---------------------------------------------------------------- input, head, loss, optimiser

// lower face coefficient of cell (x, y, z) along d, 0 on walls
__device__ __forceinline__ float face_lo(const float* a, int D, int H, int W, const int* per, int d, int x, int y,
                                         int z)
{
    int c[3] = {x, y, z};
    const int n[3] = {W, H, D};
    for (int e = 0; e < 3; ++e) {
        if (c[e] < 0 || c[e] >= n[e]) {
            if (!per[e]) return 0.f;
            c[e] = (c[e] % n[e] + n[e]) % n[e];
        }
    }
    if (c[d] == 0 && !per[d]) return 0.f;
    return a[((int64_t)c[2] * H + c[1]) * W + c[0]];
}

// p at (x, y, z) with periodic wrap; 0 outside a wall (its face is 0 there)
__device__ __forceinline__ float p_at(const float* p, int D, int H, int W, const int* per, int x, int y, int z)
{
    int c[3] = {x, y, z};
    const int n[3] = {W, H, D};
    for (int e = 0; e < 3; ++e) {
        if (c[e] < 0 || c[e] >= n[e]) {
            if (!per[e]) return 0.f;
            c[e] = (c[e] % n[e] + n[e]) % n[e];
        }
    }
    return p[((int64_t)c[2] * H + c[1]) * W + c[0]];
}

struct PackCell {
    float b, r, mean;
};

// b, the residual b - A p_prev (difference form, FP32) and the mean of the six faces of one cell
__device__ __forceinline__ PackCell pack_cell(int D, int H, int W, const float* b, const float* pp, const float* bx,
                                              const float* by, const float* bz, const int* per, int64_t i)
{
    const int x = (int)(i % W), y = (int)((i / W) % H), z = (int)(i / ((int64_t)W * H));
    const float fx0 = face_lo(bx, D, H, W, per, 0, x, y, z), fx1 = face_lo(bx, D, H, W, per, 0, x + 1, y, z);
    const float fy0 = face_lo(by, D, H, W, per, 1, x, y, z), fy1 = face_lo(by, D, H, W, per, 1, x, y + 1, z);
    const float fz0 = face_lo(bz, D, H, W, per, 2, x, y, z), fz1 = face_lo(bz, D, H, W, per, 2, x, y, z + 1);
    PackCell c;
    c.b = b[i];
    c.mean = (fx0 + fx1 + fy0 + fy1 + fz0 + fz1) / 6.f;
    c.r = c.b;
    if (pp) {
        const float p = pp[i];
        const float flux = ((fx0 * (p_at(pp, D, H, W, per, x - 1, y, z) - p) +
                             fx1 * (p_at(pp, D, H, W, per, x + 1, y, z) - p)) +
                            (fy0 * (p_at(pp, D, H, W, per, x, y - 1, z) - p) +
                             fy1 * (p_at(pp, D, H, W, per, x, y + 1, z) - p))) +
                           (fz0 * (p_at(pp, D, H, W, per, x, y, z - 1) - p) +
                            fz1 * (p_at(pp, D, H, W, per, x, y, z + 1) - p));
        c.r = c.b - flux;
    }
    return c;
}

// red[0] += sum b^2, red[1] += sum r^2
__global__ void k_pack_sums(int D, int H, int W, const float* b, const float* pp, const float* bx, const float* by,
                            const float* bz, int px, int py, int pz, double* red)
{
    const int per[3] = {px, py, pz};
    const int64_t n = (int64_t)D * H * W;
    double sb = 0.0, sr = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const PackCell c = pack_cell(D, H, W, b, pp, bx, by, bz, per, i);
        sb += (double)c.b * c.b;
        sr += (double)c.r * c.r;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(red, sb);
        atomicAdd(red + 1, sr);
    }
}

// s[0] = RMS(b), s[1] = RMS(r) (1 where zero)
__global__ void k_scales(const double* red, int64_t n, float* s)
{
    for (int k = 0; k < 2; ++k) {
        const double v = sqrt(red[k] / (double)n);
        s[k] = v > 0.0 ? (float)v : 1.f;
    }
}

__global__ void k_pack_input(int D, int H, int W, const float* b, const float* pp, const float* bx, const float* by,
                             const float* bz, int px, int py, int pz, const float* s, bf16* x0)
{
    const int per[3] = {px, py, pz};
    const int64_t n = (int64_t)D * H * W;
    const float inv = 1.f / s[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const PackCell c = pack_cell(D, H, W, b, pp, bx, by, bz, per, i);
        bf16* o = x0 + i * 16;
        o[0] = __float2bfloat16_rn(c.b * inv);
        o[1] = __float2bfloat16_rn(c.mean);
        o[2] = __float2bfloat16_rn(pp ? pp[i] * inv : 0.f);
        o[3] = __float2bfloat16_rn(c.r * inv);
        for (int k = 4; k < 16; ++k) o[k] = __float2bfloat16_rn(0.f);
    }
}

// flux sum_f beta_f (v_nb - v_c) of the solver's operator at cell i (difference form)
__device__ __forceinline__ float flux_of(const float* v, int D, int H, int W, const float* bx, const float* by,
                                         const float* bz, const int* per, int64_t i)
{
    const int x = (int)(i % W), y = (int)((i / W) % H), z = (int)(i / ((int64_t)W * H));
    const float c = v[i];
    return ((face_lo(bx, D, H, W, per, 0, x, y, z) * (p_at(v, D, H, W, per, x - 1, y, z) - c) +
             face_lo(bx, D, H, W, per, 0, x + 1, y, z) * (p_at(v, D, H, W, per, x + 1, y, z) - c)) +
            (face_lo(by, D, H, W, per, 1, x, y, z) * (p_at(v, D, H, W, per, x, y - 1, z) - c) +
             face_lo(by, D, H, W, per, 1, x, y + 1, z) * (p_at(v, D, H, W, per, x, y + 1, z) - c))) +
           (face_lo(bz, D, H, W, per, 2, x, y, z) * (p_at(v, D, H, W, per, x, y, z - 1) - c) +
            face_lo(bz, D, H, W, per, 2, x, y, z + 1) * (p_at(v, D, H, W, per, x, y, z + 1) - c));
}

// p0 = p_prev + s out
__global__ void k_rloss_p0(int64_t n, const float* out, const float* pp, const float* s, float* p0)
{
    const float sc = *s;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p0[i] = pp ? fmaf(sc, out[i], pp[i]) : sc * out[i];
}

// r = b - A p0; red[0] += sum r^2, red[1] += sum b^2
__global__ void k_rloss_r(int D, int H, int W, const float* p0, const float* b, const float* bx, const float* by,
                          const float* bz, int px, int py, int pz, float* r, double* red)
{
    const int per[3] = {px, py, pz};
    const int64_t n = (int64_t)D * H * W;
    double sr = 0.0, sb = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = b[i] - flux_of(p0, D, H, W, bx, by, bz, per, i);
        r[i] = v;
        sr += (double)v * v;
        sb += (double)b[i] * b[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(red, sr);
        atomicAdd(red + 1, sb);
    }
}

// gout = s (-2 A r / |b|^2); loss = |r|^2 / |b|^2
__global__ void k_rloss_grad(int D, int H, int W, const float* r, const float* bx, const float* by, const float* bz,
                             int px, int py, int pz, const float* s, const double* red, float* gout, double* loss)
{
    const int per[3] = {px, py, pz};
    const int64_t n = (int64_t)D * H * W;
    const double den = red[1] > 0.0 ? red[1] : 1.0;
    const float scale = (float)(-2.0 * (double)*s / den);
    if (blockIdx.x == 0 && threadIdx.x == 0) *loss = red[0] / den;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        gout[i] = scale * flux_of(r, D, H, W, bx, by, bz, per, i);
}

__global__ void k_head(int64_t n, const bf16* h, int ch, const float* w, const float* b, float* out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float s = b[0];
        for (int c = 0; c < 16; ++c) s += w[c] * __bfloat162float(h[i * ch + c]);
        out[i] = s;
    }
}

// prediction q = out + p_prev / s in units of s
__device__ __forceinline__ double pred(const float* out, const float* p_prev, double inv, int64_t i)
{
    return p_prev ? (double)out[i] + (double)p_prev[i] * inv : (double)out[i];
}

// red[0] = sum q, red[1] = sum t, (second pass) red[2] = sum (t - mt)^2, red[3] = sum diff^2
__global__ void k_loss_sums(int64_t n, const float* out, const float* target, const float* p_prev, const float* s,
                            double* red, int pass)
{
    const double inv = 1.0 / (double)*s;
    const double mo = pass ? red[0] / (double)n : 0.0, mt = pass ? red[1] / (double)n : 0.0;
    double a = 0.0, c = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double t = (double)target[i] * inv;
        if (pass == 0) {
            a += pred(out, p_prev, inv, i);
            c += t;
        } else {
            const double tc = t - mt, d = (pred(out, p_prev, inv, i) - mo) - tc;
            a += tc * tc;
            c += d * d;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(red + 2 * pass, a);
        atomicAdd(red + 2 * pass + 1, c);
    }
}

__global__ void k_loss_grad(int64_t n, const float* out, const float* target, const float* p_prev, const float* s,
                            const double* red, float* gout, double* loss)
{
    const double inv = 1.0 / (double)*s;
    const double mo = red[0] / (double)n, mt = red[1] / (double)n, den = red[2] > 0.0 ? red[2] : 1.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *loss = red[3] / den;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = (pred(out, p_prev, inv, i) - mo) - ((double)target[i] * inv - mt);
        gout[i] = (float)(2.0 * d / den);
    }
}

__global__ void k_head_backward(int64_t n, const float* gout, const bf16* h, int ch, const float* w, bf16* gh,
                                float* dw, float* db)
{
    float aw[16];
    for (int c = 0; c < 16; ++c) aw[c] = 0.f;
    float ab = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float g = gout[i];
        ab += g;
        for (int c = 0; c < 16; ++c) {
            aw[c] += g * __bfloat162float(h[i * ch + c]);
            gh[i * 16 + c] = __float2bfloat16_rn(w[c] * g);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ab += __shfl_xor_sync(0xffffffffu, ab, o);
        for (int c = 0; c < 16; ++c) aw[c] += __shfl_xor_sync(0xffffffffu, aw[c], o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(db, ab);
        for (int c = 0; c < 16; ++c) atomicAdd(dw + c, aw[c]);
    }
}

__global__ void k_unscale(int64_t n, const float* out, const float* s, const float* p_prev, float* p0)
{
    const float sc = *s;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p0[i] = p_prev ? fmaf(sc, out[i], p_prev[i]) : sc * out[i];
}

// Adam; weights packed [27][co][ci] also land as BF16 and, flipped and
// transposed ([26 - t][ci][co]), as the input-gradient weights
__global__ void k_adam(int64_t n, float* w, const float* g, float* m, float* v, float lr, float b1, float b2,
                       float eps, float c1, float c2, bf16* wb, bf16* wt, int co, int ci)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16_rn(wi);
        if (wt && ci > 0) {
            const int64_t t = i / ((int64_t)co * ci);
            const int rem = (int)(i - t * co * ci);
            const int o = rem / ci, c = rem - o * ci;
            wt[((26 - t) * ci + c) * co + o] = __float2bfloat16_rn(wi);
        }
    }
}

__global__ void k_zero(int64_t n, float* a)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = 0.f;
}

}  // namespace

// ---------------------------------------------------------------- C ABI

extern "C" {

int gmg_net_conv3(int D, int H, int W, const gmg_bf16* x, int cx, int ci, const gmg_bf16* w, const float* bias,
                  int co, int relu, gmg_bf16* y, int cy, int yoff, void* stream)
{
    if (D < 1 || H < 1 || W < 1 || !x || !w || !y || ci < 16 || ci % 16 || co < 16 || co % 16 || co > 96 ||
        cx < ci || cx % 8 || cy % 2 || yoff % 2 || cy < yoff + co)
        return 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int tc = gmgnet::conv3_tc(D, H, W, x, cx, ci, w, bias, co, relu, y, cy, yoff, s);
    if (tc != 1) return tc;
    ConvArgs a{D, H, W, reinterpret_cast<const bf16*>(x), cx, ci, reinterpret_cast<const bf16*>(w), bias, relu,
               reinterpret_cast<bf16*>(y), cy, yoff};
    switch (co / 8) {
    case 2: return status(launch_conv3<2>(a, s));
    case 4: return status(launch_conv3<4>(a, s));
    case 6: return status(launch_conv3<6>(a, s));
    case 8: return status(launch_conv3<8>(a, s));
    case 12: return status(launch_conv3<12>(a, s));
    default: return 1;
    }
}

int gmg_net_conv3_wgrad(int D, int H, int W, const gmg_bf16* x, int cx, int ci, const gmg_bf16* g, int cg, int co,
                        float* dw, float* db, void* stream)
{
    if (D < 1 || H < 1 || W < 1 || !x || !g || !dw || ci < 16 || ci % 16 || cx < ci || cx % 8 || cg % 8 ||
        cg < co)
        return 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t ncell = (int64_t)D * H * W;
    const int64_t runs = (ncell + kWgRun - 1) / kWgRun;
    const int splits = (int)std::min<int64_t>(runs, std::max<int64_t>(1, ((int64_t)gmg::sm_count() * 8) / (27 * (ci / 16))));
    const dim3 grid(27, ci / 16, splits);
    const bf16* xb = reinterpret_cast<const bf16*>(x);
    const bf16* gb = reinterpret_cast<const bf16*>(g);
    switch (co) {
    case 16: k_conv3_wgrad<1><<<grid, kWgThreads, 0, s>>>(D, H, W, xb, cx, ci, gb, cg, dw); break;
    case 32: k_conv3_wgrad<2><<<grid, kWgThreads, 0, s>>>(D, H, W, xb, cx, ci, gb, cg, dw); break;
    case 64: k_conv3_wgrad<4><<<grid, kWgThreads, 0, s>>>(D, H, W, xb, cx, ci, gb, cg, dw); break;
    default: return 1;
    }
    if (db) k_bias_grad<<<grid_of(ncell, 128), 128, 0, s>>>(ncell, gb, cg, co, db);
    return status(cudaGetLastError());
}

int gmg_net_relu_backward(int D, int H, int W, gmg_bf16* g, int cg, const gmg_bf16* y, int cy, int C, void* stream)
{
    if (!g || !y || C < 1) return 1;
    const int64_t n = (int64_t)D * H * W;
    if (chunked({cg, cy, C}, {g, y})) {
        k_relu_backward_v<<<grid_of(n * C / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
            n, reinterpret_cast<bf16*>(g), cg, reinterpret_cast<const bf16*>(y), cy, C);
        return status(cudaGetLastError());
    }
    k_relu_backward<<<grid_of(n * C), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n, reinterpret_cast<bf16*>(g), cg, reinterpret_cast<const bf16*>(y), cy, C);
    return status(cudaGetLastError());
}

int gmg_net_pool2(int D, int H, int W, const gmg_bf16* x, int cx, int C, gmg_bf16* y, int cy, int yoff, void* stream)
{
    if (!x || !y || D % 2 || H % 2 || W % 2 || C < 1) return 1;
    if (chunked({cx, cy, yoff, C}, {x, y})) {
        k_pool2_v<<<grid_of((int64_t)D * H * W * C / 64), 256, 0, static_cast<cudaStream_t>(stream)>>>(
            D / 2, H / 2, W / 2, reinterpret_cast<const bf16*>(x), cx, C, reinterpret_cast<bf16*>(y), cy, yoff);
        return status(cudaGetLastError());
    }
    k_pool2<<<grid_of((int64_t)D * H * W * C / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        D / 2, H / 2, W / 2, reinterpret_cast<const bf16*>(x), cx, C, reinterpret_cast<bf16*>(y), cy, yoff);
    return status(cudaGetLastError());
}

int gmg_net_pool2_backward(int D, int H, int W, const gmg_bf16* gy, int cgy, int C, gmg_bf16* gx, int cgx,
                           const gmg_bf16* add, int cadd, int addoff, void* stream)
{
    if (!gy || !gx || D % 2 || H % 2 || W % 2 || C < 1) return 1;
    if (chunked({cgy, cgx, C, add ? cadd : 0, add ? addoff : 0}, {gy, gx, add})) {
        k_pool2_backward_v<<<grid_of((int64_t)D * H * W * C / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
            D, H, W, reinterpret_cast<const bf16*>(gy), cgy, C, reinterpret_cast<bf16*>(gx), cgx,
            reinterpret_cast<const bf16*>(add), cadd, addoff);
        return status(cudaGetLastError());
    }
    k_pool2_backward<<<grid_of((int64_t)D * H * W * C), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        D, H, W, reinterpret_cast<const bf16*>(gy), cgy, C, reinterpret_cast<bf16*>(gx), cgx,
        reinterpret_cast<const bf16*>(add), cadd, addoff);
    return status(cudaGetLastError());
}

int gmg_net_up2(int D, int H, int W, const gmg_bf16* x, int cx, int C, gmg_bf16* y, int cy, int yoff, void* stream)
{
    if (!x || !y || C < 1) return 1;
    if (chunked({cx, cy, yoff, C}, {x, y})) {
        k_up2_v<<<grid_of((int64_t)D * H * W * C), 256, 0, static_cast<cudaStream_t>(stream)>>>(
            D, H, W, reinterpret_cast<const bf16*>(x), cx, C, reinterpret_cast<bf16*>(y), cy, yoff);
        return status(cudaGetLastError());
    }
    k_up2<<<grid_of((int64_t)8 * D * H * W * C), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        D, H, W, reinterpret_cast<const bf16*>(x), cx, C, reinterpret_cast<bf16*>(y), cy, yoff);
    return status(cudaGetLastError());
}

int gmg_net_up2_backward(int D, int H, int W, const gmg_bf16* gy, int cgy, int goff, int C, gmg_bf16* gx, int cgx,
                         void* stream)
{
    if (!gy || !gx || C < 1) return 1;
    if (chunked({cgy, goff, cgx, C}, {gy, gx})) {
        k_up2_backward_v<<<grid_of((int64_t)D * H * W * C / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
            D, H, W, reinterpret_cast<const bf16*>(gy), cgy, goff, C, reinterpret_cast<bf16*>(gx), cgx);
        return status(cudaGetLastError());
    }
    k_up2_backward<<<grid_of((int64_t)D * H * W * C), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        D, H, W, reinterpret_cast<const bf16*>(gy), cgy, goff, C, reinterpret_cast<bf16*>(gx), cgx);
    return status(cudaGetLastError());
}

int gmg_net_pack_input(int D, int H, int W, const float* b, const float* p_prev, const float* bx, const float* by,
                       const float* bz, const int* periodic, gmg_bf16* x0, float* s_out, double* red, void* stream)
{
    if (!b || !bx || !by || !bz || !x0 || !s_out || !red) return 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = (int64_t)D * H * W;
    cudaError_t e = cudaMemsetAsync(red, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return 2;
    const int px = periodic ? periodic[0] != 0 : 0, py = periodic ? periodic[1] != 0 : 0,
              pz = periodic ? periodic[2] != 0 : 0;
    k_pack_sums<<<grid_of(n), 256, 0, s>>>(D, H, W, b, p_prev, bx, by, bz, px, py, pz, red);
    k_scales<<<1, 1, 0, s>>>(red, n, s_out);
    k_pack_input<<<grid_of(n), 256, 0, s>>>(D, H, W, b, p_prev, bx, by, bz, px, py, pz, s_out,
                                            reinterpret_cast<bf16*>(x0));
    return status(cudaGetLastError());
}

int gmg_net_head(int D, int H, int W, const gmg_bf16* h, int ch, const float* w, const float* b, float* out,
                 void* stream)
{
    if (!h || !w || !b || !out || ch < 16) return 1;
    const int64_t n = (int64_t)D * H * W;
    k_head<<<grid_of(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, reinterpret_cast<const bf16*>(h), ch, w, b,
                                                                      out);
    return status(cudaGetLastError());
}

int gmg_net_loss(int D, int H, int W, const float* out, const float* target, const float* p_prev, const float* s,
                 float* gout, double* loss, double* red, void* stream)
{
    if (!out || !target || !s || !gout || !loss || !red) return 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = (int64_t)D * H * W;
    cudaError_t e = cudaMemsetAsync(red, 0, 4 * sizeof(double), st);
    if (e != cudaSuccess) return 2;
    k_loss_sums<<<grid_of(n), 256, 0, st>>>(n, out, target, p_prev, s, red, 0);
    k_loss_sums<<<grid_of(n), 256, 0, st>>>(n, out, target, p_prev, s, red, 1);
    k_loss_grad<<<grid_of(n), 256, 0, st>>>(n, out, target, p_prev, s, red, gout, loss);
    return status(cudaGetLastError());
}

int gmg_net_residual_loss(int D, int H, int W, const float* out, const float* p_prev, const float* s, const float* b,
                          const float* bx, const float* by, const float* bz, const int* periodic, float* work,
                          float* gout, double* loss, double* red, void* stream)
{
    if (!out || !s || !b || !bx || !by || !bz || !work || !gout || !loss || !red) return 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = (int64_t)D * H * W;
    const int px = periodic ? periodic[0] != 0 : 0, py = periodic ? periodic[1] != 0 : 0,
              pz = periodic ? periodic[2] != 0 : 0;
    cudaError_t e = cudaMemsetAsync(red, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess) return 2;
    float* p0 = work;
    float* r = work + n;
    k_rloss_p0<<<grid_of(n), 256, 0, st>>>(n, out, p_prev, s, p0);
    k_rloss_r<<<grid_of(n), 256, 0, st>>>(D, H, W, p0, b, bx, by, bz, px, py, pz, r, red);
    k_rloss_grad<<<grid_of(n), 256, 0, st>>>(D, H, W, r, bx, by, bz, px, py, pz, s, red, gout, loss);
    return status(cudaGetLastError());
}

int gmg_net_head_backward(int D, int H, int W, const float* gout, const gmg_bf16* h, int ch, const float* w,
                          gmg_bf16* gh, float* dw, float* db, void* stream)
{
    if (!gout || !h || !w || !gh || !dw || !db || ch < 16) return 1;
    const int64_t n = (int64_t)D * H * W;
    k_head_backward<<<grid_of(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n, gout, reinterpret_cast<const bf16*>(h), ch, w, reinterpret_cast<bf16*>(gh), dw, db);
    return status(cudaGetLastError());
}

int gmg_net_unscale(long long n, const float* out, const float* s, const float* p_prev, float* p0, void* stream)
{
    if (!out || !s || !p0 || n < 0) return 1;
    k_unscale<<<grid_of(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, out, s, p_prev, p0);
    return status(cudaGetLastError());
}

int gmg_net_adam(long long n, float* w, const float* g, float* m, float* v, int t, float lr, float b1, float b2,
                 float eps, gmg_bf16* wb, gmg_bf16* wt, int co, int ci, void* stream)
{
    if (!w || !g || !m || !v || t < 1 || n < 0) return 1;
    if (wt && (ci <= 0 || co <= 0 || n != 27LL * co * ci)) return 1;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<grid_of(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, w, g, m, v, lr, b1, b2, eps, c1, c2,
                                                                      reinterpret_cast<bf16*>(wb),
                                                                      reinterpret_cast<bf16*>(wt), co, ci);
    return status(cudaGetLastError());
}

int gmg_net_zero(long long n, float* a, void* stream)
{
    if (!a || n < 0) return 1;
    k_zero<<<grid_of(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, a);
    return status(cudaGetLastError());
}

}  // extern "C"
