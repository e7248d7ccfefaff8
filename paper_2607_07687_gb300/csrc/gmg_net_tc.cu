// gmg_net_tc.cu -- the warm-start network's 3x3x3 convolution on the fifth-
// generation tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// Implicit GEMM per CTA: T row tiles, each D_r[128 cells x N out-channels]
// (FP32, T x N columns of TMEM) = sum over 16-channel input slices s and taps t
// of A_{s,t,r}[128 x 16] B_{s,t}[16 x N].  The 128 cells of row tile r are
// consecutive x positions of row y0 + r of plane z0.  For a slice, all 128
// threads bring the input window x0-1 .. x0+128, y0-1 .. y0+T, z0-1 .. z0+1
// into shared memory as [chunk][3 z][T+2 y][130 x][8 channels] (two 8-channel
// chunks; zeros outside the grid = zero padding) and the slice's weights as
// [chunk][27 taps][N][8], shared by the T row tiles, with 16-byte asynchronous
// copies (one per position and chunk, zero-filled outside the grid).  For tap
// (dz, dy, dx) and row tile r the A
// operand is the 128 consecutive positions that start at window row
// (dz, r + dy), column dx: a uniform layout of 8-row x 16-byte core matrices
// (stride 128 B along M, one chunk region along K), so every (tap, row) is one
// descriptor and one MMA of K = 16 without any im2col copy.
//
// One thread issues the MMAs; their completion is tracked by an mbarrier with
// bounded waits.  The epilogue reads TMEM (tcgen05.ld 32x32b), adds the bias,
// applies ReLU and writes BF16 channels-last.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>
#include <algorithm>

#include "gmg_hw.h"

namespace gmgnet {

namespace {

using bf16 = __nv_bfloat16;

constexpr int kTcM = 128;                      // cells per row tile (one MMA's M)
constexpr int kTcHX = kTcM + 2;                // window columns
constexpr int kTcThreads = 128;
constexpr int kWaitTries = 1 << 22;

// row tiles per CTA for N output channels (T x N TMEM columns, shared memory)
__host__ __device__ constexpr int tc_rows(int n) { return 4; }
// bytes of one 8-channel window chunk (3 x (T+2) x 130 x 16 B) ...
__host__ __device__ constexpr uint32_t tc_box_a(int t) { return 3u * (t + 2) * kTcHX * 16; }
// ... padded so that every operand region starts on a 128-byte boundary
__host__ __device__ constexpr uint32_t tc_chunk_a(int t) { return (tc_box_a(t) + 127) / 128 * 128; }

__device__ int g_tc_fault = 0;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity)
{
    for (int i = 0; i < kWaitTries; ++i)
        if (try_wait(bar, parity)) return true;
    return false;
}

// shared-memory matrix descriptor: no swizzle, K-major core matrices of 8 rows x 16 bytes
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);   // version 1, layout 0 (none)
}

// instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M = 128, N
__host__ __device__ constexpr uint32_t idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

// Epilogue of one output plane z0: warp w owns TMEM lanes (cells) 32w .. 32w+31 of
// every row tile; accumulators at columns [tmem + r N, tmem + (r + 1) N) for row tile r
template <int N, int T>
__device__ __forceinline__ void conv_epilogue(uint32_t tmem, int warp, int lane, int x0, int y0, int z0, int H, int W,
                                              const float* __restrict__ bias, int relu, bf16* __restrict__ y, int cy,
                                              int yoff)
{
    const int cell_x = x0 + warp * 32 + lane;
    for (int r = 0; r < T; ++r) {
        const int yr = y0 + r;
        bf16* out = y + (((int64_t)z0 * H + (yr < H ? yr : 0)) * W + cell_x) * cy + yoff;
        const bool valid = cell_x < W && yr < H;
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t q[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(r * N + c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];\n"
                : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
                  "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]),
                  "=r"(q[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (valid) {
                uint32_t packed[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float v0 = __uint_as_float(q[2 * j]), v1 = __uint_as_float(q[2 * j + 1]);
                    if (bias) {
                        v0 += bias[c0 + 2 * j];
                        v1 += bias[c0 + 2 * j + 1];
                    }
                    if (relu) {
                        v0 = fmaxf(v0, 0.f);
                        v1 = fmaxf(v1, 0.f);
                    }
                    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                    packed[j] = *reinterpret_cast<const uint32_t*>(&h);
                }
                uint4* o4 = reinterpret_cast<uint4*>(out + c0);
                o4[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                o4[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
            }
        }
    }
}

template <int N>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_conv3_tc(const bf16* __restrict__ x, int cx, const bf16* __restrict__ w, int D, int H, int W, int ci,
               const float* __restrict__ bias, int relu, bf16* __restrict__ y, int cy, int yoff)
{
    static_assert(N % 16 == 0 && N >= 16 && N <= 128, "N: multiple of 16 up to 128");
    constexpr int T = tc_rows(N);
    constexpr int WR = T + 2;                                  // window rows per plane
    constexpr uint32_t kChunkA = tc_chunk_a(T);
    constexpr uint32_t kChunkB = 27 * N * 16;                 // bytes of one 8-channel weight chunk
    static_assert(kChunkA % 128 == 0 && kChunkB % 128 == 0, "operand regions: 128-byte aligned");
    constexpr int kCols = T * N <= 32 ? 32 : (T * N <= 64 ? 64 : (T * N <= 128 ? 128 : (T * N <= 256 ? 256 : 512)));
    static_assert(T * N <= 512, "accumulators fit in TMEM");
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* sA = smem;                                  // [2][3][T+2][130][8] bf16
    unsigned char* sB = smem + 2 * kChunkA;                    // [2][27][N][8] bf16
    __shared__ __align__(8) uint64_t mma_done;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = (W + kTcM - 1) / kTcM, tiles_y = (H + T - 1) / T;
    const int x0 = (blockIdx.x % tiles_x) * kTcM;
    const int yb = (blockIdx.x / tiles_x) % tiles_y;
    const int y0 = yb * T, z0 = blockIdx.x / (tiles_x * tiles_y);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tmem_base)),
                     "n"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&mma_done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    bool ok = true;
    const uint32_t a0 = su32(sA), b0 = su32(sB);
    const int slices = ci / 16;
    const int nrow = 3 * WR;                                   // window rows (z, y)
    for (int s = 0; s < slices && ok; ++s) {
        const uint32_t par = (uint32_t)s & 1u;
        // window: position p of window row (rz, ry), chunk c -> sA + c kChunkA + ((rz WR + ry) 130 + p) 16.
        // The 2 x nrow x 130 copies are spread evenly over the block: thread tid takes
        // items tid, tid + 128, ... of the (row, position) sequence for both chunks,
        // advancing (row, p) by carries.
        {
            int row = tid / kTcHX, p = tid - row * kTcHX;
            constexpr int drow = kTcThreads / kTcHX, dp = kTcThreads % kTcHX;
            for (; row < nrow;) {
                const int rz = row / WR, ry = row - rz * WR;
                const int gz = z0 - 1 + rz, gy = y0 - 1 + ry, gx = x0 - 1 + p;
                const bool okp = gz >= 0 && gz < D && gy >= 0 && gy < H && gx >= 0 && gx < W;
                const bf16* src = okp ? x + (((int64_t)gz * H + gy) * W + gx) * cx + s * 16 : x;
                const unsigned sa = su32(sA + ((size_t)row * kTcHX + p) * 16);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(okp ? 16 : 0)
                             : "memory");
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa + kChunkA),
                             "l"(okp ? src + 8 : x), "r"(okp ? 16 : 0)
                             : "memory");
                p += dp;
                row += drow;
                if (p >= kTcHX) {
                    p -= kTcHX;
                    ++row;
                }
            }
        }
        // weights of the slice: [chunk][tap][o][8 channels]
        for (int e = tid; e < 2 * 27 * N; e += kTcThreads) {
            const int c = e / (27 * N), rem = e - c * 27 * N;   // rem = tap * N + o
            const unsigned sa = su32(sB + c * kChunkB + rem * 16);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa),
                         "l"(w + (int64_t)rem * ci + s * 16 + c * 8)
                         : "memory");
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // generic writes -> tensor-core reads
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            // descriptors of tap 0 / row 0; the start-address field counts 16-byte units, so a
            // (tap, row) operand is the base descriptor plus its offset in those units
            const uint64_t ad0 = smem_desc(a0, kChunkA, 128), bd0 = smem_desc(b0, kChunkB, 128);
#pragma unroll
            for (int t = 0; t < 27; ++t) {
                const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
                const uint64_t bd = bd0 + (uint64_t)(t * N);
#pragma unroll
                for (int r = 0; r < T; ++r) {
                    const uint64_t ad = ad0 + (uint64_t)((dz * WR + r + dy) * kTcHX + dx);
                    if (s == 0 && t == 0) {
                        asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 0;\n" ::"r"(
                                         tmem + (uint32_t)(r * N)),
                                     "l"(ad), "l"(bd), "r"(idesc_bf16(N))
                                     : "memory");
                    } else {
                        asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n" ::"r"(
                                         tmem + (uint32_t)(r * N)),
                                     "l"(ad), "l"(bd), "r"(idesc_bf16(N))
                                     : "memory");
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             su32(&mma_done))
                         : "memory");
        }
        // the next slice's copies overwrite the operands: every thread waits for these MMAs
        ok = !__syncthreads_or(!wait_bounded(&mma_done, par));
    }
    // every thread learns whether the accumulation finished
    const int failed = __syncthreads_or(!ok);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!failed) {
        conv_epilogue<N, T>(tmem, warp, lane, x0, y0, z0, H, W, bias, relu, y, cy, yoff);
    } else if (tid == 0) {
        atomicExch(&g_tc_fault, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(kCols) : "memory");
}


// ------------------------------------------------------------------ z-marching form
//
// Layers with 16 input channels (one slice) run in k_conv3_tcz: one CTA marches a
// (128-cell x T-row) column through zc consecutive output planes.  The slice's
// weights stay in shared memory for the whole column, and the input window is a
// ring of kZSlots planes ([chunk][slot][T+2 rows][130][8]): output plane z reads the
// slots of planes z-1, z and z+1, so each plane is copied once per column instead
// of three times.  The accumulators are double-buffered in TMEM: the MMAs of plane
// z run while the block drains plane z-1's accumulators (epilogue) and copies
// plane z+2 into the slot that plane z-2 left.  A plane's MMAs are those of
// k_conv3_tc (taps in the same order), so both kernels give the same bits.
constexpr int kZSlots = 4;

template <int N>
__host__ __device__ constexpr uint32_t tcz_chunk_a()
{
    return ((uint32_t)kZSlots * (tc_rows(N) + 2) * kTcHX * 16 + 127) / 128 * 128;
}

template <int N>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_conv3_tcz(const bf16* __restrict__ x, int cx, const bf16* __restrict__ w, int D, int H, int W,
                const float* __restrict__ bias, int relu, bf16* __restrict__ y, int cy, int yoff, int zc)
{
    static_assert(N % 16 == 0 && N >= 16 && N <= 64, "N: multiple of 16 up to 64 (two accumulator buffers)");
    constexpr int T = tc_rows(N);
    constexpr int WR = T + 2;
    constexpr uint32_t kChunkA = tcz_chunk_a<N>();
    constexpr uint32_t kChunkB = 27 * N * 16;
    static_assert(kChunkA % 128 == 0 && kChunkB % 128 == 0 && (kChunkA >> 4) < (1u << 14), "descriptor fields");
    constexpr int kCols = 2 * T * N <= 32 ? 32 : (2 * T * N <= 64 ? 64 : (2 * T * N <= 128 ? 128 : (2 * T * N <= 256 ? 256 : 512)));
    static_assert(2 * T * N <= 512, "two accumulator buffers fit in TMEM");
    static_assert(T <= kTcThreads / 32, "one issuing warp per row tile");
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* sA = smem;                                  // [2][kZSlots][T+2][130][8] bf16
    unsigned char* sB = smem + 2 * kChunkA;                    // [2][27][N][8] bf16
    __shared__ __align__(8) uint64_t mma_done[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = (W + kTcM - 1) / kTcM, tiles_y = (H + T - 1) / T;
    const int x0 = (blockIdx.x % tiles_x) * kTcM;
    const int y0 = ((blockIdx.x / tiles_x) % tiles_y) * T;
    const int zb = (int)(blockIdx.x / (tiles_x * tiles_y)) * zc;
    const int ze = min(D, zb + zc);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tmem_base)),
                     "n"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        // one arrival per issuing warp (warp r issues row tile r's MMAs)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(&mma_done[0])), "n"(T) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(&mma_done[1])), "n"(T) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t a0 = su32(sA), b0 = su32(sB);

    // plane gz of the window (rows y0-1 .. y0+T, columns x0-1 .. x0+128, both chunks)
    // into its ring slot, zeros outside the grid; 16-byte copies spread over the block
    auto copy_plane = [&](int gz) {
        const int slot = gz & (kZSlots - 1);                  // gz >= -1
        int row = tid / kTcHX, p = tid - row * kTcHX;
        constexpr int drow = kTcThreads / kTcHX, dp = kTcThreads % kTcHX;
        for (; row < WR;) {
            const int gy = y0 - 1 + row, gx = x0 - 1 + p;
            const bool okp = gz >= 0 && gz < D && gy >= 0 && gy < H && gx >= 0 && gx < W;
            const bf16* src = okp ? x + (((int64_t)gz * H + gy) * W + gx) * cx : x;
            const unsigned sa = su32(sA + ((size_t)(slot * WR + row) * kTcHX + p) * 16);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(okp ? 16 : 0)
                         : "memory");
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa + kChunkA), "l"(okp ? src + 8 : x),
                         "r"(okp ? 16 : 0)
                         : "memory");
            p += dp;
            row += drow;
            if (p >= kTcHX) {
                p -= kTcHX;
                ++row;
            }
        }
    };

    // weights of the one slice, then planes zb-1 .. zb+1
    for (int e = tid; e < 2 * 27 * N; e += kTcThreads) {
        const int c = e / (27 * N), rem = e - c * 27 * N;    // rem = tap * N + o
        const unsigned sa = su32(sB + c * kChunkB + rem * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(w + (int64_t)rem * 16 + c * 8)
                     : "memory");
    }
    copy_plane(zb - 1);
    copy_plane(zb);
    copy_plane(zb + 1);
    asm volatile("cp.async.commit_group;\n" ::: "memory");

    bool ok = true;
    for (int z = zb; z < ze; ++z) {
        const int k = z - zb;
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // generic writes -> tensor-core reads
        __syncthreads();
        // row tile r's 27 MMAs are issued by lane 0 of warp r, so the T row tiles'
        // small MMAs (M 128, N up to 64, K 16) are issued in parallel
        if (lane == 0 && warp < T) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint64_t ad0 = smem_desc(a0, kChunkA, 128), bd0 = smem_desc(b0, kChunkB, 128);
            const uint32_t acc = tmem + (uint32_t)((k & 1) * T * N);
            const int r = warp;
#pragma unroll
            for (int t = 0; t < 27; ++t) {
                const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
                const int slot = (z - 1 + dz) & (kZSlots - 1);
                const uint64_t bd = bd0 + (uint64_t)(t * N);
                {
                    const uint64_t ad = ad0 + (uint64_t)((slot * WR + r + dy) * kTcHX + dx);
                    if (t == 0) {
                        asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 0;\n" ::"r"(
                                         acc + (uint32_t)(r * N)),
                                     "l"(ad), "l"(bd), "r"(idesc_bf16(N))
                                     : "memory");
                    } else {
                        asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n" ::"r"(
                                         acc + (uint32_t)(r * N)),
                                     "l"(ad), "l"(bd), "r"(idesc_bf16(N))
                                     : "memory");
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             su32(&mma_done[k & 1]))
                         : "memory");
        }
        // once plane z-1's MMAs are done, the slot of plane z-2 takes plane z+2 and
        // plane z-1 leaves the other accumulator buffer, both while these MMAs run
        const int pb = (k - 1) & 1;
        if (k > 0) {
            ok = !__syncthreads_or(!wait_bounded(&mma_done[pb], (uint32_t)(((k - 1) >> 1) & 1)));
            if (!ok) break;
        }
        if (z + 2 <= ze) copy_plane(z + 2);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        if (k > 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            conv_epilogue<N, T>(tmem + (uint32_t)(pb * T * N), warp, lane, x0, y0, z - 1, H, W, bias, relu, y, cy,
                                yoff);
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        }
    }
    if (ok) {
        const int k = ze - 1 - zb, pb = k & 1;
        ok = !__syncthreads_or(!wait_bounded(&mma_done[pb], (uint32_t)((k >> 1) & 1)));
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            conv_epilogue<N, T>(tmem + (uint32_t)(pb * T * N), warp, lane, x0, y0, ze - 1, H, W, bias, relu, y, cy,
                                yoff);
        }
    }
    if (!ok && tid == 0) atomicExch(&g_tc_fault, 1);
    asm volatile("cp.async.wait_all;\n" ::: "memory");          // no copy in flight when the block ends
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(kCols) : "memory");
}

template <int N>
cudaError_t launch_z(const bf16* x, int cx, const bf16* w, int D, int H, int W, const float* bias, int relu,
                     bf16* y, int cy, int yoff, cudaStream_t s)
{
    constexpr int T = tc_rows(N);
    const size_t smem = 2 * (size_t)tcz_chunk_a<N>() + 2 * (size_t)(27 * N * 16);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_conv3_tcz<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // planes per column: about two waves of one CTA per SM, at least 2 planes a column
    const int64_t cols = (int64_t)((W + kTcM - 1) / kTcM) * ((H + T - 1) / T);
    const int64_t target = 2 * (int64_t)gmg::sm_count();
    int zc = (int)std::max<int64_t>(2, (D * cols + target - 1) / target);
    if (zc > D) zc = D;
    const int64_t blocks = cols * ((D + zc - 1) / zc);
    k_conv3_tcz<N><<<(unsigned)blocks, kTcThreads, smem, s>>>(x, cx, w, D, H, W, bias, relu, y, cy, yoff, zc);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch(const bf16* x, int cx, const bf16* w, int D, int H, int W, int ci, const float* bias, int relu,
                   bf16* y, int cy, int yoff, cudaStream_t s)
{
    constexpr int T = tc_rows(N);
    const size_t smem = 2 * (size_t)tc_chunk_a(T) + 2 * (size_t)(27 * N * 16);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_conv3_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t tiles = (int64_t)((W + kTcM - 1) / kTcM) * ((H + T - 1) / T) * D;
    k_conv3_tc<N><<<(unsigned)tiles, kTcThreads, smem, s>>>(x, cx, w, D, H, W, ci, bias, relu, y, cy, yoff);
    return cudaGetLastError();
}

}  // namespace

// Returns 0 on success, 1 if the shapes do not fit this kernel (the caller then
// uses the mma.sync kernel), 2 on a CUDA error.
int conv3_tc(int D, int H, int W, const void* x, int cx, int ci, const void* w, const float* bias, int co, int relu,
             void* y, int cy, int yoff, cudaStream_t s)
{
    if (ci % 16 || co % 16 || co > 128 || cx % 8 || cy % 8 || yoff % 8 || ((uintptr_t)x & 15) ||
        ((uintptr_t)w & 15) || ((uintptr_t)y & 15))
        return 1;
    const bf16* xb = static_cast<const bf16*>(x);
    const bf16* wb = static_cast<const bf16*>(w);
    bf16* yb = static_cast<bf16*>(y);
    cudaError_t e;
    if (ci == 16 && co <= 64 && co != 48) {   // one input slice: the z-marching form
        switch (co) {
        case 16: e = launch_z<16>(xb, cx, wb, D, H, W, bias, relu, yb, cy, yoff, s); break;
        case 32: e = launch_z<32>(xb, cx, wb, D, H, W, bias, relu, yb, cy, yoff, s); break;
        default: e = launch_z<64>(xb, cx, wb, D, H, W, bias, relu, yb, cy, yoff, s); break;
        }
        return e == cudaSuccess ? 0 : 2;
    }
    switch (co) {
    case 16: e = launch<16>(xb, cx, wb, D, H, W, ci, bias, relu, yb, cy, yoff, s); break;
    case 32: e = launch<32>(xb, cx, wb, D, H, W, ci, bias, relu, yb, cy, yoff, s); break;
    case 48: e = launch<48>(xb, cx, wb, D, H, W, ci, bias, relu, yb, cy, yoff, s); break;
    case 64: e = launch<64>(xb, cx, wb, D, H, W, ci, bias, relu, yb, cy, yoff, s); break;
    case 96: e = launch<96>(xb, cx, wb, D, H, W, ci, bias, relu, yb, cy, yoff, s); break;
    default: return 1;
    }
    return e == cudaSuccess ? 0 : 2;
}

int conv3_tc_fault()
{
    int f = 0;
    cudaMemcpyFromSymbol(&f, g_tc_fault, sizeof(int));
    return f;
}

}  // namespace gmgnet
