// gmg_dense.cu -- the coarsest level's pseudo-inverse for the dense coarse solve.
//
// With coarse_mode 1 the V-cycle (paper Sec. 3) solves its coarsest level
// exactly, in the least-squares minimum-norm sense: p = A^+ b, with A^+ the
// Moore-Penrose pseudo-inverse of the coarsest operator (Sec. 3.2 ties the
// coarsest level's treatment to how well low frequencies decay).  A^+ is built
// once per gmg_set_coeffs on the device, in FP64:
//
//   L = -A is a weighted graph Laplacian (symmetric, positive semi-definite),
//   whose null space is spanned by the indicator vectors 1_C of the connected
//   components C of the cells (faces with beta > 0 connect; a cell with no
//   open face is its own component).  With P = sum_C 1_C 1_C^T / |C| (the
//   orthogonal projector onto that null space), M = L + P is symmetric
//   positive definite and M^-1 = L^+ + P, hence A^+ = -L^+ = -(M^-1 - P).
//
// Steps: k_dense_assemble (one CTA) builds M row by row and labels the
// components by min-label propagation; M^-1 by Gauss-Jordan elimination
// without pivoting (M is SPD), one grid launch per pivot reading one FP64
// buffer and writing the other; k_dense_finish writes A^+ in FP32.  The cost
// is about n^3 FP64 multiply-adds for n coarsest cells (n <= kDenseMaxCells).
#include "gmg_internal.h"
#include "gmg_device.cuh"

namespace gmg {
namespace {

using namespace dev;

constexpr int kAsmThreads = 1024;

// neighbour of cell (x, y, z) along axis d in direction s, or -1 across a wall
__device__ int dense_nbr(const Geo& g, int x, int y, int z, int d, int s)
{
    int c[3] = {x, y, z};
    c[d] += s;
    if (!wrapc(c[d], g.n[d], g.per[d])) return -1;
    return (c[2] * g.n[1] + c[1]) * g.n[0] + c[0];
}

// M = L + P (row-major n x n FP64), component labels and sizes
__global__ void __launch_bounds__(kAsmThreads) k_dense_assemble(Geo g, const float* __restrict__ bx,
                                                                 const float* __restrict__ by,
                                                                 const float* __restrict__ bz, double* M,
                                                                 int* label_out, int* size_out)
{
    __shared__ int lab[kDenseMaxCells];
    __shared__ int cnt[kDenseMaxCells];
    const int n = g.n[0] * g.n[1] * g.n[2];
    const float* beta[3] = {bx, by, bz};
    // rows of L: row i gets +f on its diagonal and -f at the neighbour across each open face
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double* row = M + (int64_t)i * n;
        for (int j = 0; j < n; ++j) row[j] = 0.0;
        const int x = i % g.n[0], y = (i / g.n[0]) % g.n[1], z = i / (g.n[0] * g.n[1]);
        const int c[3] = {x, y, z};
        for (int d = 0; d < 3; ++d) {
            for (int s = -1; s <= 1; s += 2) {
                const int j = dense_nbr(g, x, y, z, d, s);
                if (j < 0) continue;
                // lower face of this cell, or lower face of the upper neighbour
                const float f = s < 0 ? ((c[d] == 0 && !g.per[d]) ? 0.f : beta[d][i]) : beta[d][j];
                row[i] += (double)f;
                row[j] -= (double)f;
            }
        }
        lab[i] = i;
        cnt[i] = 0;
    }
    __syncthreads();
    // components: every cell takes the smallest label among itself and its open
    // neighbours until nothing changes (at most n rounds)
    for (int round = 0; round < n; ++round) {
        int changed = 0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const double* row = M + (int64_t)i * n;
            const int x = i % g.n[0], y = (i / g.n[0]) % g.n[1], z = i / (g.n[0] * g.n[1]);
            int m = lab[i];
            for (int d = 0; d < 3; ++d)
                for (int s = -1; s <= 1; s += 2) {
                    const int j = dense_nbr(g, x, y, z, d, s);
                    if (j >= 0 && row[j] < 0.0) m = min(m, lab[j]);
                }
            if (m < lab[i]) {
                lab[i] = m;   // monotone: racing reads of a neighbour's label only delay convergence
                changed = 1;
            }
        }
        if (!__syncthreads_or(changed)) break;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&cnt[lab[i]], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        label_out[i] = lab[i];
        size_out[i] = cnt[lab[i]];
    }
    __syncthreads();
    // + P: 1 / |C| where both cells lie in component C
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
        const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
        if (lab[i] == lab[j]) M[e] += 1.0 / (double)cnt[lab[i]];
    }
}

// one Gauss-Jordan step at pivot k, in place in the sense of the classical
// inversion (column k ends as the inverse's column): B = step(A)
__global__ void k_gj_pivot(const double* __restrict__ A, double* __restrict__ B, int n, int k)
{
    const double piv = 1.0 / A[(int64_t)k * n + k];
    const int64_t total = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
        const double rk = (j == k ? 1.0 : A[(int64_t)k * n + j]) * piv;   // scaled pivot row
        if (i == k) {
            B[e] = rk;
        } else {
            const double f = A[(int64_t)i * n + k];
            B[e] = (j == k ? 0.0 : A[e]) - f * rk;
        }
    }
}

// A^+ = -(M^-1 - P), FP32
__global__ void k_dense_finish(const double* __restrict__ Minv, const int* __restrict__ label,
                               const int* __restrict__ size, int n, float* __restrict__ pinv)
{
    const int64_t total = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
        const double p = label[i] == label[j] ? 1.0 / (double)size[i] : 0.0;
        pinv[e] = (float)(-(Minv[e] - p));
    }
}

}  // namespace

cudaError_t build_dense_pinv(const Geo& g, const float* bx, const float* by, const float* bz, float* pinv,
                             cudaStream_t s)
{
    const int n = g.n[0] * g.n[1] * g.n[2];
    if (n < 1 || n > kDenseMaxCells) return cudaErrorInvalidValue;
    double* A = nullptr;
    double* B = nullptr;
    int* lab = nullptr;
    cudaError_t e = cudaMalloc(&A, sizeof(double) * (size_t)n * n);
    if (e == cudaSuccess) e = cudaMalloc(&B, sizeof(double) * (size_t)n * n);
    if (e == cudaSuccess) e = cudaMalloc(&lab, sizeof(int) * 2 * (size_t)n);
    if (e == cudaSuccess) {
        k_dense_assemble<<<1, kAsmThreads, 0, s>>>(g, bx, by, bz, A, lab, lab + n);
        e = cudaGetLastError();
    }
    const int64_t total = (int64_t)n * n;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count() * 8);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        k_gj_pivot<<<grid, 256, 0, s>>>(A, B, n, k);
        e = cudaGetLastError();
        double* t = A;
        A = B;
        B = t;
    }
    if (e == cudaSuccess) {
        k_dense_finish<<<grid, 256, 0, s>>>(A, lab, lab + n, n, pinv);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(A);
    cudaFree(B);
    cudaFree(lab);
    return e;
}

}  // namespace gmg
