// gmg_tma.cu -- host-side encoding of the tensor maps that the pipelined sweep
// and residual kernels use to copy whole tile planes with the tensor memory
// accelerator (one instruction per plane instead of one 16-byte copy per thread).
#include "gmg_internal.h"

#include <cudaTypedefs.h>
#include <cstring>
#include <mutex>

namespace gmg {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool encode_one(CUtensorMap* m, const float* base, const Geo& g)
{
    std::memset(m, 0, sizeof(*m));
    if (!base) return true;                      // unused role: left zero
    auto fn = encoder();
    if (!fn) return false;
    const cuuint64_t dim[3] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
    const cuuint64_t stride[2] = {(cuuint64_t)g.n[0] * sizeof(float), (cuuint64_t)g.n[0] * g.n[1] * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)(kSweepTX + 8), (cuuint32_t)(kSweepTY + 4), 1};
    const cuuint32_t estride[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dim, stride, box, estride,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool aligned(const void* p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

bool encode_tma_planes(TmaPlanes* out, const Geo& g, const float* const p[3], const float* b, const float* bx,
                       const float* by, const float* bz)
{
    if (g.n[0] % 4) return false;
    const float* all[7] = {p[0], p[1], p[2], b, bx, by, bz};
    for (const float* a : all)
        if (a && !aligned(a)) return false;
    if (!b || !bx || !by || !bz) return false;
    bool ok = true;
    for (int r = 0; r < 3; ++r) ok = ok && encode_one(&out->p[r], p[r], g);
    ok = ok && encode_one(&out->b, b, g) && encode_one(&out->x, bx, g) && encode_one(&out->y, by, g) &&
         encode_one(&out->z, bz, g);
    return ok;
}

}  // namespace gmg
