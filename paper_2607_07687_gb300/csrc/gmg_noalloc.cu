// gmg_noalloc.cu -- residual norm that allocates nothing.
//
// gmg_op_residual_norm keeps its per-tile partial sums in a device buffer the
// library allocates on first use.  Some callers cannot let a library call
// cudaMalloc: real-time loops that must never meet the device-wide
// synchronisation cudaMalloc / cudaFree can cause, and programs that run under
// a device-memory budget fixed before they start.  For them,
// gmg_op_residual_norm_noalloc computes the same quantity with its scratch in
// a fixed-size array that is part of the library image: every GPU that loads
// the library holds it (512 KB of partial sums plus one double) until the
// process exits, and no call allocates or frees anything.
//
// In host code the array's name is only a host-side stand-in, not a device
// address; the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the entry point's first
// call there.
#include "gmg_internal.h"
#include "../../include/gmg.h"

#include <mutex>
#include <string>
#include <vector>

namespace {

constexpr int kNoAllocMaxTiles = 1 << 16;   // partial sums the static scratch holds

// Shared by every call on a device; each call writes every entry it reads
// (one partial per tile, then the total), so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxTiles];
static __device__ __align__(256) double g_noalloc_total[1];

struct DeviceScratch {
    int device;
    double* partials;   // device address of g_noalloc_partials on that device
    double* total;      // device address of g_noalloc_total on that device
};

std::mutex g_setup_mutex;
std::vector<DeviceScratch> g_setups;

// Device addresses of the static scratch on the current device (looked up on
// the first call per device).  Returns a CUDA error, or cudaSuccess.
cudaError_t scratch_addresses(double** partials, double** total)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    for (const DeviceScratch& s : g_setups)
        if (s.device == dev) {
            *partials = s.partials;
            *total = s.total;
            return cudaSuccess;
        }
    DeviceScratch s{dev, nullptr, nullptr};
    e = cudaGetSymbolAddress((void**)&s.partials, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress((void**)&s.total, g_noalloc_total);
    if (e != cudaSuccess) return e;
    g_setups.push_back(s);
    *partials = s.partials;
    *total = s.total;
    return cudaSuccess;
}

int ceil_div_i(int a, int b) { return (a + b - 1) / b; }

}  // namespace

extern "C" int gmg_op_residual_norm_noalloc(int nx, int ny, int nz, const int* periodic,
                                            const float* bx, const float* by, const float* bz,
                                            const float* b, const float* p, double* rr,
                                            void* stream)
{
    using namespace gmg;
    std::string geo_msg;
    if (validate_geometry(nx, ny, nz, periodic, geo_msg) != GMG_OK) {
        set_api_error(("gmg_op_residual_norm_noalloc: " + geo_msg).c_str());
        return GMG_ERR_ARG;
    }
    if (!bx || !by || !bz || !b || !p || !rr) {
        set_api_error("gmg_op_residual_norm_noalloc: null pointer");
        return GMG_ERR_ARG;
    }
    const int tx = ceil_div_i(nx, kResTX), ty = ceil_div_i(ny, kResTY), tz = ceil_div_i(nz, kResTZ);
    const long long tiles = (long long)tx * ty * tz;
    if (tiles > kNoAllocMaxTiles) {
        std::string msg = "gmg_op_residual_norm_noalloc: the grid needs " + std::to_string(tiles) +
                          " partial sums but the static scratch holds " + std::to_string(kNoAllocMaxTiles) +
                          " (one per " + std::to_string(kResTX) + "x" + std::to_string(kResTY) + "x" +
                          std::to_string(kResTZ) + " tile, about 16.7 M cells); use gmg_op_residual_norm";
        set_api_error(msg.c_str());
        return GMG_ERR_ARG;
    }
    double* partials = nullptr;
    double* total = nullptr;
    cudaError_t e = scratch_addresses(&partials, &total);
    if (e != cudaSuccess) {
        set_api_error(cudaGetErrorString(e));
        return GMG_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ResTask<float> t{};
    t.g.n[0] = nx;
    t.g.n[1] = ny;
    t.g.n[2] = nz;
    for (int d = 0; d < 3; ++d) t.g.per[d] = periodic ? (periodic[d] != 0) : 0;
    t.bx = bx;
    t.by = by;
    t.bz = bz;
    t.b = b;
    t.buf[0] = t.buf[1] = t.buf[2] = const_cast<float*>(p);
    t.rot = nullptr;
    t.role = 0;
    t.bc = nullptr;
    t.cf[0] = t.cf[1] = t.cf[2] = 1;
    t.tiles_x = tx;
    t.tiles_y = ty;
    t.tiles_z = tz;
    t.partials = partials;
    t.ctl = nullptr;
    TaskList<ResTask<float>> tl{};
    tl.ntasks = 1;
    tl.total = (int)tiles;
    tl.single = t;
    e = launch_residual(tl, persistent_grid(tiles), s);
    if (e == cudaSuccess) e = launch_sum_partials(partials, (int)tiles, total, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rr, total, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_api_error(cudaGetErrorString(e));
        return GMG_ERR_CUDA;
    }
    return GMG_OK;
}
