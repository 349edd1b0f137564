// Allocation-free box density: scola_box_density_noalloc.
//
// Some callers cannot allocate device memory when they need a density:
// services that account every byte through their own pool and forbid hidden
// allocations, and real-time loops that must not call the allocator.  For them this entry point computes the sCOLA box density
// (the same B^sCOLA cloud-in-cell deposit as scola_pm_force) with its scratch
// held in a fixed, file-scope device array instead of a context arena.
//
// The scratch is kNoAllocMaxCells 64-bit fixed-point counters (16 MiB).  Every
// GPU that loads this library holds that array until the process exits.  All
// calls share it and it keeps the last call's contents, so each call clears
// the part it uses first; calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it and must be serialised by the
// caller.  Host code cannot pass the array's name to a kernel (in host code it
// is a host-side stand-in, not a device address), so the device address is
// looked up with cudaGetSymbolAddress once per device, on the first call made
// with that device current.
#include <cmath>
#include <mutex>

#include "device_util.cuh"

namespace scola {
namespace {

constexpr long long kNoAllocMaxCells = 128LL * 128 * 128;

static __device__ __align__(256) unsigned long long g_noalloc_acc[kNoAllocMaxCells];

std::mutex g_noalloc_mutex;
constexpr int kMaxDevices = 64;
unsigned long long *g_noalloc_ptr[kMaxDevices] = {};

__global__ void __launch_bounds__(256)
k_noalloc_deposit(const float *__restrict__ s, int nsc, int ng, float q2u, float inv_dg,
                  unsigned long long *__restrict__ acc) {
    const long long n = (long long)nsc * nsc * nsc;
    const long long local = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (local >= n) return;
    int b[3];
    decode_local((int)local, nsc, b[0], b[1], b[2]);
    int i0[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float u = fmaf(s[a * n + local], inv_dg, fmaf((float)b[a], q2u, 0.5f * q2u - 0.5f));
        u = fminf(fmaxf(u, -2.0f), (float)ng + 1.0f);
        const float fl = floorf(u);
        i0[a] = (int)fl;
        f[a] = u - fl;
    }
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
        const int cx = i0[0] + dx;
        if ((unsigned)cx >= (unsigned)ng) continue;
        const float wx = dx ? f[0] : 1.0f - f[0];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int cy = i0[1] + dy;
            if ((unsigned)cy >= (unsigned)ng) continue;
            const float wxy = wx * (dy ? f[1] : 1.0f - f[1]);
#pragma unroll
            for (int dz = 0; dz < 2; ++dz) {
                const int cz = i0[2] + dz;
                if ((unsigned)cz >= (unsigned)ng) continue;
                const float w = wxy * (dz ? f[2] : 1.0f - f[2]);
                atomicAdd(acc + ((long long)cx * ng + cy) * ng + cz, weight_to_fixed(w));
            }
        }
    }
}

__global__ void k_noalloc_finish(const unsigned long long *__restrict__ acc, long long cells,
                                 float scale, float *__restrict__ delta) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < cells) delta[i] = fixed_to_float(acc[i]) * scale - 1.0f;
}

}  // namespace
}  // namespace scola

using namespace scola;

extern "C" scola_status scola_box_density_noalloc(const float *s_dev, int32_t nsc, int32_t ng,
                                                  double dq, float *delta_dev, void *stream) {
    if (!s_dev || !delta_dev) {
        set_error("scola_box_density_noalloc: NULL pointer");
        return SCOLA_ERR_INVALID_ARG;
    }
    if (nsc < 1 || ng < nsc || !(dq > 0)) {
        set_error("scola_box_density_noalloc: need nsc >= 1, ng >= nsc and dq > 0");
        return SCOLA_ERR_INVALID_ARG;
    }
    const long long cells = (long long)ng * ng * ng;
    if (cells > kNoAllocMaxCells) {
        set_error("scola_box_density_noalloc: ng^3 exceeds the fixed scratch of 128^3 cells");
        return SCOLA_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_error(std::string("scola_box_density_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return SCOLA_ERR_CUDA;
    }
    unsigned long long *acc = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_acc);
            if (e != cudaSuccess) {
                set_error(std::string("scola_box_density_noalloc: cudaGetSymbolAddress: ") +
                          cudaGetErrorString(e));
                return SCOLA_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = static_cast<unsigned long long *>(p);
        }
        acc = g_noalloc_ptr[dev];
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (size_t)cells, st);
    if (e == cudaSuccess) {
        const double dg = nsc * dq / ng;
        const long long n = (long long)nsc * nsc * nsc;
        k_noalloc_deposit<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            s_dev, nsc, ng, (float)((double)ng / nsc), (float)(1.0 / dg), acc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const float nbar_inv = (float)std::pow((double)ng / nsc, 3);
        k_noalloc_finish<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(
            acc, cells, nbar_inv * 2.3283064365386963e-10f, delta_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error(std::string("scola_box_density_noalloc: ") + cudaGetErrorString(e));
        return SCOLA_ERR_CUDA;
    }
    return SCOLA_OK;
}
