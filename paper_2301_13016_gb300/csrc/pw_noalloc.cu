// pw_weighted_dot_noalloc: the weighted FP64 inner product of pw_weighted_dot
// with its scratch in a fixed, statically allocated device array instead of
// memory the handle allocates on first use.
//
// For callers that must not allocate device memory at call time: a host
// model that owns the whole device memory budget through its own allocator
// and forbids libraries from allocating, or a time loop where an allocation
// failure or the latency of cudaMalloc cannot be handled.  Such a caller
// creates its handle at start-up and can then run the conservation check
// (sum_k wk[k] sum_ij a*b) without any further cudaMalloc or cudaFree.
#include <mutex>

#include "pw_device.cuh"
#include "pw_internal.h"

namespace pw {

// Scratch layout (doubles): [0, 4*(kNoallocMaxBlocks+1)) per-block partials and
// the final result, then up to kNoallocMaxLevels level weights.
constexpr int kNoallocMaxBlocks = 1024;
constexpr int kNoallocMaxLevels = 4096;       // nz + 2 <= 4096
constexpr size_t kNoallocScratchDoubles = 4 * (size_t)(kNoallocMaxBlocks + 1) + kNoallocMaxLevels;

// 64.8 KB on every device that loads the library, held until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

constexpr int kMaxDevices = 64;
static double* g_scratch_addr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

// Device address of the static array on the current device, looked up once
// per device (host code cannot use the symbol's name as a device pointer).
static cudaError_t noalloc_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace pw

using namespace pw;

extern "C" pw_status_t pw_weighted_dot_noalloc(pw_handle_t h, const void* a, float sa, const void* b, float sb,
                                               const double* wk, int32_t k0, int32_t k1, double* out,
                                               pw_stream_t stream) {
    PW_RANGE("pw_weighted_dot_noalloc");
    pw_grid_t g;
    int num_sms = 0;
    if (!internal_handle_grid(h, &g, &num_sms)) return internal_fail(PW_ERR_ARG, "handle is NULL");
    if (!a || !b || !out) return internal_fail(PW_ERR_ARG, "a pointer is NULL");
    const void* dp[2] = {a, b};
    pw_status_t st = internal_check_device_ptrs(h, dp, 2);
    if (st != PW_OK) return st;
    // the static array's address is per device: the handle's GPU must be current
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != internal_handle_device(h))
        return internal_fail(PW_ERR_ARG, "pw_weighted_dot_noalloc: the handle's GPU %d is not the current device",
                             internal_handle_device(h));
    if (k0 < 1 || k1 > g.nz || k0 > k1) return internal_fail(PW_ERR_ARG, "need 1 <= k0 <= k1 <= nz");
    if (g.nz + 2 > kNoallocMaxLevels)
        return internal_fail(PW_ERR_UNSUPPORTED,
                                "pw_weighted_dot_noalloc: nz + 2 = %d exceeds the static scratch limit of %d levels "
                                "(use pw_weighted_dot)",
                                g.nz + 2, kNoallocMaxLevels);
    double* scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return internal_cuda_fail(e, "static scratch address lookup");
    int nblocks = norm_blocks(num_sms);
    if (nblocks > kNoallocMaxBlocks) nblocks = kNoallocMaxBlocks;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double* d_wk = nullptr;
    if (wk) {
        d_wk = scratch + 4 * (size_t)(kNoallocMaxBlocks + 1);
        e = cudaMemcpyAsync(d_wk, wk, (g.nz + 2) * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return internal_cuda_fail(e, "weight copy");
    }
    GridDev gd;
    gd.nx = g.nx;
    gd.ny = g.ny;
    gd.nz = g.nz;
    gd.halo = g.halo;
    gd.pj = g.pitch_j;
    gd.pk = g.pitch_k;
    gd.origin = g.origin;
    // Every block writes its own partial and the reduction writes the result,
    // so nothing in the array has to start at zero.
    e = launch_weighted_dot(g.dtype, gd, a, sa, b, sb, d_wk, k0, k1, scratch, nblocks, s);
    if (e != cudaSuccess) return internal_cuda_fail(e, "dot kernel launch");
    double r[4];
    e = cudaMemcpyAsync(r, scratch + 4 * (size_t)nblocks, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return internal_cuda_fail(e, "dot result copy");
    out[0] = r[2];
    return PW_OK;
}
