// Periodic lateral halo swap of one field (the doubly periodic boundary the
// scheme needs before each evaluation, Sec. 2.2).
#include "pw_device.cuh"
#include "pw_internal.h"

namespace pw {

// One thread per halo cell of levels 1..nz.  Every halo cell copies its
// periodic image directly (i' = 1 + (i-1) mod nx, likewise j), which equals
// the x-then-y two-pass swap including the corners.  Pure element copies in
// the storage type (E = 4 or 2 bytes).
template <typename E>
__global__ void fill_halo_kernel(const GridDev g, E* __restrict__ f) {
    const int h = g.halo;
    const long long wx = g.nx + 2 * h;
    const long long rows = 2LL * h * wx;              // halo rows, full width
    const long long cols = 2LL * h * g.ny;            // halo columns of interior rows
    const long long per_level = rows + cols;
    const long long total = per_level * g.nz;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k = 1 + (int)(idx / per_level);
        long long t = idx % per_level;
        int i, j;
        if (t < rows) {
            const int b = (int)(t / wx);
            i = 1 - h + (int)(t % wx);
            j = (b < h) ? (1 - h + b) : (g.ny + 1 + b - h);
        } else {
            t -= rows;
            const int b = (int)(t / g.ny);
            j = 1 + (int)(t % g.ny);
            i = (b < h) ? (1 - h + b) : (g.nx + 1 + b - h);
        }
        const int si = 1 + (((i - 1) % g.nx) + g.nx) % g.nx;
        const int sj = 1 + (((j - 1) % g.ny) + g.ny) % g.ny;
        const long long base = g.origin + (long long)k * g.pk;
        f[base + (long long)j * g.pj + i] = f[base + (long long)sj * g.pj + si];
    }
}

cudaError_t launch_fill_halo(pw_dtype_t dt, const GridDev& g, void* f, int num_sms, cudaStream_t s) {
    const long long per_level = 2LL * g.halo * (g.nx + 2 * g.halo) + 2LL * g.halo * g.ny;
    const long long total = per_level * g.nz;
    const int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
    if (blocks < 1) blocks = 1;
    if (dtype_size(dt) == 4)
        fill_halo_kernel<uint32_t><<<(unsigned)blocks, threads, 0, s>>>(g, (uint32_t*)f);
    else
        fill_halo_kernel<uint16_t><<<(unsigned)blocks, threads, 0, s>>>(g, (uint16_t*)f);
    return cudaGetLastError();
}

}  // namespace pw
