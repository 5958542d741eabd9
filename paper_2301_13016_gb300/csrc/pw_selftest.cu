// Self-test of the bounded-wait path: a kernel waits on an mbarrier phase that
// nothing completes, gives up after the limit, and records the timeout in the
// handle's status word exactly as the TMA kernels do.  No copy is in flight
// and the wait always ends, so the context stays usable.
#include "pw_device.cuh"
#include "pw_internal.h"

namespace pw {

__global__ void selftest_wait_kernel(uint64_t limit_ns, int* err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    bool ok = true;
    if (threadIdx.x == 0) ok = mbar_wait_bounded(&bar, 0, limit_ns);   // phase 0 never completes
    __syncthreads();
    if (threadIdx.x == 0 && !ok) report_error(err, DEV_TIMEOUT_TMA_WAIT);
}

cudaError_t launch_selftest_wait(uint64_t limit_ns, int* err, cudaStream_t s) {
    selftest_wait_kernel<<<1, 32, 0, s>>>(limit_ns, err);
    return cudaGetLastError();
}

}  // namespace pw
