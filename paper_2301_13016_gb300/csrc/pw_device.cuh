// Device-side helpers shared by the PW kernels: storage types, PTX wrappers
// for mbarriers and TMA bulk-tensor copies (sm_100-family), bounded waits.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace pw {

// ---------------------------------------------------------------------------
// Storage types.  Arithmetic is always FP32; T is how fields sit in HBM.
template <typename T> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float to_f(float x) { return x; }
    static __device__ __forceinline__ float from_f(float x) { return x; }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
    static __device__ __forceinline__ __nv_bfloat16 from_f(float x) { return __float2bfloat16_rn(x); }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float to_f(__half x) { return __half2float(x); }
    static __device__ __forceinline__ __half from_f(float x) { return __float2half_rn(x); }
};

// Four consecutive elements <-> float[4].  p must be aligned to 4*sizeof(T).
__device__ __forceinline__ void load4(const float* p, float (&o)[4]) {
    float4 t = *reinterpret_cast<const float4*>(p);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void load4(const __nv_bfloat16* p, float (&o)[4]) {
    uint2 t = *reinterpret_cast<const uint2*>(p);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&t.x);
    __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&t.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    o[0] = fa.x; o[1] = fa.y; o[2] = fb.x; o[3] = fb.y;
}
__device__ __forceinline__ void load4(const __half* p, float (&o)[4]) {
    uint2 t = *reinterpret_cast<const uint2*>(p);
    __half2 a = *reinterpret_cast<__half2*>(&t.x);
    __half2 b = *reinterpret_cast<__half2*>(&t.y);
    float2 fa = __half22float2(a), fb = __half22float2(b);
    o[0] = fa.x; o[1] = fa.y; o[2] = fb.x; o[3] = fb.y;
}

__device__ __forceinline__ void store4(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(__nv_bfloat16* p, const float (&v)[4]) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
    __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 t;
    t.x = *reinterpret_cast<uint32_t*>(&a);
    t.y = *reinterpret_cast<uint32_t*>(&b);
    *reinterpret_cast<uint2*>(p) = t;
}
__device__ __forceinline__ void store4(__half* p, const float (&v)[4]) {
    __half2 a = __floats2half2_rn(v[0], v[1]);
    __half2 b = __floats2half2_rn(v[2], v[3]);
    uint2 t;
    t.x = *reinterpret_cast<uint32_t*>(&a);
    t.y = *reinterpret_cast<uint32_t*>(&b);
    *reinterpret_cast<uint2*>(p) = t;
}

// N consecutive elements (N = 4 or 8) <-> float[N]; p aligned to N*sizeof(T)
// (8 16-bit elements are one 16-byte access).
template <int N, typename T>
__device__ __forceinline__ void loadv(const T* p, float (&o)[N]) {
    if constexpr (N == 4) {
        load4(p, o);
    } else {
        static_assert(N == 8, "N must be 4 or 8");
        if constexpr (sizeof(T) == 4) {
            float a[4], b[4];
            load4(p, a);
            load4(p + 4, b);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                o[q] = a[q];
                o[4 + q] = b[q];
            }
        } else {
            const uint4 t = *reinterpret_cast<const uint4*>(p);
            const uint32_t w4[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2 f;
                if constexpr (sizeof(T) == 2 && std::is_same<T, __half>::value)
                    f = __half22float2(*reinterpret_cast<const __half2*>(&w4[q]));
                else
                    f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w4[q]));
                o[2 * q] = f.x;
                o[2 * q + 1] = f.y;
            }
        }
    }
}

template <int N, typename T>
__device__ __forceinline__ void storev(T* p, const float (&v)[N]) {
    if constexpr (N == 4) {
        store4(p, v);
    } else {
        static_assert(N == 8, "N must be 4 or 8");
        if constexpr (sizeof(T) == 4) {
            const float a[4] = {v[0], v[1], v[2], v[3]}, b[4] = {v[4], v[5], v[6], v[7]};
            store4(p, a);
            store4(p + 4, b);
        } else {
            uint32_t w4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if constexpr (std::is_same<T, __half>::value) {
                    __half2 h = __floats2half2_rn(v[2 * q], v[2 * q + 1]);
                    w4[q] = *reinterpret_cast<uint32_t*>(&h);
                } else {
                    __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                    w4[q] = *reinterpret_cast<uint32_t*>(&h);
                }
            }
            *reinterpret_cast<uint4*>(p) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
    }
}

// ---------------------------------------------------------------------------
// Error flag values written by kernels into the handle's device status word.
enum : int {
    DEV_OK = 0,
    DEV_TIMEOUT_TMA_WAIT = 1,   // an mbarrier wait for a TMA copy ran out of time
    DEV_TIMEOUT_QUEUE = 2,      // a work-queue wait ran out of time
    DEV_OOB_STORE = 3,          // debug bounds build: a store outside the field's cells was skipped
};

// Wait limit for any spin in these kernels (nanoseconds of %globaltimer).
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s
constexpr uint64_t kDrainLimitNs = 200000000ull;   // 0.2 s

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory loads at a 32-bit shared address (ordered like any memory
// access: after the mbarrier wait that made the data visible).
__device__ __forceinline__ uint4 lds_u128(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(a)
                 : "memory");
    return v;
}
__device__ __forceinline__ uint2 lds_u64(uint32_t a) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Add to a shared-memory counter with acquire-release ordering at CTA scope;
// returns the previous value.
__device__ __forceinline__ uint32_t atom_add_acq_rel_cta(uint32_t* p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;"
                 : "=r"(old)
                 : "r"(smem_u32(p)), "r"(v)
                 : "memory");
    return old;
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// try_wait that lets the thread sleep until the phase completes or hint_ns
// passes, so waiting warps do not spend issue slots polling.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return done != 0;
}

constexpr uint32_t kSuspendHintNs = 1000000u;   // 1 ms per sleep, well below the wait limit

// Bounded wait on one mbarrier phase.  Returns false if the limit passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait_sleep(bar, parity, kSuspendHintNs)) {
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// 3D tiled TMA load of one box into shared memory, completing on `bar`.
// x must be a multiple of 16 bytes / sizeof(element); y and z are free.
__device__ __forceinline__ void tma_load_3d(void* smem_dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Raise a kernel's dynamic shared-memory limit once per (kernel, device)
// (a host-side attribute call, kept out of the per-launch path).
cudaError_t set_smem_attr_once_impl(const void* kern, int bytes);
template <typename K>
__host__ inline cudaError_t set_smem_attr_once(K kern, int bytes) {
    return set_smem_attr_once_impl(reinterpret_cast<const void*>(kern), bytes);
}

__device__ __forceinline__ void report_error(int* flag, int code) {
    if (flag) atomicCAS(flag, DEV_OK, code);
}

}  // namespace pw
