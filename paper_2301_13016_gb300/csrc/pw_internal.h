// Internal (non-ABI) declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pw.h"

// NVTX ranges around the library's launching entry points, so a timeline
// tool shows each C-ABI call by name.  NVTX v3 is header-only: with no tool
// attached a range costs two calls of empty functions.  Build with
// -DPW_NVTX=0 to compile them out.
#ifndef PW_NVTX
#define PW_NVTX 1
#endif
#if PW_NVTX && __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define PW_HAVE_NVTX 1
#else
#define PW_HAVE_NVTX 0
#endif

namespace pw {

struct NvtxRange {
#if PW_HAVE_NVTX
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
#else
    explicit NvtxRange(const char*) {}
#endif
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define PW_RANGE(name) const ::pw::NvtxRange pw_nvtx_range_(name)

// Field geometry as the kernels see it: element (k, j, i) of a field sits at
// ptr[origin + k*pk + j*pj + i], with i in [1-halo, nx+halo], j likewise,
// k in [0, nz+1].
struct GridDev {
    int nx, ny, nz, halo;
    long long pj, pk, origin;
};

// Cells o .. o+n-1 of a field (element offsets from the field pointer, one
// row) lie on levels 1..nz and inside the interior (interior_only) or the
// interior and its lateral halo, never in row padding or beyond: the check of
// the debug bounds build, on the host and the device alike.
#ifndef PW_DEBUG_BOUNDS
#define PW_DEBUG_BOUNDS 0
#endif
__host__ __device__ inline bool layout_cells_ok(const GridDev& g, long long o, int n, bool interior_only) {
    const int h = g.halo;
    const long long rel = o - g.origin - (long long)(1 - h) * g.pj - (1 - h);   // from (k, 1-h, 1-h)
    if (rel < 0 || n < 1) return false;
    const long long k = rel / g.pk, r = rel - k * g.pk;
    const long long jj = r / g.pj, ii = r - jj * g.pj;
    const long long j = jj + 1 - h, i0 = ii + 1 - h, i1 = i0 + n - 1;
    if (k < 1 || k > g.nz) return false;
    if (interior_only) return j >= 1 && j <= g.ny && i0 >= 1 && i1 <= g.nx;
    return j <= g.ny + h && i1 <= g.nx + h;
}

// Per-field storage scales: physical = stored * in[f]; stored = physical * out[f].
struct Scales {
    float in[3];
    float out[3];
};

// Scheme coefficients on the device: tz holds tzc1, tzc2, tzd1, tzd2, each
// nz+2 floats, back to back.
struct CoefDev {
    float tcx, tcy;
    const float* tz;
};

// The scheme's coefficients with the storage scales folded in, per output
// field (su, sv, sw).  Every term of the scheme is c * a * (b + d) with b and d
// of one field, so on stored values (physical = stored * in) the term is
// (c * in_a * in_b * out) * a~ * (b~ + d~) with out the output's scale: the
// x terms pair u values, the y terms v values, the z terms w values, hence
//   kx[f] = tcx * in_u * a_f,  ky[f] = tcy * in_v * a_f,  kz[f] = in_w * a_f,
// a_f = in_f * out_f (kz multiplies the per-level tz coefficients).  With
// power-of-two scales this is exact: the k-march then computes on stored
// values directly, bit for bit what it computed on dequantised ones.
struct FoldedCoef {
    float kx[3], ky[3], kz[3];
    const float* tz;   // tzc1 | tzc2 | tzd1 | tzd2, nz+2 each
};

__host__ __device__ inline FoldedCoef fold_coef(const CoefDev& cf, const Scales& sc) {
    FoldedCoef k;
    for (int f = 0; f < 3; ++f) {
        const float a = sc.in[f] * sc.out[f];
        k.kx[f] = cf.tcx * sc.in[0] * a;
        k.ky[f] = cf.tcy * sc.in[1] * a;
        k.kz[f] = sc.in[2] * a;
    }
    k.tz = cf.tz;
    return k;
}

// Launch shape of the TMA k-march kernel.
struct TmaConfig {
    int lx;      // lanes per row: 32 (tile 128 columns wide) or 16 (64 columns)
    int ty;      // interior rows per CTA
    int stages;  // planes resident or in flight per CTA
    int nseg;    // k segments the levels are split into
    int nc = 4;         // cells per thread along x (8: 16-bit storage only)
    int seg0 = 0;       // first segment to launch
    int seg_count = 0;  // segments to launch (0 = all nseg)
    int rp = 1;         // rows per thread: 1, or 2 (packed FP32x2 arithmetic on row pairs)
    int xp = 0;         // 1: one row per thread, its nc cells packed as FP32x2 pairs (cell q, cell q + nc/2)
};

// Launch shape of the two-step (temporal blocking) k-march kernel.
struct Step2Config {
    int ty;      // q1 rows per CTA (q2 rows: ty - 2)
    int stages;  // q0 planes resident or in flight per CTA
    int nseg;    // k segments
    int minb;    // register budget: 1 or 2 resident CTAs per SM
};

size_t dtype_size(pw_dtype_t t);

cudaError_t launch_tend_generic(pw_dtype_t dt, const GridDev& g, const void* u, const void* v, const void* w,
                                void* su, void* sv, void* sw, const Scales& sc, bool scaled,
                                const CoefDev& cf, int num_sms, cudaStream_t s);

// Box width (elements along x) of one TMA load for this dtype and tile width.
int tma_box_width(pw_dtype_t dt, int lx, int nc = 4);
// True if an instantiation exists for (dtype, ty, stages).
bool tma_config_supported(pw_dtype_t dt, const TmaConfig& c);
size_t tma_smem_bytes(pw_dtype_t dt, const TmaConfig& c);

cudaError_t launch_tend_tma(pw_dtype_t dt, const GridDev& g, int ox, const CUtensorMap* maps /*u,v,w*/,
                            void* su, void* sv, void* sw, const Scales& sc, const CoefDev& cf,
                            int* err, const TmaConfig& c, cudaStream_t s);

// Forward-Euler step kernels: (nu, nv, nw) = (u, v, w) + tstep * s(u, v, w),
// interior levels 1..nz plus the periodic images of boundary cells in the halo.
cudaError_t launch_step_generic(pw_dtype_t dt, const GridDev& g, const void* u, const void* v, const void* w,
                                void* nu, void* nv, void* nw, const Scales& sc, bool scaled, const CoefDev& cf,
                                float tstep, int num_sms, cudaStream_t s);
cudaError_t launch_step_tma(pw_dtype_t dt, const GridDev& g, int ox, const CUtensorMap* maps, void* nu, void* nv,
                            void* nw, const Scales& sc, const CoefDev& cf, float tstep, int* err,
                            const TmaConfig& c, cudaStream_t s);

// Two forward-Euler steps per pass (temporal blocking): (nu, nv, nw) = q2
// with q1 = q + tstep*s(q), q2 = q1 + tstep*s(q1); needs a lateral halo of
// at least 2 and maps encoded with box step2_box_width() x (ty + 2).
cudaError_t launch_step2_tma(pw_dtype_t dt, const GridDev& g, int ox, const CUtensorMap* maps, void* nu, void* nv,
                             void* nw, const Scales& sc, const CoefDev& cf, float tstep, int* err,
                             const Step2Config& c, cudaStream_t s);
bool step2_config_supported(const Step2Config& c);
int step2_box_width();
int step2_tile_cols();
int step2_blocks_per_sm(pw_dtype_t dt, const Step2Config& c);

// Adjoint gather kernel (FP32 fields): g = [g | l | 0] + alpha * J(u,v,w)^T l.
cudaError_t launch_adjoint(const GridDev& g, const float* u, const float* v, const float* w, const float* lu,
                           const float* lv, const float* lw, float* gu, float* gv, float* gw, float alpha,
                           int accumulate, int add_lambda, int periodic, const CoefDev& cf, int num_sms,
                           cudaStream_t s);

// Launch shape of the TMA adjoint: na cells per thread along x (a CTA covers
// 32*na columns), ty rows per CTA, stages ring slots.
struct AdjConfig {
    int na = 0, ty = 0, stages = 0, nseg = 0;
};
// TMA k-march adjoint (periodic mode, FP32): maps6 = u, v, w, lsu, lsv, lsw
// encoded for 32 lanes of c.na cells and c.ty rows; halos must be periodic.
cudaError_t launch_adjoint_tma(const GridDev& g, int ox, const CUtensorMap* maps6, float* gu, float* gv, float* gw,
                               float alpha, int accumulate, int add_lambda, const CoefDev& cf, int nseg, int* err,
                               const AdjConfig& c, cudaStream_t s);
bool adjoint_config_supported(const AdjConfig& c);
AdjConfig adjoint_default_config();
int adjoint_blocks_per_sm(const AdjConfig& c);

// Blocks of the TMA kernel resident per SM for a config (0 if it cannot launch).
int tma_blocks_per_sm(pw_dtype_t dt, const TmaConfig& c);

cudaError_t launch_fill_halo(pw_dtype_t dt, const GridDev& g, void* f, int num_sms, cudaStream_t s);

// Bounded-wait self-test (see pw_selftest_wait_timeout).
cudaError_t launch_selftest_wait(uint64_t limit_ns, int* err, cudaStream_t s);

// FP64 validation reductions.  scratch holds 4*(nblocks+1) doubles; the
// result lands in scratch[4*nblocks .. 4*nblocks+3].
int norm_blocks(int num_sms);
cudaError_t launch_error_norms(pw_dtype_t dt, const GridDev& g, const void* t, float scale, const double* ref,
                               int k0, int k1, double* scratch, int nblocks, cudaStream_t s);
cudaError_t launch_weighted_dot(pw_dtype_t dt, const GridDev& g, const void* a, float sa, const void* b, float sb,
                                const double* wk, int k0, int k1, double* scratch, int nblocks, cudaStream_t s);

// Error reporting and handle access for translation units other than
// pw_api.cu (set the thread-local message pw_last_error returns).
pw_status_t internal_fail(pw_status_t s, const char* fmt, ...);

// Host-side failure injection (pw_inject_failures): true when this operation
// of `kind` is to fail (one pending failure consumed).
enum { INJECT_ALLOC = 0, INJECT_TENSOR_MAP = 1, INJECT_KINDS = 2 };
bool inject_failure(int kind);
// cudaMalloc / cudaMallocHost, failing with cudaErrorMemoryAllocation (and a
// null pointer) when an allocation failure is injected.
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
    if (inject_failure(INJECT_ALLOC)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}
template <class T>
inline cudaError_t host_malloc_pinned(T** p, size_t bytes) {
    if (inject_failure(INJECT_ALLOC)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}
pw_status_t internal_cuda_fail(cudaError_t e, const char* what);
bool internal_handle_grid(pw_handle_t h, pw_grid_t* g, int* num_sms);
// The GPU a handle was created on.
int internal_handle_device(pw_handle_t h);
// Every pointer in ps[0..n) is device memory of the handle's GPU (the same
// check, and the same per-handle cache of checked pointers, as the field
// arguments of every other entry point).
pw_status_t internal_check_device_ptrs(pw_handle_t h, const void* const* ps, int n);

// Layout checks and TMA descriptors shared by the single-grid and batched paths.
pw_status_t validate_grid(const pw_grid_t* g);
bool tma_layout_ok(const pw_grid_t& g, int* ox_out, const char** why);
bool aligned16(const void* p);
// p is device (or managed) memory of the given GPU.
bool is_device_ptr(const void* p, int device);
// L2 promotion of the TMA loads (build knobs; CUtensorMapL2promotion: 0 none,
// 1 64 B, 2 128 B, 3 256 B). The single-grid maps promote to 256 B. The batch
// maps promote to 64 B: its boxes are narrow (64 or 128 columns plus halo
// granules), and 256-byte promotion fetched the sectors beyond each box row
// (512-grid batch, 32 grids: BF16 reads 1.44 -> 1.09 GB, FP32 1.86 -> 1.65 GB,
// the kernel time unchanged; the single grid runs alike at 0, 1 and 3).
#ifndef PW_TMA_L2_PROMOTION
#define PW_TMA_L2_PROMOTION 3
#endif
#ifndef PW_BATCH_L2_PROMOTION
#define PW_BATCH_L2_PROMOTION 1
#endif
pw_status_t encode_tensor_map(const pw_grid_t& g, const void* ptr, int lx, int ty, CUtensorMap* out, int nc = 4,
                              int l2_promotion = PW_TMA_L2_PROMOTION);
// Same with an explicit box (box_w elements along x, box_h rows).
pw_status_t encode_tensor_map_box(const pw_grid_t& g, const void* ptr, int box_w, int box_h, CUtensorMap* out,
                                  int l2_promotion = PW_TMA_L2_PROMOTION);

}  // namespace pw
