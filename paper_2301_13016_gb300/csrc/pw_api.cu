// C ABI of the PW library: handles, argument validation, TMA descriptors,
// kernel selection and launch.  See include/pw.h for the contract.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "pw_device.cuh"
#include "pw_internal.h"

namespace pw {

size_t dtype_size(pw_dtype_t t) { return t == PW_F32 ? 4 : 2; }

static thread_local std::string g_err;

static pw_status_t fail(pw_status_t s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

static pw_status_t cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? PW_ERR_OOM : PW_ERR_CUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

#define PW_CUDA(call, what)                          \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
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

struct MapCacheEntry {
    const void* ptr = nullptr;
    int box_w = 0, box_h = 0;
    CUtensorMap map;
};

}  // namespace pw

using namespace pw;

struct pw_handle_s {
    pw_grid_t grid;
    int device = 0;
    int num_sms = 0;
    float tcx = 0.f, tcy = 0.f;
    float* d_tz = nullptr;      // tzc1 | tzc2 | tzd1 | tzd2, nz+2 each
    int* d_err = nullptr;       // device status word (bounded-wait timeouts)
    int kernel_kind = 0;        // 0 auto, 1 generic, 2 TMA
    int last_kernel = 0;
    // user overrides: every field 0 = automatic (nc and rp too, whose struct
    // defaults are the values a launch uses)
    TmaConfig tma_user{0, 0, 0, 0, 0, 0, 0, 0};
    TmaConfig tma_auto[2] = {{0, 0, 0, 0}, {0, 0, 0, 0}};   // per mode (source terms, steps); ty == 0: not chosen yet
    int steps_per_pass = 0;           // pw_step temporal blocking: 0 auto (= 1), 1, 2
    Step2Config step2_user{0, 0, 0, 0};
    Step2Config step2_auto{0, 0, 0, 0};   // ty == 0: not chosen yet
    AdjConfig adj_user{0, 0, 0, 0};       // TMA adjoint shape; 0 = automatic
    AdjConfig adj_auto{0, 0, 0, 0};       // the shape in use; na == 0: not chosen yet
    MapCacheEntry maps[8];
    int map_next = 0;   // round-robin replacement
    // field pointers already found to be device memory of this handle's GPU
    static constexpr int kDevCache = 32;
    const void* dev_ok[kDevCache] = {};
    int dev_next = 0;
    // pw_tendencies_host staging and its copy / compute pipeline
    void* d_stage[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaStream_t hs[3] = {nullptr, nullptr, nullptr};   // copy in, compute, copy out
    static constexpr int kMaxChunks = 32;
    cudaEvent_t ev_in[kMaxChunks] = {}, ev_comp[kMaxChunks] = {}, ev_out[kMaxChunks] = {};
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;
    bool host_prev_plain = false;   // the last host-path call took the one-launch path (it recorded ev_end on its stream)
    // validation scratch: 4*(nblocks+1) doubles + wk (nz+2 doubles)
    double* d_scratch = nullptr;
    int nblocks = 0;
};

static GridDev to_dev(const pw_grid_t& g) {
    GridDev d;
    d.nx = g.nx;
    d.ny = g.ny;
    d.nz = g.nz;
    d.halo = g.halo;
    d.pj = g.pitch_j;
    d.pk = g.pitch_k;
    d.origin = g.origin;
    return d;
}

// Element count a field allocation must hold for this layout.
static long long alloc_elems_of(const pw_grid_t& g) {
    return g.origin + (long long)(g.nz + 1) * g.pitch_k + (long long)(g.ny + g.halo) * g.pitch_j + g.nx + g.halo +
           1;
}

pw_status_t pw::validate_grid(const pw_grid_t* g) {
    if (!g) return fail(PW_ERR_ARG, "grid is NULL");
    if (g->dtype != PW_F32 && g->dtype != PW_BF16 && g->dtype != PW_F16)
        return fail(PW_ERR_ARG, "unknown dtype %d", (int)g->dtype);
    if (g->nx < 1 || g->ny < 1) return fail(PW_ERR_ARG, "nx, ny must be >= 1 (got %d, %d)", g->nx, g->ny);
    if (g->nz < 3) return fail(PW_ERR_ARG, "nz must be >= 3 (got %d)", g->nz);
    if (g->halo < 1) return fail(PW_ERR_ARG, "halo must be >= 1 (got %d)", g->halo);
    if (g->halo > g->nx || g->halo > g->ny)
        return fail(PW_ERR_ARG, "halo %d exceeds the interior (%d x %d)", g->halo, g->nx, g->ny);
    if (g->pitch_j < (long long)g->nx + 2 * g->halo)
        return fail(PW_ERR_ARG, "pitch_j %lld < nx + 2*halo", (long long)g->pitch_j);
    if (g->pitch_k < g->pitch_j * ((long long)g->ny + 2 * g->halo))
        return fail(PW_ERR_ARG, "pitch_k %lld < pitch_j*(ny + 2*halo)", (long long)g->pitch_k);
    if (g->origin < (long long)(g->halo - 1) * (g->pitch_j + 1))
        return fail(PW_ERR_ARG, "origin %lld leaves no room for the halo", (long long)g->origin);
    return PW_OK;
}

// TMA eligibility of the layout (pointer alignment is checked per call).
// Writes the x offset `ox` of element i = 0 within its padded row.
bool pw::tma_layout_ok(const pw_grid_t& g, int* ox_out, const char** why) {
    const long long es = (long long)dtype_size(g.dtype);
    const long long padx = 16 / es;
    if (g.nx % 4) { *why = "nx is not a multiple of 4"; return false; }
    if ((g.pitch_j * es) % 16 || (g.pitch_k * es) % 16) { *why = "pitches are not multiples of 16 bytes"; return false; }
    const long long r = g.origin - (long long)(g.halo - 1) * g.pitch_j;
    if (r < 0 || r >= g.pitch_j) { *why = "origin is not within the first padded row"; return false; }
    if ((r + 1) % padx) { *why = "interior rows do not start on a 16-byte boundary"; return false; }
    if (r + g.nx + g.halo + 1 > g.pitch_j) { *why = "row does not fit its pitch"; return false; }
    if (g.nz + 2 > (1 << 30) || g.ny + 2 * g.halo > (1 << 30)) { *why = "grid too large for a tensor map"; return false; }
    *ox_out = (int)r;
    return true;
}

bool pw::aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Device (or managed) memory of `device`?  A host address handed to a kernel
// would fault the GPU, so every field pointer is checked on the host first.
bool pw::is_device_ptr(const void* p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // clear the sticky-free error of the query
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

// Tensor map of a field for a box of box_w x box_h elements, from the
// handle's cache of recently encoded maps.
static pw_status_t encode_map_box(pw_handle_t h, const void* ptr, int box_w, int box_h, CUtensorMap* out) {
    for (auto& c : h->maps)
        if (c.ptr == ptr && c.box_w == box_w && c.box_h == box_h) {
            *out = c.map;
            return PW_OK;
        }
    MapCacheEntry& e = h->maps[h->map_next];
    h->map_next = (h->map_next + 1) % (int)(sizeof(h->maps) / sizeof(h->maps[0]));
    pw_status_t st = encode_tensor_map_box(h->grid, ptr, box_w, box_h, out);
    if (st != PW_OK) return st;
    e.ptr = ptr;
    e.box_w = box_w;
    e.box_h = box_h;
    e.map = *out;
    return PW_OK;
}

// Tensor map for the single-grid k-march shape (lx lanes x nc cells, ty rows).
static pw_status_t encode_map(pw_handle_t h, const void* ptr, int lx, int ty, CUtensorMap* out, int nc = 4) {
    return encode_map_box(h, ptr, tma_box_width(h->grid.dtype, lx, nc), ty + 2, out);
}

pw_status_t pw::encode_tensor_map(const pw_grid_t& g, const void* ptr, int lx, int ty, CUtensorMap* out, int nc,
                                  int l2_promotion) {
    return encode_tensor_map_box(g, ptr, tma_box_width(g.dtype, lx, nc), ty + 2, out, l2_promotion);
}

// 3D map of one field: x = the padded row from its first element (element
// i = 0 at x = ox), y = rows from j = 1-halo, z = levels 0..nz+1.  Boxes of
// box_w x box_h x 1; out-of-range elements read as zero.
pw_status_t pw::encode_tensor_map_box(const pw_grid_t& g, const void* ptr, int box_w, int box_h, CUtensorMap* out,
                                      int l2_promotion) {
    auto fn = encode_fn();
    if (!fn) return fail(PW_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if (inject_failure(INJECT_TENSOR_MAP)) return fail(PW_ERR_CUDA, "cuTensorMapEncodeTiled failed (injected)");
    int ox = 0;
    const char* why = "";
    if (!tma_layout_ok(g, &ox, &why)) return fail(PW_ERR_UNSUPPORTED, "layout not TMA-eligible: %s", why);
    const size_t es = dtype_size(g.dtype);
    CUtensorMapDataType dt = g.dtype == PW_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                             : g.dtype == PW_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                  : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    cuuint64_t dims[3] = {(cuuint64_t)(ox + g.nx + g.halo + 1), (cuuint64_t)(g.ny + 2 * g.halo),
                          (cuuint64_t)(g.nz + 2)};
    cuuint64_t strides[2] = {(cuuint64_t)(g.pitch_j * es), (cuuint64_t)(g.pitch_k * es)};
    cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(out, dt, 3, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, (CUtensorMapL2promotion)l2_promotion,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(PW_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return PW_OK;
}

// Every pointer in ps[0..n) is device memory of the handle's GPU (checked
// once per pointer, then remembered).
static pw_status_t check_device_ptrs(pw_handle_t h, const void* const* ps, int n) {
    for (int a = 0; a < n; ++a) {
        const void* p = ps[a];
        bool known = false;
        for (auto q : h->dev_ok) known = known || (q == p);
        if (known) continue;
        if (!is_device_ptr(p, h->device))
            return fail(PW_ERR_ARG, "field pointer %p is not device memory of GPU %d", p, h->device);
        h->dev_ok[h->dev_next] = p;
        h->dev_next = (h->dev_next + 1) % pw_handle_s::kDevCache;
    }
    return PW_OK;
}

// Launch shape of the TMA kernel for the source terms (step = false) or the
// fused step (step = true).  A shape the user fixed (pw_set_tma_config) is used
// as given, unset fields at the scalar defaults (32 lanes x 4 cells x 4 rows, 4
// stages, one row per thread).  Otherwise the shape measured fastest on GB300
// (2048^2 x 64):
//   FP32:                       32 lanes x 4 cells x 4 rows (HBM-bound);
//   16-bit (source terms; steps when nx % 8 = 0):
//                               16 lanes x 8 cells x 8 rows, each thread's
//                               cells packed as FP32x2 pairs along x (BF16
//                               401, FP16 400 Gcell/s; two rows per thread
//                               315, 331);
//   16-bit steps, nx % 8 = 4:   32 lanes x 4 cells x 4 rows in x pairs;
//   nx <= 64:                   16 lanes x 4 cells x 4 rows;
// 4 stages, and the k segments chosen below.
static TmaConfig choose_tma(pw_handle_t h, bool step) {
    TmaConfig& cache = h->tma_auto[step ? 1 : 0];
    if (cache.ty) return cache;
    const TmaConfig& u = h->tma_user;
    const pw_grid_t& gr = h->grid;
    TmaConfig c;
    if (u.lx || u.nc || u.ty || u.stages || u.rp) {
        c.lx = u.lx ? u.lx : 32;
        c.nc = u.nc ? u.nc : 4;
        c.ty = u.ty ? u.ty : 4;
        c.stages = u.stages ? u.stages : 4;
        c.rp = u.rp ? u.rp : 1;
        if (c.rp == 3) {   // one row per thread, cells paired along x
            c.rp = 1;
            c.xp = 1;
        }
    } else {
        const bool half = dtype_size(gr.dtype) == 2;
        c.lx = 32;
        c.nc = 4;
        c.ty = 4;
        c.stages = 4;
        c.rp = 1;
        if (gr.nx <= 64) {
            c.lx = 16;
        } else if (half && (!step || gr.nx % 8 == 0)) {
            c.lx = 16;   // x pairs of 8 cells: tiles of 128 columns
            c.nc = 8;
            c.ty = 8;
            c.xp = 1;
        } else if (half) {
            c.xp = 1;    // x pairs of 4 cells
        }
    }
    if (u.nseg) {
        c.nseg = u.nseg;
    } else {
        const long long tiles =
            (long long)((gr.nx + c.nc * c.lx - 1) / (c.nc * c.lx)) * ((gr.ny + c.ty - 1) / c.ty);
        int bps = tma_blocks_per_sm(gr.dtype, c);
        if (bps < 1) bps = 1;
        const long long slots = (long long)h->num_sms * bps;
        // the count that minimises (waves of CTAs) x (planes each CTA marches:
        // its levels plus the two beyond them), down to 2 levels per segment;
        // more segments only for a gain of >= 3 %; and a single wave is
        // widened to two when that costs <= 5 % (one partial wave leaves SMs
        // with unequal CTA counts).  Measured on GB300 (FP32, 64 levels,
        // Gcell/s): 256^2 145 -> 181 (4 segments instead of 16), 1024^2
        // 236 -> 249 (2 instead of 1), 512^2 216 (1 segment) / 221 (2); 64^3
        // keeps 32 segments of 2 levels (4.0 us per call in a CUDA graph, 7.0
        // with 8)
        auto waves = [&](int n) { return (tiles * n + slots - 1) / slots; };
        auto cost = [&](int n) { return (double)waves(n) * ((double)gr.nz / n + 2.0); };
        int nseg = 1;
        for (int n = 2; gr.nz / n >= 2; ++n)
            if (cost(n) < 0.97 * cost(nseg)) nseg = n;
        if (waves(nseg) < 2)
            for (int n = nseg + 1; gr.nz / n >= 2; ++n)
                if (waves(n) >= 2) {
                    if (cost(n) <= 1.05 * cost(nseg)) nseg = n;
                    break;
                }
        c.nseg = nseg;
    }
    if (c.nseg > gr.nz / 2) c.nseg = std::max(1, gr.nz / 2);
    cache = c;
    return c;
}

static void make_scales(const float* scale, Scales* sc, bool* scaled) {
    *scaled = false;
    for (int q = 0; q < 3; ++q) {
        sc->in[q] = scale ? scale[q] : 1.f;
        sc->out[q] = scale ? scale[3 + q] : 1.f;
        if (sc->in[q] != 1.f || sc->out[q] != 1.f) *scaled = true;
    }
}

namespace pw {

pw_status_t internal_fail(pw_status_t s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

pw_status_t internal_cuda_fail(cudaError_t e, const char* what) { return cuda_fail(e, what); }

static std::atomic<int> g_inject[INJECT_KINDS];

bool inject_failure(int kind) {
    int n = g_inject[kind].load(std::memory_order_relaxed);
    while (n > 0)
        if (g_inject[kind].compare_exchange_weak(n, n - 1, std::memory_order_relaxed)) return true;
    return false;
}

cudaError_t set_smem_attr_once_impl(const void* kern, int bytes) {
    static std::mutex mu;
    static std::vector<std::pair<const void*, int>> done;   // (kernel, device)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (auto& d : done)
        if (d.first == kern && d.second == dev) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    // all the shared memory an SM has, so that shared memory does not hold the
    // resident CTAs below what the registers allow (the kernels stage their
    // data in shared memory and barely use the L1 cache)
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) done.emplace_back(kern, dev);
    return e;
}

bool internal_handle_grid(pw_handle_t h, pw_grid_t* g, int* num_sms) {
    if (!h) return false;
    *g = h->grid;
    *num_sms = h->num_sms;
    return true;
}

int internal_handle_device(pw_handle_t h) { return h ? h->device : -1; }

pw_status_t internal_check_device_ptrs(pw_handle_t h, const void* const* ps, int n) {
    return check_device_ptrs(h, ps, n);
}

}  // namespace pw

extern "C" {

pw_status_t pw_grid_default(int32_t nx, int32_t ny, int32_t nz, int32_t halo, pw_dtype_t dtype, pw_grid_t* out,
                            int64_t* alloc_elems) {
    if (!out) return fail(PW_ERR_ARG, "out is NULL");
    if (dtype != PW_F32 && dtype != PW_BF16 && dtype != PW_F16) return fail(PW_ERR_ARG, "unknown dtype");
    if (nx < 1 || ny < 1 || nz < 3 || halo < 1) return fail(PW_ERR_ARG, "need nx, ny >= 1, nz >= 3, halo >= 1");
    const long long line = 128 / (long long)dtype_size(dtype);   // elements per 128 bytes
    // interior i = 1 at x = ox + 1, a multiple of `line`, with room for the halo
    const long long ox = ((halo + line - 1) / line) * line - 1;
    const long long pj = ((ox + 1 + nx + halo + line - 1) / line) * line;
    const long long pk = pj * (ny + 2LL * halo);
    pw_grid_t g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.halo = halo;
    g.pitch_j = pj;
    g.pitch_k = pk;
    g.origin = ox + (long long)(halo - 1) * pj;
    g.dtype = dtype;
    *out = g;
    if (alloc_elems) *alloc_elems = pk * (nz + 2LL);
    return PW_OK;
}

pw_status_t pw_create(const pw_grid_t* grid, const pw_coeffs_t* coeffs, pw_handle_t* out) {
    if (!out) return fail(PW_ERR_ARG, "out is NULL");
    *out = nullptr;
    pw_status_t s = validate_grid(grid);
    if (s != PW_OK) return s;
    if (!coeffs || !coeffs->tzc1 || !coeffs->tzc2 || !coeffs->tzd1 || !coeffs->tzd2)
        return fail(PW_ERR_ARG, "coefficients or one of the vertical coefficient arrays is NULL");
    pw_handle_s* h = new (std::nothrow) pw_handle_s();
    if (!h) return fail(PW_ERR_OOM, "host allocation of the handle failed");
    h->grid = *grid;
    h->tcx = (float)coeffs->tcx;
    h->tcy = (float)coeffs->tcy;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    const int n = grid->nz + 2;
    std::vector<float> tz(4 * (size_t)n);
    for (int k = 0; k < n; ++k) {
        tz[k] = (float)coeffs->tzc1[k];
        tz[n + k] = (float)coeffs->tzc2[k];
        tz[2 * n + k] = (float)coeffs->tzd1[k];
        tz[3 * n + k] = (float)coeffs->tzd2[k];
    }
    if (e == cudaSuccess) e = dev_malloc(&h->d_tz, tz.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(h->d_tz, tz.data(), tz.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dev_malloc(&h->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(int));
    // the upload and the clear run on the legacy default stream, which the
    // caller's non-blocking streams do not wait for: finish them here
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
        pw_destroy(h);
        return cuda_fail(e, "pw_create");
    }
    *out = h;
    return PW_OK;
}

pw_status_t pw_destroy(pw_handle_t h) {
    if (!h) return PW_OK;
    for (auto& st : h->hs)   // an asynchronous host call may still be running
        if (st) cudaStreamSynchronize(st);
    for (auto& st : h->hs)
        if (st) cudaStreamDestroy(st);
    for (int c = 0; c < pw_handle_s::kMaxChunks; ++c) {
        if (h->ev_in[c]) cudaEventDestroy(h->ev_in[c]);
        if (h->ev_comp[c]) cudaEventDestroy(h->ev_comp[c]);
        if (h->ev_out[c]) cudaEventDestroy(h->ev_out[c]);
    }
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    if (h->ev_end) cudaEventDestroy(h->ev_end);
    cudaFree(h->d_tz);
    cudaFree(h->d_err);
    for (auto& p : h->d_stage) cudaFree(p);
    cudaFree(h->d_scratch);
    delete h;
    return PW_OK;
}

pw_status_t pw_set_kernel(pw_handle_t h, int32_t kind) {
    if (!h) return fail(PW_ERR_ARG, "handle is NULL");
    if (kind < 0 || kind > 2) return fail(PW_ERR_ARG, "kernel kind must be 0, 1 or 2");
    h->kernel_kind = kind;
    return PW_OK;
}

pw_status_t pw_set_tma_config(pw_handle_t h, int32_t lanes_x, int32_t cells, int32_t ty, int32_t stages,
                              int32_t nseg, int32_t rows_per_thread) {
    if (!h) return fail(PW_ERR_ARG, "handle is NULL");
    if (nseg < 0 || nseg > h->grid.nz / 2) return fail(PW_ERR_ARG, "nseg must be in 0..nz/2");
    if (rows_per_thread < 0 || rows_per_thread > 3)
        return fail(PW_ERR_ARG, "rows_per_thread must be 0, 1, 2 or 3");
    TmaConfig c{lanes_x ? lanes_x : 32, ty ? ty : 4, stages ? stages : 4, 1};
    c.nc = cells ? cells : 4;
    c.rp = rows_per_thread ? rows_per_thread : 1;
    if (c.rp == 3) {
        c.rp = 1;
        c.xp = 1;
    }
    if (!tma_config_supported(h->grid.dtype, c))
        return fail(PW_ERR_UNSUPPORTED,
                    "no TMA kernel instance for lanes_x=%d cells=%d ty=%d stages=%d rows_per_thread=%d (dtype %d)",
                    c.lx, c.nc, c.ty, c.stages, rows_per_thread ? rows_per_thread : 1, (int)h->grid.dtype);
    h->tma_user = TmaConfig{lanes_x, ty, stages, nseg};
    h->tma_user.nc = cells;
    h->tma_user.rp = rows_per_thread;
    h->tma_auto[0] = h->tma_auto[1] = TmaConfig{0, 0, 0, 0};
    for (auto& m : h->maps) m.ptr = nullptr;
    return PW_OK;
}

pw_status_t pw_set_step_blocking(pw_handle_t h, int32_t steps_per_pass, int32_t ty, int32_t stages,
                                 int32_t ctas_per_sm, int32_t nseg) {
    if (!h) return fail(PW_ERR_ARG, "handle is NULL");
    if (steps_per_pass < 0 || steps_per_pass > 2) return fail(PW_ERR_ARG, "steps_per_pass must be 0, 1 or 2");
    if (nseg < 0 || nseg > h->grid.nz / 2) return fail(PW_ERR_ARG, "nseg must be in 0..nz/2");
    Step2Config c{ty ? ty : 16, stages ? stages : 3, 1, ctas_per_sm ? ctas_per_sm : 1};
    if (!step2_config_supported(c))
        return fail(PW_ERR_UNSUPPORTED, "no two-step kernel instance for ty=%d stages=%d ctas_per_sm=%d", c.ty,
                    c.stages, c.minb);
    h->steps_per_pass = steps_per_pass;
    h->step2_user = Step2Config{ty, stages, nseg, ctas_per_sm};
    h->step2_auto = Step2Config{0, 0, 0, 0};
    return PW_OK;
}

// Launch shape of the two-step kernel: user overrides, else 16 rows, 3 stages,
// one CTA of 16 warps per SM (the fastest measured on GB300, 2048^2 x 64:
// FP32 208, BF16 201 Gcell-steps/s, against 156 and 152 with 8 rows), and k
// segments doubled until about two waves of CTAs cover the SMs (each segment
// keeps >= 8 levels).
static Step2Config choose_step2(pw_handle_t h) {
    if (h->step2_auto.ty) return h->step2_auto;
    const Step2Config& u = h->step2_user;
    Step2Config c{u.ty ? u.ty : 16, u.stages ? u.stages : 3, 1, u.minb ? u.minb : 1};
    if (u.nseg) {
        c.nseg = u.nseg;
    } else {
        const long long tiles = (long long)((h->grid.nx + step2_tile_cols() - 1) / step2_tile_cols()) *
                                ((h->grid.ny + c.ty - 3) / (c.ty - 2));
        int bps = step2_blocks_per_sm(h->grid.dtype, c);
        if (bps < 1) bps = 1;
        const long long slots = (long long)h->num_sms * bps;
        int nseg = 1;
        while (tiles * nseg < 2 * slots && h->grid.nz / (nseg * 2) >= 8) nseg *= 2;
        c.nseg = nseg;
    }
    if (c.nseg > h->grid.nz / 2) c.nseg = std::max(1, h->grid.nz / 2);
    h->step2_auto = c;
    return c;
}

// Launch shape of the TMA adjoint: each field the user fixed, else the
// automatic shape's.  k segments (automatic): the count that minimises the
// waves of CTAs times the planes each CTA marches (its levels plus the two
// it reads beyond them); segments keep >= 8 levels.  The adjoint holds few
// CTAs per SM (2 to 5), so a partly filled last wave costs much: at
// 512^2 x 64 with 64 x 4 tiles, 1024 CTAs fill 760 slots 1.35 times, and two
// segments turn that into 2.7 waves of half-length CTAs.
static AdjConfig choose_adjoint(pw_handle_t h) {
    if (h->adj_auto.na) return h->adj_auto;
    const AdjConfig d = adjoint_default_config();
    const AdjConfig& u = h->adj_user;
    AdjConfig c{u.na ? u.na : d.na, u.ty ? u.ty : d.ty, u.stages ? u.stages : d.stages, u.nseg};
    const pw_grid_t& gr = h->grid;
    if (!c.nseg) {
        const int tx = 32 * c.na;
        const long long tiles = (long long)((gr.nx + tx - 1) / tx) * ((gr.ny + c.ty - 1) / c.ty);
        int bps = adjoint_blocks_per_sm(c);
        if (bps < 1) bps = 1;
        const long long slots = (long long)h->num_sms * bps;
        c.nseg = 1;
        double best = 0.0;
        for (int n = 1; n <= 16 && (n == 1 || gr.nz / n >= 8); ++n) {
            const long long waves = (tiles * n + slots - 1) / slots;
            const double cost = (double)waves * ((double)gr.nz / n + 2.0);
            if (n == 1 || cost < 0.999 * best) {
                best = cost;
                c.nseg = n;
            }
        }
    }
    if (c.nseg > gr.nz) c.nseg = gr.nz;
    h->adj_auto = c;
    return c;
}

pw_status_t pw_set_adjoint_config(pw_handle_t h, int32_t cells, int32_t ty, int32_t stages, int32_t nseg) {
    if (!h) return fail(PW_ERR_ARG, "handle is NULL");
    if (cells < 0 || ty < 0 || stages < 0) return fail(PW_ERR_ARG, "cells, ty and stages must be >= 0");
    if (nseg < 0 || nseg > h->grid.nz) return fail(PW_ERR_ARG, "nseg must be in 0..nz");
    const AdjConfig d = adjoint_default_config();
    const AdjConfig c{cells ? cells : d.na, ty ? ty : d.ty, stages ? stages : d.stages, nseg};
    if (!adjoint_config_supported(c))
        return fail(PW_ERR_UNSUPPORTED, "no TMA adjoint instance for cells=%d ty=%d stages=%d", c.na, c.ty,
                    c.stages);
    h->adj_user = AdjConfig{cells, ty, stages, nseg};
    h->adj_auto = AdjConfig{0, 0, 0, 0};
    return PW_OK;
}

pw_status_t pw_get_adjoint_config(pw_handle_t h, int32_t out[4]) {
    if (!h || !out) return fail(PW_ERR_ARG, "handle or out is NULL");
    const AdjConfig c = choose_adjoint(h);
    out[0] = c.na;
    out[1] = c.ty;
    out[2] = c.stages;
    out[3] = c.nseg;
    return PW_OK;
}

pw_status_t pw_get_tma_config(pw_handle_t h, int32_t step, int32_t out[6]) {
    if (!h || !out) return fail(PW_ERR_ARG, "handle or out is NULL");
    const TmaConfig c = choose_tma(h, step != 0);
    out[0] = c.lx;
    out[1] = c.nc;
    out[2] = c.ty;
    out[3] = c.stages;
    out[4] = c.nseg;
    out[5] = c.xp ? 3 : c.rp;
    return PW_OK;
}

int32_t pw_last_kernel(pw_handle_t h) { return h ? h->last_kernel : 0; }

pw_status_t pw_tendencies(pw_handle_t h, const void* u, const void* v, const void* w, void* su, void* sv,
                          void* sw, const float* scale, pw_stream_t stream) {
    PW_RANGE("pw_tendencies");
    if (!h) return fail(PW_ERR_ARG, "handle is NULL");
    if (!u || !v || !w || !su || !sv || !sw) return fail(PW_ERR_ARG, "a field pointer is NULL");
    const void* ins[3] = {u, v, w};
    const void* outs[3] = {su, sv, sw};
    for (auto o : outs)
        for (auto i : ins)
            if (o == i) return fail(PW_ERR_ARG, "an output aliases an input");
    if (su == sv || su == sw || sv == sw) return fail(PW_ERR_ARG, "outputs alias each other");
    {
        const void* all[6] = {u, v, w, su, sv, sw};
        pw_status_t dst = check_device_ptrs(h, all, 6);
        if (dst != PW_OK) return dst;
    }
    if (scale)
        for (int q = 0; q < 6; ++q)
            if (!(scale[q] > 0.f) || !(scale[q] < 3.0e38f)) return fail(PW_ERR_ARG, "scales must be finite and > 0");
    Scales sc;
    bool scaled;
    make_scales(scale, &sc, &scaled);
    const GridDev g = to_dev(h->grid);
    CoefDev cf{h->tcx, h->tcy, h->d_tz};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    int ox = 0;
    const char* why = "";
    bool layout_ok = tma_layout_ok(h->grid, &ox, &why);
    bool ptrs_ok = true;
    for (auto p : ins) ptrs_ok = ptrs_ok && aligned16(p);
    for (auto p : outs) ptrs_ok = ptrs_ok && aligned16(p);
    bool use_tma = (h->kernel_kind == 2) || (h->kernel_kind == 0 && layout_ok && ptrs_ok);
    if (h->kernel_kind == 2) {
        if (!layout_ok) return fail(PW_ERR_UNSUPPORTED, "TMA kernel requested but %s", why);
        if (!ptrs_ok) return fail(PW_ERR_ALIGN, "TMA kernel requested but a field pointer is not 16-byte aligned");
    }
    if (use_tma) {
        TmaConfig c = choose_tma(h, false);
        CUtensorMap maps[3];
        for (int q = 0; q < 3; ++q) {
            pw_status_t st = encode_map(h, ins[q], c.lx, c.ty, &maps[q], c.nc);
            if (st != PW_OK) return st;
        }
        cudaError_t e = launch_tend_tma(h->grid.dtype, g, ox, maps, su, sv, sw, sc, cf, h->d_err, c, s);
        if (e != cudaSuccess) return cuda_fail(e, "TMA tendency kernel launch");
        h->last_kernel = 2;
    } else {
        cudaError_t e = launch_tend_generic(h->grid.dtype, g, u, v, w, su, sv, sw, sc, scaled, cf, h->num_sms, s);
        if (e != cudaSuccess) return cuda_fail(e, "generic tendency kernel launch");
        h->last_kernel = 1;
    }
    return PW_OK;
}

// Levels per chunk of the host path's copy / compute pipeline (build knob).
// The first chunk's copy in and the last chunk's copy out run alone, so
// smaller chunks overlap more; measured on GB300 (2048^2 x 64 FP32, pitched
// box copies): 16 levels 11.8, 8: 12.5-12.7, 4: 13.0-13.1, 2: 13.1 Gcell/s.
#ifndef PW_HOST_CHUNK_LEVELS
#define PW_HOST_CHUNK_LEVELS 4
#endif

// Copy the box i0..i0+ni-1, j0..j0+nj-1, levels k0..k1 of a field between
// host and device buffers of the same layout: one 3D copy when a level is a
// whole number of rows, else one 2D copy per level.  Only the box travels
// (no row padding, no rows or columns outside it).
static cudaError_t copy_box(const pw_grid_t& g, void* dst, const void* src, int i0, int ni, int j0, int nj, int k0,
                            int k1, cudaMemcpyKind kind, cudaStream_t s) {
    const size_t es = dtype_size(g.dtype);
    const size_t pitch = (size_t)g.pitch_j * es;
    auto at = [&](const void* base, int k) {
        return (char*)base + (size_t)(g.origin + (long long)k * g.pitch_k + (long long)j0 * g.pitch_j + i0) * es;
    };
    if (g.pitch_k % g.pitch_j == 0) {
        const size_t rows = (size_t)(g.pitch_k / g.pitch_j);
        cudaMemcpy3DParms p = {};
        p.srcPtr = make_cudaPitchedPtr(at(src, k0), pitch, (size_t)ni * es, rows);
        p.dstPtr = make_cudaPitchedPtr(at(dst, k0), pitch, (size_t)ni * es, rows);
        p.extent = make_cudaExtent((size_t)ni * es, (size_t)nj, (size_t)(k1 - k0 + 1));
        p.kind = kind;
        return cudaMemcpy3DAsync(&p, s);
    }
    for (int k = k0; k <= k1; ++k) {
        cudaError_t e = cudaMemcpy2DAsync(at(dst, k), pitch, at(src, k), pitch, (size_t)ni * es, (size_t)nj, kind, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The host path; wait = return once the results are in host memory, else
// once the work is enqueued (the caller's stream waits for its last copy).
static pw_status_t tendencies_host(pw_handle_t h, const void* u, const void* v, const void* w, void* su, void* sv,
                                   void* sw, const float* scale, pw_stream_t stream, bool wait) {
    PW_RANGE(wait ? "pw_tendencies_host" : "pw_tendencies_host_async");
    if (!h) return fail(PW_ERR_ARG, "handle is NULL");
    if (!u || !v || !w || !su || !sv || !sw) return fail(PW_ERR_ARG, "a field pointer is NULL");
    const pw_grid_t& g = h->grid;
    const size_t es = dtype_size(g.dtype);
    const size_t bytes = (size_t)alloc_elems_of(g) * es;
    for (auto& p : h->d_stage)
        if (!p) {
            cudaError_t e = dev_malloc(&p, bytes);
            if (e != cudaSuccess) return cuda_fail(e, "pw_tendencies_host staging allocation");
            e = cudaMemsetAsync(p, 0, bytes, reinterpret_cast<cudaStream_t>(stream));   // before the copies
            if (e != cudaSuccess) return cuda_fail(e, "pw_tendencies_host staging clear");
        }
    cudaStream_t us = reinterpret_cast<cudaStream_t>(stream);
    const void* hin[3] = {u, v, w};
    void* hout[3] = {su, sv, sw};
    // what travels: levels a..b of the inputs with their one-cell lateral
    // halo (all the scheme reads), and the interior of levels a..b of the
    // outputs
    auto copy_in = [&](int q, int a, int b, cudaStream_t s) {
        return copy_box(g, h->d_stage[q], hin[q], 0, g.nx + 2, 0, g.ny + 2, a, b, cudaMemcpyHostToDevice, s);
    };
    auto copy_out = [&](int q, int a, int b, cudaStream_t s) {
        return copy_box(g, hout[q], h->d_stage[3 + q], 1, g.nx, 1, g.ny, a, b, cudaMemcpyDeviceToHost, s);
    };

    int ox = 0;
    const char* why = "";
    bool ptrs_ok = true;
    for (auto p : h->d_stage) ptrs_ok = ptrs_ok && aligned16(p);
    const bool pipelined = h->kernel_kind != 1 && ptrs_ok && tma_layout_ok(g, &ox, &why) && g.nz >= 8;
    // Every call of either path ends by recording ev_end after its last copy
    // out.  The one-launch path runs on the caller's stream only, so it first
    // waits for the whole of the previous call (which may have run on another
    // stream); a pipelined call does the same after a one-launch call, and
    // after a pipelined call relies on the per-chunk events below.
    if (!h->ev_end) PW_CUDA(cudaEventCreateWithFlags(&h->ev_end, cudaEventDisableTiming), "pipeline event");
    if (!pipelined || h->host_prev_plain) PW_CUDA(cudaStreamWaitEvent(us, h->ev_end, 0), "pipeline wait");
    if (!pipelined) {   // one copy in, one launch, one copy out
        for (int q = 0; q < 3; ++q) PW_CUDA(copy_in(q, 1, g.nz, us), "pw_tendencies_host input copy");
        pw_status_t st = pw_tendencies(h, h->d_stage[0], h->d_stage[1], h->d_stage[2], h->d_stage[3], h->d_stage[4],
                                       h->d_stage[5], scale, stream);
        if (st != PW_OK) return st;
        for (int q = 0; q < 3; ++q) PW_CUDA(copy_out(q, 1, g.nz, us), "pw_tendencies_host output copy");
        PW_CUDA(cudaEventRecord(h->ev_end, us), "pipeline event");
        h->host_prev_plain = true;
        if (wait) PW_CUDA(cudaStreamSynchronize(us), "pw_tendencies_host synchronize");
        return PW_OK;
    }

    // Pipelined over k chunks: chunk c's input planes travel on stream 0
    // while chunk c-1 is computed on stream 1 and chunk c-2's outputs travel
    // back on stream 2 (the two copy directions and the kernels overlap).
    // Calls on one handle share the staging buffers, and a call may start
    // before the previous one has finished (the asynchronous form): chunk c's
    // input copy first waits for the previous call's kernels that read those
    // levels (chunks up to c+2), and chunk c's kernel for the previous call's
    // copy out of chunk c, so one call's inputs travel while the last one's
    // outputs come back.
    for (auto& st : h->hs)
        if (!st) PW_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "pipeline stream");
    for (int c = 0; c < pw_handle_s::kMaxChunks; ++c) {
        if (!h->ev_in[c]) PW_CUDA(cudaEventCreateWithFlags(&h->ev_in[c], cudaEventDisableTiming), "pipeline event");
        if (!h->ev_comp[c]) PW_CUDA(cudaEventCreateWithFlags(&h->ev_comp[c], cudaEventDisableTiming), "pipeline event");
        if (!h->ev_out[c]) PW_CUDA(cudaEventCreateWithFlags(&h->ev_out[c], cudaEventDisableTiming), "pipeline event");
    }
    if (!h->ev_start) PW_CUDA(cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming), "pipeline event");
    const int C = std::min(pw_handle_s::kMaxChunks, std::max(2, g.nz / PW_HOST_CHUNK_LEVELS));
    Scales sc;
    bool scaled;
    if (scale)
        for (int q = 0; q < 6; ++q)
            if (!(scale[q] > 0.f) || !(scale[q] < 3.0e38f)) return fail(PW_ERR_ARG, "scales must be finite and > 0");
    make_scales(scale, &sc, &scaled);
    TmaConfig cfg = choose_tma(h, false);
    cfg.nseg = C;
    cfg.seg_count = 1;
    CUtensorMap maps[3];
    for (int q = 0; q < 3; ++q) {
        pw_status_t st = encode_map(h, h->d_stage[q], cfg.lx, cfg.ty, &maps[q], cfg.nc);
        if (st != PW_OK) return st;
    }
    const GridDev gd = to_dev(g);
    CoefDev cf{h->tcx, h->tcy, h->d_tz};
    PW_CUDA(cudaEventRecord(h->ev_start, us), "pipeline event");
    for (auto st : h->hs) PW_CUDA(cudaStreamWaitEvent(st, h->ev_start, 0), "pipeline wait");
    int copied = 0;   // input levels 1..copied are on their way
    for (int c = 0; c < C; ++c) {
        const int kb = 1 + (int)(((long long)c * g.nz) / C);
        const int ke = (int)(((long long)(c + 1) * g.nz) / C);
        const int need = std::min(ke + 1, g.nz);
        if (need > copied) {
            // (an event not recorded yet, as on a handle's first call, is no wait)
            PW_CUDA(cudaStreamWaitEvent(h->hs[0], h->ev_comp[std::min(c + 2, C - 1)], 0), "pipeline wait");
            for (int q = 0; q < 3; ++q)
                PW_CUDA(copy_in(q, copied + 1, need, h->hs[0]), "pw_tendencies_host input copy");
            copied = need;
        }
        PW_CUDA(cudaEventRecord(h->ev_in[c], h->hs[0]), "pipeline event");
        PW_CUDA(cudaStreamWaitEvent(h->hs[1], h->ev_in[c], 0), "pipeline wait");
        PW_CUDA(cudaStreamWaitEvent(h->hs[1], h->ev_out[c], 0), "pipeline wait");
        cfg.seg0 = c;
        cudaError_t e = launch_tend_tma(g.dtype, gd, ox, maps, h->d_stage[3], h->d_stage[4], h->d_stage[5], sc,
                                        cf, h->d_err, cfg, h->hs[1]);
        if (e != cudaSuccess) return cuda_fail(e, "TMA tendency kernel launch");
        PW_CUDA(cudaEventRecord(h->ev_comp[c], h->hs[1]), "pipeline event");
        PW_CUDA(cudaStreamWaitEvent(h->hs[2], h->ev_comp[c], 0), "pipeline wait");
        for (int q = 0; q < 3; ++q) PW_CUDA(copy_out(q, kb, ke, h->hs[2]), "pw_tendencies_host output copy");
        PW_CUDA(cudaEventRecord(h->ev_out[c], h->hs[2]), "pipeline event");
    }
    h->last_kernel = 2;
    PW_CUDA(cudaEventRecord(h->ev_end, h->hs[2]), "pipeline event");
    h->host_prev_plain = false;
    PW_CUDA(cudaStreamWaitEvent(us, h->ev_end, 0), "pipeline wait");
    if (wait) PW_CUDA(cudaStreamSynchronize(h->hs[2]), "pw_tendencies_host synchronize");
    return PW_OK;
}

pw_status_t pw_tendencies_host(pw_handle_t h, const void* u, const void* v, const void* w, void* su, void* sv,
                               void* sw, const float* scale, pw_stream_t stream) {
    return tendencies_host(h, u, v, w, su, sv, sw, scale, stream, true);
}

pw_status_t pw_tendencies_host_async(pw_handle_t h, const void* u, const void* v, const void* w, void* su, void* sv,
                                     void* sw, const float* scale, pw_stream_t stream) {
    return tendencies_host(h, u, v, w, su, sv, sw, scale, stream, false);
}

// Storage scales of a step call: the state is read and written with the same
// per-field scale (NULL = 1).
static pw_status_t step_scales(const float* scale, Scales* sc, bool* scaled) {
    *scaled = false;
    for (int q = 0; q < 3; ++q) {
        const float x = scale ? scale[q] : 1.f;
        if (!(x > 0.f) || !(x < 3.0e38f)) return fail(PW_ERR_ARG, "scales must be finite and > 0");
        sc->in[q] = x;
        sc->out[q] = 1.f / x;   // the next state is stored with the same scale
        if (x != 1.f) *scaled = true;
    }
    return PW_OK;
}

// One single-step pass src -> dst (interior levels 1..nz and the periodic
// images of the lateral halo), on the TMA k-march or the generic kernel.
static pw_status_t step_pass(pw_handle_t h, const GridDev& g, const void* const* src, void* const* dst,
                             const Scales& sc, bool scaled, const CoefDev& cf, float dt, bool use_tma, int ox,
                             const TmaConfig& c, cudaStream_t s) {
    const pw_dtype_t dtp = h->grid.dtype;
    cudaError_t e;
    if (use_tma) {
        CUtensorMap maps[3];
        for (int q = 0; q < 3; ++q) {
            pw_status_t st = encode_map(h, src[q], c.lx, c.ty, &maps[q], c.nc);
            if (st != PW_OK) return st;
        }
        e = launch_step_tma(dtp, g, ox, maps, dst[0], dst[1], dst[2], sc, cf, dt, h->d_err, c, s);
        // the single-step k-march writes the images of a one-cell halo only
        for (int q = 0; q < 3 && e == cudaSuccess && g.halo != 1; ++q)
            e = launch_fill_halo(dtp, g, dst[q], h->num_sms, s);
    } else {
        e = launch_step_generic(dtp, g, src[0], src[1], src[2], dst[0], dst[1], dst[2], sc, scaled, cf, dt,
                                h->num_sms, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
    return PW_OK;
}

// TMA or generic for the step entry points: what pw_set_kernel asked for,
// else TMA when the layout and every pointer qualify.
static pw_status_t step_kernel_choice(pw_handle_t h, void* const* bufs, int n, bool* use_tma, int* ox) {
    const char* why = "";
    const bool layout_ok = tma_layout_ok(h->grid, ox, &why);
    bool ptrs_ok = true;
    for (int a = 0; a < n; ++a) ptrs_ok = ptrs_ok && aligned16(bufs[a]);
    if (h->kernel_kind == 2) {
        if (!layout_ok) return fail(PW_ERR_UNSUPPORTED, "TMA kernel requested but %s", why);
        if (!ptrs_ok) return fail(PW_ERR_ALIGN, "TMA kernel requested but a field pointer is not 16-byte aligned");
    }
    *use_tma = (h->kernel_kind == 2) || (h->kernel_kind == 0 && layout_ok && ptrs_ok);
    return PW_OK;
}

pw_status_t pw_step_to(pw_handle_t h, const void* u, const void* v, const void* w, void* nu, void* nv, void* nw,
                       float dt, const float* scale, pw_stream_t stream) {
    PW_RANGE("pw_step_to");
    if (!h) return fail(PW_ERR_ARG, "handle is NULL");
    void* bufs[6] = {const_cast<void*>(u), const_cast<void*>(v), const_cast<void*>(w), nu, nv, nw};
    for (int a = 0; a < 6; ++a) {
        if (!bufs[a]) return fail(PW_ERR_ARG, "a field pointer is NULL");
        for (int b = 0; b < a; ++b)
            if (bufs[a] == bufs[b]) return fail(PW_ERR_ARG, "the six fields must be distinct buffers");
    }
    if (!(dt == dt) || dt > 3.0e38f || dt < -3.0e38f) return fail(PW_ERR_ARG, "dt must be finite");
    Scales sc;
    bool scaled = false;
    pw_status_t st = step_scales(scale, &sc, &scaled);
    if (st != PW_OK) return st;
    st = check_device_ptrs(h, bufs, 6);
    if (st != PW_OK) return st;
    bool use_tma = false;
    int ox = 0;
    st = step_kernel_choice(h, bufs, 6, &use_tma, &ox);
    if (st != PW_OK) return st;
    const GridDev g = to_dev(h->grid);
    CoefDev cf{h->tcx, h->tcy, h->d_tz};
    TmaConfig c{};
    if (use_tma) c = choose_tma(h, true);
    if (use_tma && h->grid.nx % c.nc)
        return fail(PW_ERR_UNSUPPORTED, "fused steps with cells=%d need nx to be a multiple of %d", c.nc, c.nc);
    st = step_pass(h, g, bufs, bufs + 3, sc, scaled, cf, dt, use_tma, ox, c, reinterpret_cast<cudaStream_t>(stream));
    if (st != PW_OK) return st;
    h->last_kernel = use_tma ? 2 : 1;
    return PW_OK;
}

pw_status_t pw_step(pw_handle_t h, void* u, void* v, void* w, void* tmp_u, void* tmp_v, void* tmp_w, float dt,
                    int32_t nsteps, const float* scale, pw_stream_t stream) {
    PW_RANGE("pw_step");
    if (!h) return fail(PW_ERR_ARG, "handle is NULL");
    void* bufs[6] = {u, v, w, tmp_u, tmp_v, tmp_w};
    for (int a = 0; a < 6; ++a) {
        if (!bufs[a]) return fail(PW_ERR_ARG, "a field pointer is NULL");
        for (int b = 0; b < a; ++b)
            if (bufs[a] == bufs[b]) return fail(PW_ERR_ARG, "state and scratch buffers must be distinct");
    }
    if (nsteps < 0) return fail(PW_ERR_ARG, "nsteps must be >= 0");
    if (!(dt == dt) || dt > 3.0e38f || dt < -3.0e38f) return fail(PW_ERR_ARG, "dt must be finite");
    Scales sc;
    bool scaled = false;
    pw_status_t sst = step_scales(scale, &sc, &scaled);
    if (sst != PW_OK) return sst;
    sst = check_device_ptrs(h, bufs, 6);
    if (sst != PW_OK) return sst;
    const GridDev g = to_dev(h->grid);
    CoefDev cf{h->tcx, h->tcy, h->d_tz};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const pw_dtype_t dtp = h->grid.dtype;
    for (int q = 0; q < 3; ++q) {
        cudaError_t e = launch_fill_halo(dtp, g, bufs[q], h->num_sms, s);
        if (e != cudaSuccess) return cuda_fail(e, "halo fill launch");
    }
    int ox = 0;
    bool use_tma = false;
    sst = step_kernel_choice(h, bufs, 6, &use_tma, &ox);
    if (sst != PW_OK) return sst;
    // two steps per pass: TMA path, a lateral halo >= 2, and interior rows
    // starting at least 7 elements into their padded row (the q0 box begins
    // 7 columns before the first interior column)
    const bool tb2_ok = use_tma && g.halo >= 2 && ox >= 7;
    if (h->steps_per_pass == 2 && nsteps >= 2 && !tb2_ok)
        return fail(PW_ERR_UNSUPPORTED, "two steps per pass need the TMA path, a halo >= 2 and >= 7 columns before "
                                        "the interior in each padded row");
    // automatic (0) is one step per pass: on GB300 the two-step pass is bound
    // by instruction issue, not HBM, and runs slower per step
    const bool use_tb2 = tb2_ok && h->steps_per_pass == 2;
    TmaConfig c{};
    if (use_tma) c = choose_tma(h, true);
    if (use_tma && h->grid.nx % c.nc)
        return fail(PW_ERR_UNSUPPORTED, "fused steps with cells=%d need nx to be a multiple of %d", c.nc, c.nc);
    Step2Config c2{};
    if (use_tb2 && nsteps >= 2) c2 = choose_step2(h);
    int done = 0, passes = 0, kind = use_tma ? 2 : 1;
    while (done < nsteps) {
        void** src = (passes % 2 == 0) ? bufs : bufs + 3;
        void** dst = (passes % 2 == 0) ? bufs + 3 : bufs;
        if (use_tb2 && nsteps - done >= 2) {
            CUtensorMap maps[3];
            for (int q = 0; q < 3; ++q) {
                pw_status_t st = encode_map_box(h, src[q], step2_box_width(), c2.ty + 2, &maps[q]);
                if (st != PW_OK) return st;
            }
            cudaError_t e = launch_step2_tma(dtp, g, ox, maps, dst[0], dst[1], dst[2], sc, cf, dt, h->d_err, c2, s);
            done += 2;
            kind = 3;
            if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
        } else {
            pw_status_t st = step_pass(h, g, src, dst, sc, scaled, cf, dt, use_tma, ox, c, s);
            if (st != PW_OK) return st;
            done += 1;
        }
        ++passes;
    }
    h->last_kernel = kind;
    if (passes % 2 == 1) {   // the last state is in the scratch buffers: copy levels 1..nz back
        const size_t es = dtype_size(dtp);
        const pw_grid_t& gg = h->grid;
        const size_t lo = (size_t)(gg.origin + gg.pitch_k + (long long)(1 - gg.halo) * gg.pitch_j + 1 - gg.halo);
        const size_t hi = (size_t)(gg.origin + (long long)gg.nz * gg.pitch_k +
                                   (long long)(gg.ny + gg.halo) * gg.pitch_j + gg.nx + gg.halo + 1);
        for (int q = 0; q < 3; ++q)
            PW_CUDA(cudaMemcpyAsync((char*)bufs[q] + lo * es, (const char*)bufs[3 + q] + lo * es, (hi - lo) * es,
                                    cudaMemcpyDeviceToDevice, s),
                    "state copy");
    }
    return PW_OK;
}

pw_status_t pw_adjoint(pw_handle_t h, const void* u, const void* v, const void* w, const void* lsu,
                       const void* lsv, const void* lsw, void* gu, void* gv, void* gw, float alpha, int32_t flags,
                       pw_stream_t stream) {
    PW_RANGE("pw_adjoint");
    if (!h) return fail(PW_ERR_ARG, "handle is NULL");
    if (h->grid.dtype != PW_F32) return fail(PW_ERR_UNSUPPORTED, "pw_adjoint supports FP32 fields only");
    if (!u || !v || !w || !lsu || !lsv || !lsw || !gu || !gv || !gw) return fail(PW_ERR_ARG, "a field pointer is NULL");
    if (flags & ~(PW_ADJ_ACCUMULATE | PW_ADJ_PERIODIC | PW_ADJ_ADD_LAMBDA)) return fail(PW_ERR_ARG, "unknown flag bits");
    if ((flags & PW_ADJ_ACCUMULATE) && (flags & PW_ADJ_ADD_LAMBDA))
        return fail(PW_ERR_ARG, "PW_ADJ_ACCUMULATE and PW_ADJ_ADD_LAMBDA are exclusive");
    const void* ins[6] = {u, v, w, lsu, lsv, lsw};
    const void* outs[3] = {gu, gv, gw};
    for (auto o : outs)
        for (auto i : ins)
            if (o == i) return fail(PW_ERR_ARG, "an output aliases an input");
    if (gu == gv || gu == gw || gv == gw) return fail(PW_ERR_ARG, "outputs alias each other");
    if (!(alpha == alpha) || alpha > 3.0e38f || alpha < -3.0e38f) return fail(PW_ERR_ARG, "alpha must be finite");
    {
        pw_status_t dst = check_device_ptrs(h, ins, 6);
        if (dst == PW_OK) dst = check_device_ptrs(h, outs, 3);
        if (dst != PW_OK) return dst;
    }
    CoefDev cf{h->tcx, h->tcy, h->d_tz};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int ox = 0;
    const char* why = "";
    bool ptrs_ok = true;
    for (auto p : ins) ptrs_ok = ptrs_ok && aligned16(p);
    if ((flags & PW_ADJ_PERIODIC) && h->kernel_kind != 1 && ptrs_ok && tma_layout_ok(h->grid, &ox, &why)) {
        // TMA k-march adjoint: the sensitivities need periodic halos too
        const GridDev g = to_dev(h->grid);
        for (int q = 3; q < 6; ++q) {
            cudaError_t e = launch_fill_halo(PW_F32, g, const_cast<void*>(ins[q]), h->num_sms, s);
            if (e != cudaSuccess) return cuda_fail(e, "sensitivity halo fill");
        }
        CUtensorMap maps[6];
        const AdjConfig ac = choose_adjoint(h);
        for (int q = 0; q < 6; ++q) {
            pw_status_t st = encode_map(h, ins[q], 32, ac.ty, &maps[q], ac.na);
            if (st != PW_OK) return st;
        }
        const int nseg = ac.nseg;
        cudaError_t e = launch_adjoint_tma(g, ox, maps, (float*)gu, (float*)gv, (float*)gw, alpha,
                                           (flags & PW_ADJ_ACCUMULATE) ? 1 : 0, (flags & PW_ADJ_ADD_LAMBDA) ? 1 : 0,
                                           cf, nseg, h->d_err, ac, s);
        if (e != cudaSuccess) return cuda_fail(e, "adjoint kernel launch");
        h->last_kernel = 2;
        return PW_OK;
    }
    h->last_kernel = 1;
    cudaError_t e = launch_adjoint(to_dev(h->grid), (const float*)u, (const float*)v, (const float*)w,
                                   (const float*)lsu, (const float*)lsv, (const float*)lsw, (float*)gu, (float*)gv,
                                   (float*)gw, alpha, (flags & PW_ADJ_ACCUMULATE) ? 1 : 0,
                                   (flags & PW_ADJ_ADD_LAMBDA) ? 1 : 0, (flags & PW_ADJ_PERIODIC) ? 1 : 0, cf,
                                   h->num_sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint kernel launch");
    return PW_OK;
}

pw_status_t pw_fill_halo_periodic(pw_handle_t h, void* f, pw_stream_t stream) {
    PW_RANGE("pw_fill_halo_periodic");
    if (!h) return fail(PW_ERR_ARG, "handle is NULL");
    if (!f) return fail(PW_ERR_ARG, "field pointer is NULL");
    {
        const void* p = f;
        pw_status_t dst = check_device_ptrs(h, &p, 1);
        if (dst != PW_OK) return dst;
    }
    cudaError_t e = launch_fill_halo(h->grid.dtype, to_dev(h->grid), f, h->num_sms,
                                     reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "halo fill launch");
    return PW_OK;
}

static pw_status_t ensure_scratch(pw_handle_t h) {
    if (h->d_scratch) return PW_OK;
    h->nblocks = norm_blocks(h->num_sms);
    const size_t n = 4 * (size_t)(h->nblocks + 1) + (size_t)(h->grid.nz + 2);
    cudaError_t e = dev_malloc(&h->d_scratch, n * sizeof(double));
    if (e != cudaSuccess) {
        h->d_scratch = nullptr;
        return cuda_fail(e, "validation scratch allocation");
    }
    return PW_OK;
}

pw_status_t pw_error_norms(pw_handle_t h, const void* test, float scale, const double* ref, int32_t k0, int32_t k1,
                           double* out, pw_stream_t stream) {
    PW_RANGE("pw_error_norms");
    if (!h) return fail(PW_ERR_ARG, "handle is NULL");
    if (!test || !ref || !out) return fail(PW_ERR_ARG, "a pointer is NULL");
    if (k0 < 1 || k1 > h->grid.nz || k0 > k1) return fail(PW_ERR_ARG, "need 1 <= k0 <= k1 <= nz");
    const void* dp[2] = {test, ref};
    pw_status_t st = check_device_ptrs(h, dp, 2);
    if (st != PW_OK) return st;
    st = ensure_scratch(h);
    if (st != PW_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_error_norms(h->grid.dtype, to_dev(h->grid), test, scale, ref, k0, k1, h->d_scratch,
                                       h->nblocks, s);
    if (e != cudaSuccess) return cuda_fail(e, "norm kernel launch");
    PW_CUDA(cudaMemcpyAsync(out, h->d_scratch + 4 * (size_t)h->nblocks, 4 * sizeof(double), cudaMemcpyDeviceToHost, s),
            "norm result copy");
    PW_CUDA(cudaStreamSynchronize(s), "norm synchronize");
    return PW_OK;
}

pw_status_t pw_weighted_dot(pw_handle_t h, const void* a, float sa, const void* b, float sb, const double* wk,
                            int32_t k0, int32_t k1, double* out, pw_stream_t stream) {
    PW_RANGE("pw_weighted_dot");
    if (!h) return fail(PW_ERR_ARG, "handle is NULL");
    if (!a || !b || !out) return fail(PW_ERR_ARG, "a pointer is NULL");
    if (k0 < 1 || k1 > h->grid.nz || k0 > k1) return fail(PW_ERR_ARG, "need 1 <= k0 <= k1 <= nz");
    const void* dp[2] = {a, b};
    pw_status_t st = check_device_ptrs(h, dp, 2);
    if (st != PW_OK) return st;
    st = ensure_scratch(h);
    if (st != PW_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double* d_wk = nullptr;
    if (wk) {
        d_wk = h->d_scratch + 4 * (size_t)(h->nblocks + 1);
        PW_CUDA(cudaMemcpyAsync(d_wk, wk, (h->grid.nz + 2) * sizeof(double), cudaMemcpyHostToDevice, s),
                "weight copy");
    }
    cudaError_t e = launch_weighted_dot(h->grid.dtype, to_dev(h->grid), a, sa, b, sb, d_wk, k0, k1, h->d_scratch,
                                        h->nblocks, s);
    if (e != cudaSuccess) return cuda_fail(e, "dot kernel launch");
    double r[4];
    PW_CUDA(cudaMemcpyAsync(r, h->d_scratch + 4 * (size_t)h->nblocks, 4 * sizeof(double), cudaMemcpyDeviceToHost, s),
            "dot result copy");
    PW_CUDA(cudaStreamSynchronize(s), "dot synchronize");
    out[0] = r[2];
    return PW_OK;
}

pw_status_t pw_sync(pw_handle_t h, pw_stream_t stream) {
    if (!h) return fail(PW_ERR_ARG, "handle is NULL");
    PW_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)), "stream synchronize");
    int flag = 0;
    PW_CUDA(cudaMemcpy(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost), "status word read");
    if (flag != DEV_OK) {
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        PW_CUDA(cudaMemsetAsync(h->d_err, 0, sizeof(int), s), "status word clear");
        PW_CUDA(cudaStreamSynchronize(s), "status word clear");
        if (flag == DEV_OOB_STORE)
            return fail(PW_ERR_CUDA, "a store outside the field's cells was caught and skipped (debug bounds build)");
        return fail(PW_ERR_DEVICE_TIMEOUT, "a kernel gave up a bounded wait (code %d)", flag);
    }
    PW_CUDA(cudaGetLastError(), "pending CUDA error");
    return PW_OK;
}

int32_t pw_debug_layout_check(const pw_grid_t* g, int64_t offset, int32_t n, int32_t interior_only) {
    if (!g || validate_grid(g) != PW_OK || n < 1) return -1;
    return layout_cells_ok(to_dev(*g), (long long)offset, n, interior_only != 0) ? 1 : 0;
}

int32_t pw_debug_bounds_build(void) { return PW_DEBUG_BOUNDS ? 1 : 0; }

pw_status_t pw_inject_failures(int32_t kind, int32_t count) {
    if (kind < 0 || kind >= INJECT_KINDS) return fail(PW_ERR_ARG, "kind must be 0 (allocations) or 1 (tensor maps)");
    if (count < 0) return fail(PW_ERR_ARG, "count must be >= 0");
    g_inject[kind].store(count, std::memory_order_relaxed);
    return PW_OK;
}

pw_status_t pw_selftest_wait_timeout(pw_handle_t h, int64_t limit_ns, pw_stream_t stream) {
    PW_RANGE("pw_selftest_wait_timeout");
    if (!h) return fail(PW_ERR_ARG, "handle is NULL");
    if (limit_ns < 1000000 || limit_ns > 1000000000) return fail(PW_ERR_ARG, "limit_ns must be in [1e6, 1e9]");
    cudaError_t e = launch_selftest_wait((uint64_t)limit_ns, h->d_err, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "self-test launch");
    return PW_OK;
}

const char* pw_last_error(void) { return g_err.c_str(); }

const char* pw_status_string(pw_status_t s) {
    switch (s) {
        case PW_OK: return "PW_OK";
        case PW_ERR_ARG: return "PW_ERR_ARG";
        case PW_ERR_ALIGN: return "PW_ERR_ALIGN";
        case PW_ERR_CUDA: return "PW_ERR_CUDA";
        case PW_ERR_OOM: return "PW_ERR_OOM";
        case PW_ERR_DEVICE_TIMEOUT: return "PW_ERR_DEVICE_TIMEOUT";
        case PW_ERR_UNSUPPORTED: return "PW_ERR_UNSUPPORTED";
    }
    return "PW_ERR_UNKNOWN";
}

}  // extern "C"
