// Batched PW source terms: many independent grids of uneven sizes in one
// persistent launch, replayed from a CUDA graph.
//
// The paper scales its Versal design by decomposing the problem into
// independent compute units, each owning a 3D part of the grid (Sec. 5);
// here the units are whole grids.  Every (grid, tile) pair is a work item;
// the items go grid by grid, deepest grids first (a stable sort on nz, so
// each grid's tiles stay together in raster order and neighbouring tiles
// share their halo rows through L2), and a persistent k-march CTA per SM
// slot takes the next item from an atomic counter until none is left, so
// large and small grids share the GPU without a launch per grid.  A grid's
// last column of tiles, when it would hold at most half a tile, runs with
// tiles half as wide through the same ring (narrow last columns).  The
// per-grid records and TMA descriptors live in device tables that are
// re-uploaded only when the field pointers change; the counter reset and the
// kernel are captured once in a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <vector>

#include "pw_stencil.cuh"

namespace pw {

struct BatchGridDev {
    GridDev g;
    int ox;
    int tiles_x, tiles_y;   // the grid's wide tiles (columns, rows)
    int ntiles_y, nbx;      // narrow last column: its tiles (0: none) and its index in narrow tiles
    int nseg;
    float tcx, tcy;
    const float* tz;
    void* o[3];
};

// The tile shapes of a batched kernel: a wide one (LX, TY, NC) and,
// optionally (NC2 > 0), a narrow one of half its width and the same thread
// count (LX2, TY2, NC2) for a grid's last column when that column holds at
// most half a wide tile.  Both march through one plane ring whose mbarriers
// sit after the larger shape's ring region.
template <typename T, int LX, int TY, int S, int NC, int RP, int XP, int LX2, int TY2, int NC2>
struct BatchShapes {
    static constexpr bool DUAL = NC2 > 0;
    using LW = TmaLayout<T, LX, TY, S, NC, RP, XP>;
    using LN = TmaLayout<T, DUAL ? LX2 : LX, DUAL ? TY2 : TY, S, DUAL ? NC2 : NC, RP, XP>;
    static constexpr size_t RING = LW::RING_BYTES > LN::RING_BYTES ? LW::RING_BYTES : LN::RING_BYTES;
    static constexpr size_t SMEM =
        LW::smem_bytes(RING) > LN::smem_bytes(RING) ? LW::smem_bytes(RING) : LN::smem_bytes(RING);
    static constexpr int THREADS = LW::THREADS;
    static constexpr int MAPS = DUAL ? 6 : 3;   // tensor maps per grid (u, v, w per shape)
    static_assert(!DUAL || LN::THREADS == LW::THREADS, "both shapes use every thread of the CTA");
    static_assert(!DUAL || 2 * LN::TX == LW::TX, "the narrow shape is half as wide");
    static_assert(LN::CTAB == LW::CTAB, "one coefficient-table layout");
};

// Resident CTAs per SM the batch kernel's register budget is sized for (at
// most what shared memory and the thread limit allow; 0: as the single-grid
// k-march).  On GB300 (512-grid batch) 8 or 10 for the 64-thread tiles, 116
// or 95 registers instead of 150, ran at 221 against 224 Gcell/s.
#ifndef PW_BATCH_MINB
#define PW_BATCH_MINB 0
#endif
// 1: one CTA per work item in a plain grid launch (the hardware hands out the
// items in launch order) instead of persistent CTAs taking items from a
// counter.  Measured on GB300: 512-grid batch FP32 226.9 -> 229.9, BF16
// 320.3 -> 322.4 Gcell/s; one 2048^2 x 64 grid as a batch BF16 358.9 -> 368.3
// (the grid launch of the single-grid kernel: 382).  The persistent form
// stays the default: the work list and its order are the batch's own, and
// ctas_per_sm bounds how much of the GPU the batch holds.
#ifndef PW_BATCH_GRID_LAUNCH
#define PW_BATCH_GRID_LAUNCH 0
#endif
template <typename T, int LX, int TY, int S, int NC, int RP, int XP, int LX2, int TY2, int NC2>
constexpr int batch_min_blocks() {
    using B = BatchShapes<T, LX, TY, S, NC, RP, XP, LX2, TY2, NC2>;
    constexpr int by_smem = (int)((227u * 1024u) / B::SMEM);
    constexpr int by_threads = 2048 / B::THREADS;
    constexpr int m = by_smem < by_threads ? by_smem : by_threads;
    constexpr int want = PW_BATCH_MINB ? PW_BATCH_MINB : tma_min_blocks<T, LX, TY, S, NC, RP, XP>();
    return want < m ? want : m;
}

// NC cells per thread along x; RP = 2: two rows per thread in packed FP32x2
// arithmetic; XP = 1: the cells of one row packed as FP32x2 pairs (16-bit
// storage for both).  NC2 > 0: a grid's narrow last column runs with the
// (LX2, TY2, NC2) tiles.
template <typename T, int LX, int TY, int S, int NC, int RP, int XP, int LX2, int TY2, int NC2>
__global__ void __launch_bounds__((BatchShapes<T, LX, TY, S, NC, RP, XP, LX2, TY2, NC2>::THREADS),
                                  (batch_min_blocks<T, LX, TY, S, NC, RP, XP, LX2, TY2, NC2>()))
    tma_batch_kernel(const BatchGridDev* __restrict__ grids, const CUtensorMap* __restrict__ maps,
                     const int2* __restrict__ items, const int n_items, int* __restrict__ counter, const Scales sc,
                     int* __restrict__ err) {
    using B = BatchShapes<T, LX, TY, S, NC, RP, XP, LX2, TY2, NC2>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MarchSmem<T, LX, TY, S, NC, RP, XP> sm(smem_raw, B::RING);
    const int tid = threadIdx.y * 32 + threadIdx.x;
    sm.init(tid);
    uint32_t ring = 0;
    // (Taking the next item while the current one marches measured slower:
    // 512-grid batch FP32 7.77 -> 8.0-8.1 ms, BF16 5.51 -> 5.56-5.62 ms.  A
    // tile then starts about a tile's time after it was taken, so raster
    // neighbours no longer march together and share fewer halo rows in L2,
    // and each CTA holds one more item at the end.)
    for (;;) {
        int it;
        if constexpr (PW_BATCH_GRID_LAUNCH) {
            it = blockIdx.x;
        } else {
            if (tid == 0) sm.flag[1] = atomicAdd(counter, 1);
            __syncthreads();
            it = sm.flag[1];
            __syncthreads();   // every thread has read the item before it is overwritten
        }
        if (it >= n_items) break;
        const int2 item = items[it];
        const BatchGridDev& bg = grids[item.x];
        const int wide = bg.tiles_x * bg.tiles_y;
        const int per_seg = wide + bg.ntiles_y;
        const int seg = item.y / per_seg;
        const int rem = item.y - seg * per_seg;
        const int nz = bg.g.nz;
        const int kb = 1 + (int)(((long long)seg * nz) / bg.nseg);
        const int ke = (int)(((long long)(seg + 1) * nz) / bg.nseg);
        const CoefDev cf{bg.tcx, bg.tcy, bg.tz};
        const CUtensorMap* m = maps + B::MAPS * (size_t)item.x;
        bool ok;
        if (B::DUAL && rem >= wide) {
            if constexpr (B::DUAL) {
                MarchSmem<T, LX2, TY2, S, NC2, RP, XP> sn(smem_raw, B::RING);
                ok = march_tile<T, LX2, TY2, S, MODE_TEND, NC2, RP, XP>(
                    sn, m + 3, m + 4, m + 5, (T*)bg.o[0], (T*)bg.o[1], (T*)bg.o[2], bg.g, bg.ox, fold_coef(cf, sc),
                    0.f, bg.nbx, rem - wide, kb, ke, ring, err);
            } else {
                ok = false;
            }
        } else {
            const int by = rem / bg.tiles_x, bx = rem - by * bg.tiles_x;
            ok = march_tile<T, LX, TY, S, MODE_TEND, NC, RP, XP>(sm, m, m + 1, m + 2, (T*)bg.o[0], (T*)bg.o[1],
                                                                 (T*)bg.o[2], bg.g, bg.ox, fold_coef(cf, sc), 0.f,
                                                                 bx, by, kb, ke, ring, err);
        }
        if (!ok || PW_BATCH_GRID_LAUNCH) break;
    }
}

// Instantiated tile shapes (lanes per row, rows, stages, cells per thread,
// rows per thread, x pairs); the packed forms for 16-bit storage only.
#define PW_BATCH_CONFIGS(X) X(32, 4, 4, 4, 1, 0) X(32, 8, 4, 4, 1, 0) X(16, 4, 4, 4, 1, 0) X(16, 8, 4, 4, 1, 0) \
    X(16, 16, 4, 4, 1, 0) \
    X(32, 8, 4, 4, 2, 0) X(16, 8, 4, 4, 2, 0) X(32, 4, 4, 4, 1, 1) X(32, 8, 4, 4, 1, 1) X(16, 4, 4, 4, 1, 1)      \
    X(16, 8, 4, 4, 1, 1) X(16, 4, 4, 8, 1, 1) X(16, 8, 4, 8, 1, 1) X(8, 8, 4, 8, 1, 1) X(8, 16, 4, 8, 1, 1)        \
    X(8, 16, 4, 4, 1, 0) X(32, 16, 4, 4, 1, 0)

// Wide shapes paired with a narrow last-column shape (the second triple:
// lanes per row, rows, cells per thread; same stages, rows per thread and
// pairing); the FP32 shapes (XP = 0) for FP32 storage, the x-pair ones for
// 16-bit storage.
#define PW_BATCH_DUALS(X) X(16, 16, 4, 4, 1, 0, 8, 32, 4) X(16, 8, 4, 4, 1, 0, 8, 16, 4) \
    X(32, 8, 4, 4, 1, 0, 16, 16, 4) X(8, 16, 4, 8, 1, 1, 8, 16, 4) X(16, 8, 4, 8, 1, 1, 8, 16, 8)

template <typename T, int LX, int TY, int S, int NC, int RP, int XP, int LX2 = 0, int TY2 = 0, int NC2 = 0>
static cudaError_t batch_inst(bool query, int* bps, const BatchGridDev* grids, const CUtensorMap* maps,
                              const int2* items, int n_items, int* counter, const Scales& sc, int* err, int ctas,
                              cudaStream_t s) {
  if constexpr (!nc_ok<T, NC, RP, XP>() || (NC2 > 0 && !nc_ok<T, NC2, RP, XP>()) ||
                (NC2 > 0 && (XP == 0) != std::is_same<T, float>::value)) {
    return cudaErrorInvalidConfiguration;
  } else {
    using B = BatchShapes<T, LX, TY, S, NC, RP, XP, LX2, TY2, NC2>;
    auto kern = tma_batch_kernel<T, LX, TY, S, NC, RP, XP, LX2, TY2, NC2>;
    cudaError_t e = set_smem_attr_once(kern, (int)B::SMEM);
    if (e != cudaSuccess) return e;
    if (query) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, kern, B::THREADS, B::SMEM);
    kern<<<ctas, dim3(32, B::THREADS / 32), B::SMEM, s>>>(grids, maps, items, n_items, counter, sc, err);
    return cudaGetLastError();
  }
}

template <typename T>
static cudaError_t batch_t(const TmaConfig& c, bool dual, bool query, int* bps, const BatchGridDev* grids,
                           const CUtensorMap* maps, const int2* items, int n_items, int* counter, const Scales& sc,
                           int* err, int ctas, cudaStream_t s) {
    if (dual) {
#define PW_BDD(LX_, TY_, S_, NC_, RP_, XP_, LX2_, TY2_, NC2_)                                                 \
    if (c.lx == LX_ && c.ty == TY_ && c.stages == S_ && c.nc == NC_ && c.rp == RP_ && c.xp == XP_)             \
        return batch_inst<T, LX_, TY_, S_, NC_, RP_, XP_, LX2_, TY2_, NC2_>(query, bps, grids, maps, items, n_items, \
                                                                            counter, sc, err, ctas, s);
        PW_BATCH_DUALS(PW_BDD)
#undef PW_BDD
        return cudaErrorInvalidConfiguration;
    }
#define PW_BD(LX_, TY_, S_, NC_, RP_, XP_)                                                                     \
    if (c.lx == LX_ && c.ty == TY_ && c.stages == S_ && c.nc == NC_ && c.rp == RP_ && c.xp == XP_)             \
        return batch_inst<T, LX_, TY_, S_, NC_, RP_, XP_>(query, bps, grids, maps, items, n_items, counter, sc, err, \
                                                          ctas, s);
    PW_BATCH_CONFIGS(PW_BD)
#undef PW_BD
    return cudaErrorInvalidConfiguration;
}

static cudaError_t batch_dispatch(pw_dtype_t dt, const TmaConfig& c, bool dual, bool query, int* bps,
                                  const BatchGridDev* grids, const CUtensorMap* maps, const int2* items, int n_items,
                                  int* counter, const Scales& sc, int* err, int ctas, cudaStream_t s) {
    switch (dt) {
        case PW_F32:
            return batch_t<float>(c, dual, query, bps, grids, maps, items, n_items, counter, sc, err, ctas, s);
        case PW_BF16:
            return batch_t<__nv_bfloat16>(c, dual, query, bps, grids, maps, items, n_items, counter, sc, err, ctas,
                                          s);
        case PW_F16:
            return batch_t<__half>(c, dual, query, bps, grids, maps, items, n_items, counter, sc, err, ctas, s);
    }
    return cudaErrorInvalidValue;
}

static bool batch_config_supported(const TmaConfig& c, pw_dtype_t dt) {
    if ((c.rp == 2 || c.xp || c.nc != 4) && dt == PW_F32) return false;
#define PW_BS(LX_, TY_, S_, NC_, RP_, XP_) \
    if (c.lx == LX_ && c.ty == TY_ && c.stages == S_ && c.nc == NC_ && c.rp == RP_ && c.xp == XP_) return true;
    PW_BATCH_CONFIGS(PW_BS)
#undef PW_BS
    return false;
}

// The narrow last-column shape paired with c for this storage type, if any.
static bool narrow_partner(const TmaConfig& c, pw_dtype_t dt, TmaConfig* n) {
#define PW_BN(LX_, TY_, S_, NC_, RP_, XP_, LX2_, TY2_, NC2_)                                                  \
    if (c.lx == LX_ && c.ty == TY_ && c.stages == S_ && c.nc == NC_ && c.rp == RP_ && c.xp == XP_ &&           \
        (XP_ == 0) == (dt == PW_F32)) {                                                                        \
        *n = c;                                                                                                \
        n->lx = LX2_;                                                                                          \
        n->ty = TY2_;                                                                                          \
        n->nc = NC2_;                                                                                          \
        return true;                                                                                           \
    }
    PW_BATCH_DUALS(PW_BN)
#undef PW_BN
    return false;
}

// A grid's tiles: full-width columns, then its last column either as one
// more wide column or, when it holds at most half a wide tile and a narrow
// shape is in use, as a column of narrow tiles.
struct TilePlan {
    int tx, ty, nty, nbx;
};
static TilePlan tile_plan(const pw_grid_t& g, const TmaConfig& c, const TmaConfig* narrow) {
    const int TX = c.nc * c.lx;
    const int full = g.nx / TX, r = g.nx - full * TX;
    TilePlan p{(g.nx + TX - 1) / TX, (g.ny + c.ty - 1) / c.ty, 0, 0};
    if (narrow && r > 0 && r <= narrow->nc * narrow->lx) {
        p.tx = full;
        p.nty = (g.ny + narrow->ty - 1) / narrow->ty;
        p.nbx = full * (TX / (narrow->nc * narrow->lx));
    }
    return p;
}

}  // namespace pw

using namespace pw;

struct pw_batch_s {
    int n = 0;
    pw_dtype_t dtype = PW_F32;
    int device = 0, num_sms = 0;
    std::vector<pw_grid_t> grids;
    std::vector<int> ox;
    std::vector<float> tcx, tcy;
    std::vector<size_t> tz_off;
    float* d_tz = nullptr;
    BatchGridDev* d_grids = nullptr;
    CUtensorMap* d_maps = nullptr;
    int2* d_items = nullptr;
    int* d_counter = nullptr;
    int* d_err = nullptr;
    BatchGridDev* h_grids = nullptr;   // pinned staging
    CUtensorMap* h_maps = nullptr;
    std::vector<int2> items;
    long long cells = 0;
    TmaConfig cfg{32, 4, 4, 1};
    bool narrow_on = true;  // narrow last columns where cfg has a narrow partner
    bool dual = false;      // ... and it has one: ncfg
    TmaConfig ncfg{0, 0, 0, 1};
    int ctas_per_sm = 0;    // 0 = occupancy
    int ctas = 0;
    std::vector<const void*> ptrs;   // 6n pointers the tables were built for
    bool tables_ok = false, items_ok = false;
    Scales graph_sc{{1.f, 1.f, 1.f}, {1.f, 1.f, 1.f}};
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static pw_status_t bfail(pw_status_t s, const char* msg) { return internal_fail(s, "%s", msg); }

static void drop_graph(pw_batch_t b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Work items for the current tile shape.
// Work order: the deepest grids first (nz), each grid's tiles together
// in raster order (x fastest), so a tile's neighbours start at about the same
// time and their shared halo rows and columns come from L2.  Measured on the
// 512-grid batch: 222 Gcell/s, against 212 when the tile width was part of
// the cost (a grid's ragged last column then ran with other grids' ones) and
// 218 with y fastest.
// The work list of shape `cfg` is built and uploaded first and the batch
// switched to it only when everything succeeded: on failure the batch keeps
// its previous shape, work list and captured graph.
static pw_status_t build_items(pw_batch_t b, const TmaConfig& cfg, int ctas_per_sm, bool narrow_on) {
    TmaConfig ncfg{0, 0, 0, 1};
    const bool dual = narrow_on && narrow_partner(cfg, b->dtype, &ncfg);
    struct Item {
        int grid, tile;
        long long cost;
    };
    std::vector<Item> v;
    for (int q = 0; q < b->n; ++q) {
        const TilePlan p = tile_plan(b->grids[q], cfg, dual ? &ncfg : nullptr);
        for (int t = 0; t < p.tx * p.ty + p.nty; ++t) v.push_back({q, t, (long long)b->grids[q].nz});
    }
    std::stable_sort(v.begin(), v.end(), [](const Item& a, const Item& c) { return a.cost > c.cost; });
    std::vector<int2> items(v.size());
    for (size_t i = 0; i < v.size(); ++i) items[i] = make_int2(v[i].grid, v[i].tile);
    int bps = 0;
    Scales one{{1.f, 1.f, 1.f}, {1.f, 1.f, 1.f}};
    cudaError_t e = batch_dispatch(b->dtype, cfg, dual, true, &bps, nullptr, nullptr, nullptr, 0, nullptr, one,
                                   nullptr, 0, nullptr);
    if (e != cudaSuccess || bps < 1)
        return internal_cuda_fail(e == cudaSuccess ? cudaErrorInvalidConfiguration : e, "batch kernel occupancy");
    int2* d = nullptr;
    e = dev_malloc(&d, std::max<size_t>(1, items.size()) * sizeof(int2));
    if (e == cudaSuccess) e = cudaMemcpy(d, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice);
    // legacy-stream upload (and, at creation, the coefficient upload and the
    // status clear): complete before any launch on the caller's streams
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
        cudaFree(d);
        return internal_cuda_fail(e, "batch work list upload");
    }
    // switch over (cudaFree waits for any launch still reading the old list)
    drop_graph(b);
    cudaFree(b->d_items);
    b->d_items = d;
    b->items.swap(items);
    b->cfg = cfg;
    b->ncfg = ncfg;
    b->dual = dual;
    b->narrow_on = narrow_on;
    b->ctas_per_sm = ctas_per_sm;
    const int per_sm = ctas_per_sm ? std::min(ctas_per_sm, bps) : bps;
    b->ctas = PW_BATCH_GRID_LAUNCH ? std::max<int>(1, (int)b->items.size()) : b->num_sms * per_sm;
    b->items_ok = true;
    b->tables_ok = false;
    return PW_OK;
}

extern "C" {

pw_status_t pw_batch_create(int32_t n, const pw_grid_t* grids, const pw_coeffs_t* coeffs, pw_batch_t* out) {
    if (!out) return bfail(PW_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || !grids || !coeffs) return bfail(PW_ERR_ARG, "need n >= 1 grids and coefficient sets");
    pw_batch_s* b = new (std::nothrow) pw_batch_s();
    if (!b) return bfail(PW_ERR_OOM, "host allocation of the batch failed");
    b->n = n;
    b->dtype = grids[0].dtype;
    // Starting tile (the autotuner refines it): 16-lane tiles when the cells
    // lie mostly in grids narrower than 256 columns, and for 16-bit storage
    // the packed two-row tile of 8 rows.  On the 512-grid batch (widths
    // 32..384): FP32 7.9 ms against 8.6 for 32 x 4; BF16 6.7 against 8.8.
    {
        double cells = 0.0, wx = 0.0;
        for (int q = 0; q < n; ++q) {
            const double c = (double)grids[q].nx * grids[q].ny * grids[q].nz;
            cells += c;
            wx += c * grids[q].nx;
        }
        b->cfg.lx = (cells > 0.0 && wx / cells < 256.0) ? 16 : 32;
        if (b->dtype != PW_F32) {
            b->cfg.ty = 8;
            b->cfg.rp = 2;
        }
    }
    size_t tz_total = 0;
    for (int q = 0; q < n; ++q) {
        pw_status_t s = validate_grid(&grids[q]);
        if (s != PW_OK) {
            delete b;
            return s;
        }
        if (grids[q].dtype != b->dtype) {
            delete b;
            return bfail(PW_ERR_ARG, "all grids of a batch must share one dtype");
        }
        int ox = 0;
        const char* why = "";
        if (!tma_layout_ok(grids[q], &ox, &why)) {
            delete b;
            return internal_fail(PW_ERR_UNSUPPORTED, "batch grid %d: layout not eligible for the k-march kernel (%s)",
                                 q, why);
        }
        const pw_coeffs_t& c = coeffs[q];
        if (!c.tzc1 || !c.tzc2 || !c.tzd1 || !c.tzd2) {
            delete b;
            return bfail(PW_ERR_ARG, "a vertical coefficient array is NULL");
        }
        b->grids.push_back(grids[q]);
        b->ox.push_back(ox);
        b->tcx.push_back((float)c.tcx);
        b->tcy.push_back((float)c.tcy);
        b->tz_off.push_back(tz_total);
        tz_total += 4 * (size_t)(grids[q].nz + 2);
        b->cells += (long long)grids[q].nx * grids[q].ny * grids[q].nz;
    }
    std::vector<float> tz(tz_total);
    for (int q = 0; q < n; ++q) {
        const int m = grids[q].nz + 2;
        float* t = tz.data() + b->tz_off[q];
        for (int k = 0; k < m; ++k) {
            t[k] = (float)coeffs[q].tzc1[k];
            t[m + k] = (float)coeffs[q].tzc2[k];
            t[2 * m + k] = (float)coeffs[q].tzd1[k];
            t[3 * m + k] = (float)coeffs[q].tzd2[k];
        }
    }
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = dev_malloc(&b->d_tz, tz.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tz, tz.data(), tz.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dev_malloc(&b->d_grids, n * sizeof(BatchGridDev));
    if (e == cudaSuccess) e = dev_malloc(&b->d_maps, 6 * (size_t)n * sizeof(CUtensorMap));
    if (e == cudaSuccess) e = dev_malloc(&b->d_counter, sizeof(int));
    if (e == cudaSuccess) e = dev_malloc(&b->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = host_malloc_pinned(&b->h_grids, n * sizeof(BatchGridDev));
    if (e == cudaSuccess) e = host_malloc_pinned(&b->h_maps, 6 * (size_t)n * sizeof(CUtensorMap));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        pw_batch_destroy(b);
        return internal_cuda_fail(e, "pw_batch_create");
    }
    pw_status_t s = build_items(b, b->cfg, 0, true);
    if (s != PW_OK) {
        pw_batch_destroy(b);
        return s;
    }
    *out = b;
    return PW_OK;
}

pw_status_t pw_batch_destroy(pw_batch_t b) {
    if (!b) return PW_OK;
    drop_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->d_tz);
    cudaFree(b->d_grids);
    cudaFree(b->d_maps);
    cudaFree(b->d_items);
    cudaFree(b->d_counter);
    cudaFree(b->d_err);
    cudaFreeHost(b->h_grids);
    cudaFreeHost(b->h_maps);
    delete b;
    return PW_OK;
}

pw_status_t pw_batch_set_config(pw_batch_t b, int32_t lanes_x, int32_t cells, int32_t ty, int32_t stages,
                                int32_t ctas_per_sm, int32_t rows_per_thread) {
    if (!b) return bfail(PW_ERR_ARG, "batch is NULL");
    if (rows_per_thread < 0 || rows_per_thread > 3)
        return bfail(PW_ERR_ARG, "rows_per_thread must be 0, 1, 2 or 3");
    TmaConfig c{lanes_x ? lanes_x : 32, ty ? ty : 4, stages ? stages : 4, 1};
    c.nc = cells ? cells : 4;
    c.rp = rows_per_thread ? rows_per_thread : 1;
    if (c.rp == 3) {
        c.rp = 1;
        c.xp = 1;
    }
    if (!batch_config_supported(c, b->dtype))
        return internal_fail(PW_ERR_UNSUPPORTED,
                             "no batched kernel instance for lanes_x=%d cells=%d ty=%d stages=%d rows_per_thread=%d "
                             "(dtype %d)",
                             c.lx, c.nc, c.ty, c.stages, rows_per_thread ? rows_per_thread : 1, (int)b->dtype);
    if (ctas_per_sm < 0) return bfail(PW_ERR_ARG, "ctas_per_sm must be >= 0");
    return build_items(b, c, ctas_per_sm, b->narrow_on);
}

pw_status_t pw_batch_set_narrow_columns(pw_batch_t b, int32_t enable) {
    if (!b) return bfail(PW_ERR_ARG, "batch is NULL");
    if (enable != 0 && enable != 1) return bfail(PW_ERR_ARG, "enable must be 0 or 1");
    return build_items(b, b->cfg, b->ctas_per_sm, enable != 0);
}

pw_status_t pw_batch_narrow_shape(pw_batch_t b, int32_t* lanes_x, int32_t* cells, int32_t* ty) {
    if (!b) return bfail(PW_ERR_ARG, "batch is NULL");
    if (lanes_x) *lanes_x = b->dual ? b->ncfg.lx : 0;
    if (cells) *cells = b->dual ? b->ncfg.nc : 0;
    if (ty) *ty = b->dual ? b->ncfg.ty : 0;
    return PW_OK;
}

pw_status_t pw_batch_info(pw_batch_t b, int64_t* n_items, int64_t* cells, int32_t* ctas) {
    if (!b) return bfail(PW_ERR_ARG, "batch is NULL");
    if (n_items) *n_items = (int64_t)b->items.size();
    if (cells) *cells = b->cells;
    if (ctas) *ctas = b->ctas;
    return PW_OK;
}

pw_status_t pw_batch_tendencies(pw_batch_t b, const void* const* u, const void* const* v, const void* const* w,
                                void* const* su, void* const* sv, void* const* sw, const float* scale,
                                pw_stream_t stream) {
    PW_RANGE("pw_batch_tendencies");
    if (!b) return bfail(PW_ERR_ARG, "batch is NULL");
    if (!b->items_ok || !b->d_items) return bfail(PW_ERR_ARG, "the batch has no work list");
    if (!u || !v || !w || !su || !sv || !sw) return bfail(PW_ERR_ARG, "a pointer table is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Scales sc;
    for (int q = 0; q < 3; ++q) {
        sc.in[q] = scale ? scale[q] : 1.f;
        sc.out[q] = scale ? scale[3 + q] : 1.f;
        if (!(sc.in[q] > 0.f) || !(sc.out[q] > 0.f) || !(sc.in[q] < 3.0e38f) || !(sc.out[q] < 3.0e38f))
            return bfail(PW_ERR_ARG, "scales must be finite and > 0");
    }
    // pointer tables: validate, and rebuild the device tables if they changed
    std::vector<const void*> p(6 * (size_t)b->n);
    for (int q = 0; q < b->n; ++q) {
        const void* f[6] = {u[q], v[q], w[q], su[q], sv[q], sw[q]};
        for (int a = 0; a < 6; ++a) {
            if (!f[a]) return bfail(PW_ERR_ARG, "a field pointer is NULL");
            if (!aligned16(f[a])) return bfail(PW_ERR_ALIGN, "batched fields must be 16-byte aligned");
            for (int c = 3; c < 6; ++c)
                if (a < 3 && f[a] == f[c]) return bfail(PW_ERR_ARG, "an output aliases an input");
            p[6 * (size_t)q + a] = f[a];
        }
    }
    if (!b->tables_ok || p != b->ptrs) {
        for (const void* f : p)   // a host address would fault the GPU
            if (!is_device_ptr(f, b->device)) return bfail(PW_ERR_ARG, "a field pointer is not device memory");
        // the pinned staging may still feed an earlier upload on this stream
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return internal_cuda_fail(e, "batch stream synchronize");
        const int mps = b->dual ? 6 : 3;   // tensor maps per grid
        for (int q = 0; q < b->n; ++q) {
            const pw_grid_t& g = b->grids[q];
            for (int a = 0; a < mps; ++a) {
                const TmaConfig& c = a < 3 ? b->cfg : b->ncfg;
                pw_status_t st = encode_tensor_map(g, p[6 * (size_t)q + a % 3], c.lx, c.ty,
                                                   &b->h_maps[mps * (size_t)q + a], c.nc, PW_BATCH_L2_PROMOTION);
                if (st != PW_OK) return st;
            }
            const TilePlan tp = tile_plan(g, b->cfg, b->dual ? &b->ncfg : nullptr);
            BatchGridDev& r = b->h_grids[q];
            r.g.nx = g.nx;
            r.g.ny = g.ny;
            r.g.nz = g.nz;
            r.g.halo = g.halo;
            r.g.pj = g.pitch_j;
            r.g.pk = g.pitch_k;
            r.g.origin = g.origin;
            r.ox = b->ox[q];
            r.tiles_x = tp.tx;
            r.tiles_y = tp.ty;
            r.ntiles_y = tp.nty;
            r.nbx = tp.nbx;
            r.nseg = 1;
            r.tcx = b->tcx[q];
            r.tcy = b->tcy[q];
            r.tz = b->d_tz + b->tz_off[q];
            for (int a = 0; a < 3; ++a) r.o[a] = const_cast<void*>(p[6 * (size_t)q + 3 + a]);
        }
        e = cudaMemcpyAsync(b->d_grids, b->h_grids, b->n * sizeof(BatchGridDev), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_maps, b->h_maps, mps * (size_t)b->n * sizeof(CUtensorMap),
                                cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return internal_cuda_fail(e, "batch table upload");
        b->ptrs = p;
        b->tables_ok = true;
    }
    // the graph: counter reset + persistent kernel, captured once per config and
    // per set of scales (the kernel's folded coefficients are launch parameters)
    if (b->exec && std::memcmp(&sc, &b->graph_sc, sizeof sc) != 0)
        drop_graph(b);
    if (!b->exec) {
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->cap);
        if (e == cudaSuccess)
            e = batch_dispatch(b->dtype, b->cfg, b->dual, false, nullptr, b->d_grids, b->d_maps, b->d_items,
                               (int)b->items.size(), b->d_counter, sc, b->d_err, b->ctas, b->cap);
        cudaGraph_t gr = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->cap, &gr);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, gr, 0);
        if (e != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            b->exec = nullptr;
            return internal_cuda_fail(e, "batch graph capture");
        }
        b->graph = gr;
        b->graph_sc = sc;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) return internal_cuda_fail(e, "batch graph launch");
    return PW_OK;
}

pw_status_t pw_batch_sync(pw_batch_t b, pw_stream_t stream) {
    if (!b) return bfail(PW_ERR_ARG, "batch is NULL");
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return internal_cuda_fail(e, "stream synchronize");
    int flag = 0;
    e = cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return internal_cuda_fail(e, "status word read");
    if (flag != DEV_OK) {
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        if (cudaMemsetAsync(b->d_err, 0, sizeof(int), s) == cudaSuccess) cudaStreamSynchronize(s);
        if (flag == DEV_OOB_STORE)
            return internal_fail(PW_ERR_CUDA,
                                 "a store outside the field's cells was caught and skipped (debug bounds build)");
        return internal_fail(PW_ERR_DEVICE_TIMEOUT, "a batched kernel gave up a bounded wait (code %d)", flag);
    }
    return PW_OK;
}

}  // extern "C"
