// Adjoint (transpose) of the PW scheme linearised about (u, v, w): the
// sensitivities of a scalar with respect to u, v, w given its sensitivities
// l = (lsu, lsv, lsw) with respect to the source terms (Sec. 2.2 defines the
// scheme; its transpose is what data assimilation and gradient-based
// training of the velocity fields need).
//
// Every term of the scheme has the shape c * a * (b + d) at an output cell X;
// its transpose sends c*l(X)*(b+d) to the slot of a and c*l(X)*a to the slots
// of b and d.  The kernel is written in GATHER form: one thread per input
// cell C collects, field by field, the contributions of every output X whose
// stencil touches C (up to nine per field), so no two threads write the same
// cell and no atomics are needed.  Output sensitivities outside the scheme's
// output set (levels other than 2..nz for su, sv and 2..nz-1 for sw; the
// upper vertical term only below the lid; lateral halo cells) are zero.
//
// Modes: full-array (C ranges over levels 1..nz of the interior plus the
// one-cell lateral halo; halo values of u, v, w are independent inputs), or
// periodic (C ranges over the interior; output cells wrap around the doubly
// periodic domain, which equals the full-array result folded back onto the
// interior; u, v, w must carry periodic halos).
#include <algorithm>

#include "pw_device.cuh"

#include <type_traits>
#include "pw_internal.h"

namespace pw {

struct AdjArgs {
    const float *u, *v, *w;        // linearisation point
    const float *lu, *lv, *lw;     // sensitivities to su, sv, sw
    float *gu, *gv, *gw;           // result
    float alpha;                   // g = [g or l or 0] + alpha * J^T l
    int accumulate, add_lambda, periodic;
};

__global__ void adjoint_gather_kernel(const GridDev g, const AdjArgs a, const CoefDev cf) {
    const int nx = g.nx, ny = g.ny, nz = g.nz, nzp2 = nz + 2;
    const int h = a.periodic ? 0 : 1;   // extra ring of cells covered in full-array mode
    const long long wx = nx + 2 * h, wy = ny + 2 * h;
    const long long total = wx * wy * nz;
    const float* tzc1 = cf.tz;
    const float* tzc2 = cf.tz + nzp2;
    const float* tzd1 = cf.tz + 2 * nzp2;
    const float* tzd2 = cf.tz + 3 * nzp2;
    const float tcx = cf.tcx, tcy = cf.tcy;

    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(idx % wx) + 1 - h;
        const int J = (int)((idx / wx) % wy) + 1 - h;
        const int K = 1 + (int)(idx / (wx * wy));
        auto off = [&](int k, int j, int i) { return g.origin + (long long)k * g.pk + (long long)j * g.pj + i; };
        auto U = [&](int k, int j, int i) { return __ldg(a.u + off(k, j, i)); };
        auto V = [&](int k, int j, int i) { return __ldg(a.v + off(k, j, i)); };
        auto W = [&](int k, int j, int i) { return __ldg(a.w + off(k, j, i)); };
        // output cell X = (k, j, i): is it an output of the scheme, and where
        // does its sensitivity live (wrapped in periodic mode)?
        auto out_ok = [&](int k, int j, int i, int klo, int khi, int& jj, int& ii) {
            if (k < klo || k > khi) return false;
            if (a.periodic) {
                jj = j < 1 ? j + ny : (j > ny ? j - ny : j);
                ii = i < 1 ? i + nx : (i > nx ? i - nx : i);
                return true;
            }
            jj = j;
            ii = i;
            return j >= 1 && j <= ny && i >= 1 && i <= nx;
        };
        // l at X for su (levels 2..nz), sv (2..nz), sw (2..nz-1); the upper
        // vertical terms of su, sv exist only below the lid (levels 2..nz-1)
        auto LU = [&](int k, int j, int i, int khi) {
            int jj, ii;
            return out_ok(k, j, i, 2, khi, jj, ii) ? __ldg(a.lu + off(k, jj, ii)) : 0.f;
        };
        auto LV = [&](int k, int j, int i, int khi) {
            int jj, ii;
            return out_ok(k, j, i, 2, khi, jj, ii) ? __ldg(a.lv + off(k, jj, ii)) : 0.f;
        };
        auto LW = [&](int k, int j, int i) {
            int jj, ii;
            return out_ok(k, j, i, 2, nz - 1, jj, ii) ? __ldg(a.lw + off(k, jj, ii)) : 0.f;
        };
        // c * l(X) * factor, with the factor's loads skipped when l(X) is absent
#define PW_ADD(acc, cexpr, lam, fexpr)         \
    do {                                       \
        const float l_ = (lam);                \
        if (l_ != 0.f) acc += (cexpr) * l_ * (fexpr); \
    } while (0)
        const int k = K, j = J, i = I;
        float ru = 0.f, rv = 0.f, rw = 0.f;

        // ---- gu: u(C) enters su (as a, b, d), sv (as b, d), sw (as b, d)
        PW_ADD(ru, tcx, LU(k, j, i + 1, nz), U(k, j, i + 1) + 2.f * U(k, j, i));
        PW_ADD(ru, tcx, LU(k, j, i, nz), U(k, j, i - 1));
        PW_ADD(ru, -tcx, LU(k, j, i - 1, nz), U(k, j, i - 1) + 2.f * U(k, j, i));
        PW_ADD(ru, -tcx, LU(k, j, i, nz), U(k, j, i + 1));
        PW_ADD(ru, tcy, LU(k, j + 1, i, nz), V(k, j, i) + V(k, j, i + 1));
        PW_ADD(ru, -tcy, LU(k, j - 1, i, nz), V(k, j - 1, i) + V(k, j - 1, i + 1));
        if (k + 1 <= nz) PW_ADD(ru, tzc1[k + 1], LU(k + 1, j, i, nz), W(k, j, i) + W(k, j, i + 1));
        if (k - 1 >= 2) PW_ADD(ru, -tzc2[k - 1], LU(k - 1, j, i, nz - 1), W(k - 1, j, i) + W(k - 1, j, i + 1));
        PW_ADD(ru, tcx, LV(k, j, i + 1, nz), V(k, j, i));
        PW_ADD(ru, tcx, LV(k, j - 1, i + 1, nz), V(k, j - 1, i));
        PW_ADD(ru, -tcx, LV(k, j, i, nz), V(k, j, i + 1));
        PW_ADD(ru, -tcx, LV(k, j - 1, i, nz), V(k, j - 1, i + 1));
        PW_ADD(ru, tcx, LW(k, j, i + 1), W(k, j, i));
        if (k - 1 >= 1) PW_ADD(ru, tcx, LW(k - 1, j, i + 1), W(k - 1, j, i));
        PW_ADD(ru, -tcx, LW(k, j, i), W(k, j, i + 1));
        if (k - 1 >= 1) PW_ADD(ru, -tcx, LW(k - 1, j, i), W(k - 1, j, i + 1));

        // ---- gv: v(C) enters su (as b, d), sv (as a, b, d), sw (as b, d)
        PW_ADD(rv, tcy, LU(k, j + 1, i, nz), U(k, j, i));
        PW_ADD(rv, tcy, LU(k, j + 1, i - 1, nz), U(k, j, i - 1));
        PW_ADD(rv, -tcy, LU(k, j, i, nz), U(k, j + 1, i));
        PW_ADD(rv, -tcy, LU(k, j, i - 1, nz), U(k, j + 1, i - 1));
        PW_ADD(rv, tcx, LV(k, j, i + 1, nz), U(k, j, i) + U(k, j + 1, i));
        PW_ADD(rv, -tcx, LV(k, j, i - 1, nz), U(k, j, i - 1) + U(k, j + 1, i - 1));
        PW_ADD(rv, tcy, LV(k, j + 1, i, nz), V(k, j + 1, i) + 2.f * V(k, j, i));
        PW_ADD(rv, tcy, LV(k, j, i, nz), V(k, j - 1, i));
        PW_ADD(rv, -tcy, LV(k, j - 1, i, nz), V(k, j - 1, i) + 2.f * V(k, j, i));
        PW_ADD(rv, -tcy, LV(k, j, i, nz), V(k, j + 1, i));
        if (k + 1 <= nz) PW_ADD(rv, tzc1[k + 1], LV(k + 1, j, i, nz), W(k, j, i) + W(k, j + 1, i));
        if (k - 1 >= 2) PW_ADD(rv, -tzc2[k - 1], LV(k - 1, j, i, nz - 1), W(k - 1, j, i) + W(k - 1, j + 1, i));
        PW_ADD(rv, tcy, LW(k, j + 1, i), W(k, j, i));
        if (k - 1 >= 1) PW_ADD(rv, tcy, LW(k - 1, j + 1, i), W(k - 1, j, i));
        PW_ADD(rv, -tcy, LW(k, j, i), W(k, j + 1, i));
        if (k - 1 >= 1) PW_ADD(rv, -tcy, LW(k - 1, j, i), W(k - 1, j + 1, i));

        // ---- gw: w(C) enters su (as b, d), sv (as b, d), sw (as a, b, d)
        if (k + 1 <= nz) {
            PW_ADD(rw, tzc1[k + 1], LU(k + 1, j, i, nz), U(k, j, i));
            PW_ADD(rw, tzc1[k + 1], LU(k + 1, j, i - 1, nz), U(k, j, i - 1));
            PW_ADD(rw, tzc1[k + 1], LV(k + 1, j, i, nz), V(k, j, i));
            PW_ADD(rw, tzc1[k + 1], LV(k + 1, j - 1, i, nz), V(k, j - 1, i));
            PW_ADD(rw, -tzc2[k], LU(k, j, i, nz - 1), U(k + 1, j, i));
            PW_ADD(rw, -tzc2[k], LU(k, j, i - 1, nz - 1), U(k + 1, j, i - 1));
            PW_ADD(rw, -tzc2[k], LV(k, j, i, nz - 1), V(k + 1, j, i));
            PW_ADD(rw, -tzc2[k], LV(k, j - 1, i, nz - 1), V(k + 1, j - 1, i));
            PW_ADD(rw, tcx, LW(k, j, i + 1), U(k, j, i) + U(k + 1, j, i));
            PW_ADD(rw, -tcx, LW(k, j, i - 1), U(k, j, i - 1) + U(k + 1, j, i - 1));
            PW_ADD(rw, tcy, LW(k, j + 1, i), V(k, j, i) + V(k + 1, j, i));
            PW_ADD(rw, -tcy, LW(k, j - 1, i), V(k, j - 1, i) + V(k + 1, j - 1, i));
            PW_ADD(rw, tzd1[k + 1], LW(k + 1, j, i), W(k + 1, j, i) + 2.f * W(k, j, i));
            PW_ADD(rw, -tzd2[k], LW(k, j, i), W(k + 1, j, i));
        }
        PW_ADD(rw, tzd1[k], LW(k, j, i), W(k - 1, j, i));
        if (k - 1 >= 2) PW_ADD(rw, -tzd2[k - 1], LW(k - 1, j, i), W(k - 1, j, i) + 2.f * W(k, j, i));
#undef PW_ADD

        const long long c = off(K, J, I);
        float bu = 0.f, bv = 0.f, bw = 0.f;
        if (a.accumulate) {
            bu = a.gu[c];
            bv = a.gv[c];
            bw = a.gw[c];
        } else if (a.add_lambda) {
            bu = a.lu[c];
            bv = a.lv[c];
            bw = a.lw[c];
        }
        a.gu[c] = fmaf(a.alpha, ru, bu);
        a.gv[c] = fmaf(a.alpha, rv, bv);
        a.gw[c] = fmaf(a.alpha, rw, bw);
    }
}

// ---------------------------------------------------------------------------
// TMA k-march adjoint (periodic mode, FP32).  A CTA owns 32*NA columns x TY
// rows of the interior (NA cells per thread); one thread issues 3D TMA copies
// of the u, v, w and lsu, lsv, lsw planes (tile plus one-cell halo) into a
// ring of S slots, keeping levels k-1, k, k+1 resident while S-3 more are in
// flight.  The halos of u, v, w and of l must hold periodic images.
constexpr int kAdjPAD = 4;                       // 16-byte granule of FP32

template <int NA, int TY, int S>
struct AdjLayout {
    static_assert(NA == 2 || NA == 4, "2 or 4 cells per thread");
    static constexpr int TX = 32 * NA;
    static constexpr int BW = TX + 2 * kAdjPAD;
    static constexpr int ROWS = TY + 2;
    static constexpr int FIELD_RAW = BW * ROWS;
    static constexpr int FIELD = ((FIELD_RAW * 4 + 127) / 128) * 32;   // floats, 128-byte multiple
    static constexpr int STAGE = 6 * FIELD;
    static constexpr uint32_t TX_BYTES = 6u * FIELD_RAW * 4u;
    // the ring, one mbarrier per slot, 4 flag words, one release counter per slot
    // the vertical coefficients {tzc1, tzc2, tzd1, tzd2} of levels kb-1..ke+1
    // of the CTA's k segment, one float4 per level (the host keeps a segment
    // within CTZ_LEVELS - 2 levels)
    static constexpr int CTZ_LEVELS = 256;
    static constexpr size_t CTZ_OFF = (((size_t)S * STAGE * 4 + S * sizeof(uint64_t) + 16 + 4 * S + 15) / 16) * 16;
    static constexpr size_t SMEM = CTZ_OFF + (size_t)CTZ_LEVELS * sizeof(float4);
};

struct AdjMaps {
    CUtensorMap m[6];   // u, v, w, lsu, lsv, lsw
};

// NA consecutive floats at a 4*NA-byte aligned address
template <int NA>
__device__ __forceinline__ void adj_ldv(const float* p, float (&o)[NA]) {
    if constexpr (NA == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        o[0] = t.x;
        o[1] = t.y;
        o[2] = t.z;
        o[3] = t.w;
    } else {
        const float2 t = *reinterpret_cast<const float2*>(p);
        o[0] = t.x;
        o[1] = t.y;
    }
}
template <int NA>
__device__ __forceinline__ void adj_stv(float* p, const float (&v)[NA]) {
    if constexpr (NA == 4)
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
}

// How a ring slot is handed back after a level: 0 = a CTA barrier, then one
// thread refills it; 1 = each warp counts itself out on the slot (an
// acquire-release atomic) and the last one refills it, so warps need not
// wait for each other at every level.  On GB300 the barrier was faster
// (4 x 6 shape, 512^2 / 1024^2 / 2048^2 x 64: 93.5 / 113.8 / 121.1 against
// 91.1 / 109.5 / 115.7 Gcell/s, same box), as in the forward k-march: with
// three resident levels and four slots a warp can run at most one level
// ahead anyway.
#ifndef PW_ADJ_SPLIT_ARRIVE
#define PW_ADJ_SPLIT_ARRIVE 0
#endif
// The first planes of a tile issued before (1) or after (0) the CTA fills its
// table of vertical coefficients (4 x 6 shape: 98.5 against 96.4 Gcell/s at
// 512^2 x 64, 127.8 against 127.0 at 2048^2, same box).
#ifndef PW_ADJ_ISSUE_FIRST
#define PW_ADJ_ISSUE_FIRST 1
#endif

// CTAs per SM a shape's register budget is sized for: what shared memory
// allows, at most 2 for 4 cells a thread (their gather needs 165-182
// registers), and for 2 cells as many as leave each thread >= 96 registers
// (the gather of 2 cells needs about that many without spilling).
template <int NA, int TY, int S>
constexpr int adj_min_blocks() {
    constexpr int by_smem = (int)((227u * 1024u) / AdjLayout<NA, TY, S>::SMEM);
    constexpr int cap = NA == 4 ? 2 : 65536 / (32 * TY * 96);
    constexpr int m = by_smem < cap ? by_smem : cap;
    return m < 1 ? 1 : m;
}

// ---------------------------------------------------------------------------
// The gather kernel on that ring: a thread owns NA consecutive cells of one
// row, so each (field, level, row) it needs is one 16-byte (NA = 4) or
// 8-byte (NA = 2) shared load for all of them, and the x neighbours come from
// the adjacent lanes by warp shuffles (the row's end lanes read theirs from
// the halo columns), as in the forward k-march: 30 vector loads per level.  (Four cells 32 columns
// apart, read one word at a time, took about 200 scalar loads per level and
// ran at 58 against 79 Gcell/s on GB300.)  Levels 3..nz-2 have every term and run without any masking; the
// others select away the terms that do not exist there (a select, not a
// multiplication by zero, so values read from a slot that holds another
// level, or a sensitivity outside the scheme's outputs, never reach a sum).
template <int NA, int TY, int S>
__global__ void __launch_bounds__(32 * TY, adj_min_blocks<NA, TY, S>())
    adjoint_vec_kernel(const __grid_constant__ AdjMaps maps, float* __restrict__ gu, float* __restrict__ gv,
                       float* __restrict__ gw, const GridDev g, const int ox, const int nseg, const CoefDev cf,
                       const float alpha, const int accumulate, const int add_lambda, int* __restrict__ err) {
    using L = AdjLayout<NA, TY, S>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* stages = reinterpret_cast<float*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)S * L::STAGE * 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + S);   // [0] abort, [1] planes issued
    uint32_t* cnt = reinterpret_cast<uint32_t*>(bars + S) + 4;              // warps done with each slot

    const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
    const int nz = g.nz, nzp2 = nz + 2;
    const int kb = 1 + (int)(((long long)blockIdx.z * nz) / nseg);
    const int ke = (int)(((long long)(blockIdx.z + 1) * nz) / nseg);
    if (ke < kb) return;
    const int pb = max(kb - 1, 1), pe = min(ke + 1, nz), np = pe - pb + 1;
    const int X0 = ox + 1 + L::TX * blockIdx.x - kAdjPAD;
    const int Y0 = TY * blockIdx.y + g.halo - 1;

    auto issue = [&](int p) {
        const int s = p % S;
        float* dst = stages + s * L::STAGE;
        mbar_arrive_expect_tx(&bars[s], L::TX_BYTES);
        for (int f = 0; f < 6; ++f) tma_load_3d(dst + f * L::FIELD, &maps.m[f], X0, Y0, pb + p, &bars[s]);
    };
    int issued = 0;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&bars[s], 1);
            cnt[s] = 0;
        }
        abort_flag[0] = 0;
        fence_mbar_init();
    }
    // the first planes go out before the coefficient table is filled, so that
    // their DRAM latency overlaps the table's loads (the other threads wait
    // on the planes' mbarriers only after the CTA barrier below)
    if (PW_ADJ_ISSUE_FIRST && tid == 0) {
        for (int f = 0; f < 6; ++f) prefetch_tensormap(&maps.m[f]);
        for (; issued < S && issued < np; ++issued) issue(issued);
        abort_flag[1] = issued;
    }
    float4* const ctz = reinterpret_cast<float4*>(smem_raw + L::CTZ_OFF);   // entry k - (kb-1): level k
    for (int e = tid; e <= ke - kb + 2; e += 32 * TY) {
        const int k = kb - 1 + e;
        ctz[e] = make_float4(__ldg(cf.tz + k), __ldg(cf.tz + nzp2 + k), __ldg(cf.tz + 2 * nzp2 + k),
                             __ldg(cf.tz + 3 * nzp2 + k));
    }
    __syncthreads();
    if (!PW_ADJ_ISSUE_FIRST && tid == 0) {
        for (int f = 0; f < 6; ++f) prefetch_tensormap(&maps.m[f]);
        for (; issued < S && issued < np; ++issued) issue(issued);
        abort_flag[1] = issued;
    }

    const float tcx = cf.tcx, tcy = cf.tcy;
    const int r = ty + 1;
    const int c0 = kAdjPAD + NA * lane;
    // tile-edge neighbour column: lane 0 needs x = -1, lane 31 x = TX; the
    // other lanes read lane 31's address (a broadcast)
    const int ce = (lane == 0) ? kAdjPAD - 1 : kAdjPAD + L::TX;
    const int J = TY * blockIdx.y + 1 + ty;
    const int I0 = 1 + L::TX * blockIdx.x + NA * lane;
    const bool valid = (J <= g.ny) && (I0 <= g.nx);
    const unsigned FULL = 0xffffffffu;
    int waited = 0;
    bool aborted = false;
    for (int K = kb; K <= ke; ++K) {
        const int lp = K - pb;
        bool ok = true;
        const int need_hi = (K + 1 <= pe) ? lp + 1 : lp;
        for (int p = (K == kb ? 0 : need_hi); p <= need_hi && ok; ++p)
            ok = mbar_wait_bounded(&bars[p % S], (uint32_t)((p / S) & 1), kWaitLimitNs);
        ok = __all_sync(FULL, ok);
        if (!ok) abort_flag[0] = 1;
        if (ok) {
            waited = need_hi + 1;
            const float* Pm = stages + ((lp - 1 + S) % S) * L::STAGE;   // level K-1 (valid when K-1 >= pb)
            const float* P0 = stages + (lp % S) * L::STAGE;             // level K
            const float* Pp = stages + ((lp + 1) % S) * L::STAGE;       // level K+1 (valid when K+1 <= pe)
            // X[0..NA+1] = the row at x = -1..NA relative to the thread's first cell
            auto row = [&](const float* P, int f, int dj, float (&X)[NA + 2], bool lo, bool hi) {
                const float* q = P + f * L::FIELD + (r + dj) * L::BW;
                if constexpr (NA == 4) {
                    const float4 t = *reinterpret_cast<const float4*>(q + c0);
                    X[1] = t.x;
                    X[2] = t.y;
                    X[3] = t.z;
                    X[4] = t.w;
                } else {
                    const float2 t = *reinterpret_cast<const float2*>(q + c0);
                    X[1] = t.x;
                    X[2] = t.y;
                }
                X[0] = X[NA + 1] = 0.f;
                if (lo || hi) {
                    const float e = q[ce];
                    if (lo) {
                        const float m = __shfl_up_sync(FULL, X[NA], 1);
                        X[0] = lane == 0 ? e : m;
                    }
                    if (hi) {
                        const float pv = __shfl_down_sync(FULL, X[1], 1);
                        X[NA + 1] = lane == 31 ? e : pv;
                    }
                }
            };
            // rows: [L]ambda or field, level (0: K, p: K+1, m: K-1), row (m, z, p: j-1, j, j+1)
            float LU0m[NA + 2], LU0z[NA + 2], LU0p[NA + 2], LUpz[NA + 2], LUmz[NA + 2];
            float LV0m[NA + 2], LV0z[NA + 2], LV0p[NA + 2], LVpz[NA + 2], LVpm[NA + 2], LVmz[NA + 2];
            float LW0m[NA + 2], LW0z[NA + 2], LW0p[NA + 2], LWmz[NA + 2], LWmp[NA + 2], LWpz[NA + 2];
            float U0z[NA + 2], U0p[NA + 2], Upz[NA + 2];
            float V0m[NA + 2], V0z[NA + 2], V0p[NA + 2], Vpz[NA + 2], Vpm[NA + 2];
            float W0z[NA + 2], W0p[NA + 2], Wmz[NA + 2], Wmp[NA + 2], Wpz[NA + 2];
            row(P0, 3, -1, LU0m, false, false);
            row(P0, 3, 0, LU0z, true, true);
            row(P0, 3, 1, LU0p, true, false);
            row(Pp, 3, 0, LUpz, true, false);
            row(Pm, 3, 0, LUmz, false, false);
            row(P0, 4, -1, LV0m, false, true);
            row(P0, 4, 0, LV0z, true, true);
            row(P0, 4, 1, LV0p, false, false);
            row(Pp, 4, 0, LVpz, false, false);
            row(Pp, 4, -1, LVpm, false, false);
            row(Pm, 4, 0, LVmz, false, false);
            row(P0, 5, -1, LW0m, false, false);
            row(P0, 5, 0, LW0z, true, true);
            row(P0, 5, 1, LW0p, false, false);
            row(Pm, 5, 0, LWmz, false, true);
            row(Pm, 5, 1, LWmp, false, false);
            row(Pp, 5, 0, LWpz, false, false);
            row(P0, 0, 0, U0z, true, true);
            row(P0, 0, 1, U0p, true, false);
            row(Pp, 0, 0, Upz, true, false);
            row(P0, 1, -1, V0m, false, true);
            row(P0, 1, 0, V0z, false, true);
            row(P0, 1, 1, V0p, false, false);
            row(Pp, 1, 0, Vpz, false, false);
            row(Pp, 1, -1, Vpm, false, false);
            row(P0, 2, 0, W0z, false, true);
            row(P0, 2, 1, W0p, false, false);
            row(Pm, 2, 0, Wmz, false, true);
            row(Pm, 2, 1, Wmp, false, false);
            row(Pp, 2, 0, Wpz, false, false);

            // (loading these here, after the level's rows, measured 3-5 % faster
            // on GB300 than loading them before the plane wait or one level ahead)
            const bool has_m = (K - 1 >= 1), has_p = (K + 1 <= nz);
            const float4 zm = ctz[K - kb], z0 = ctz[K - kb + 1], zp = ctz[K - kb + 2];   // levels K-1, K, K+1
            const float c1p = has_p ? zp.x : 0.f, c2m = has_m ? zm.y : 0.f, c2 = z0.y;
            const float d1p = has_p ? zp.z : 0.f, d1 = z0.z, d2 = z0.w;
            const float d2m = has_m ? zm.w : 0.f;
            float ru[NA], rv[NA], rw[NA];

            // the gather of one level; EDGE: levels where some terms do not exist
            auto body = [&](auto edge_tag) {
                constexpr bool EDGE = decltype(edge_tag)::value;
                // sensitivities exist at output levels 2..nz (su, sv; upper terms
                // 2..nz-1) and 2..nz-1 (sw)
                const bool lu0 = (K >= 2), lw0 = (K >= 2 && K <= nz - 1);
                const bool lutm = (K - 1 >= 2 && K - 1 <= nz - 1), lwm = lutm, lup = (K + 1 <= nz);
                const bool lwp = (K + 1 >= 2 && K + 1 <= nz - 1);
                const bool pu = has_p && lup, mu = has_m && lutm, mw = has_m && lwm, pw = has_p && lwp;
                auto keep = [](bool c, float t) { return EDGE ? (c ? t : 0.f) : t; };
                if (EDGE) {   // sensitivities of level K outside the scheme's outputs are ignored
#pragma unroll
                    for (int x = 0; x < NA + 2; ++x) {
                        LU0m[x] = keep(lu0, LU0m[x]);
                        LU0z[x] = keep(lu0, LU0z[x]);
                        LU0p[x] = keep(lu0, LU0p[x]);
                        LV0m[x] = keep(lu0, LV0m[x]);
                        LV0z[x] = keep(lu0, LV0z[x]);
                        LV0p[x] = keep(lu0, LV0p[x]);
                        LW0m[x] = keep(lw0, LW0m[x]);
                        LW0z[x] = keep(lw0, LW0z[x]);
                        LW0p[x] = keep(lw0, LW0p[x]);
                    }
                }
                // Each output's terms are grouped by their coefficient, so a
                // coefficient multiplies a group's sum once instead of every
                // term; products that two neighbouring cells share are formed
                // once for the row: index x of the X arrays, cell o = c + 1
                // uses x = o - 1 and o.
                float D[NA + 1], Q[NA + 1], F[NA + 1], G[NA + 1], R[NA + 1];
#pragma unroll
                for (int x = 0; x <= NA; ++x) {
                    D[x] = fmaf(LU0p[x], U0z[x], -LU0z[x] * U0p[x]);   // sv's y-pair terms, as seen from v
                    Q[x] = U0z[x] + U0p[x];                            // u(j) + u(j+1)
                    F[x] = LUpz[x] * U0z[x];                           // su's upper term at k+1, as seen from w
                    G[x] = LU0z[x] * Upz[x];                           // su's upper term at k, as seen from w
                    R[x] = U0z[x] + Upz[x];                            // u(k) + u(k+1)
                }
#pragma unroll
                for (int c = 0; c < NA; ++c) {
                    const int o = c + 1;   // the cell in the X arrays; o-1 and o+1 its x neighbours
                    // ---- gu: u(C) in su (as a, b, d), sv and sw (as b, d)
                    float ax = LU0z[o + 1] * fmaf(2.f, U0z[o], U0z[o + 1]);
                    ax = fmaf(-LU0z[o - 1], fmaf(2.f, U0z[o], U0z[o - 1]), ax);
                    ax = fmaf(LU0z[o], U0z[o - 1] - U0z[o + 1], ax);
                    ax = fmaf(LV0z[o + 1], V0z[o], ax);
                    ax = fmaf(-LV0z[o], V0z[o + 1], ax);
                    ax = fmaf(LV0m[o + 1], V0m[o], ax);
                    ax = fmaf(-LV0m[o], V0m[o + 1], ax);
                    ax = fmaf(LW0z[o + 1], W0z[o], ax);
                    ax = fmaf(-LW0z[o], W0z[o + 1], ax);
                    ax += keep(mw, fmaf(LWmz[o + 1], Wmz[o], -LWmz[o] * Wmz[o + 1]));
                    const float ay = fmaf(LU0p[o], V0z[o] + V0z[o + 1], -LU0m[o] * (V0m[o] + V0m[o + 1]));
                    const float az = keep(pu, c1p * LUpz[o] * (W0z[o] + W0z[o + 1])) -
                                     keep(mu, c2m * LUmz[o] * (Wmz[o] + Wmz[o + 1]));
                    ru[c] = fmaf(tcx, ax, fmaf(tcy, ay, az));
                    // ---- gv: v(C) in su (as b, d), sv (as a, b, d), sw (as b, d)
                    const float bx = fmaf(LV0z[o + 1], Q[o], -LV0z[o - 1] * Q[o - 1]);
                    float by = D[o] + D[o - 1];
                    by = fmaf(LV0p[o], fmaf(2.f, V0z[o], V0p[o]), by);
                    by = fmaf(-LV0m[o], fmaf(2.f, V0z[o], V0m[o]), by);
                    by = fmaf(LV0z[o], V0m[o] - V0p[o], by);
                    by = fmaf(LW0p[o], W0z[o], by);
                    by = fmaf(-LW0z[o], W0p[o], by);
                    by += keep(mw, fmaf(LWmp[o], Wmz[o], -LWmz[o] * Wmp[o]));
                    const float bz = keep(pu, c1p * LVpz[o] * (W0z[o] + W0p[o])) -
                                     keep(mu, c2m * LVmz[o] * (Wmz[o] + Wmp[o]));
                    rv[c] = fmaf(tcx, bx, fmaf(tcy, by, bz));
                    // ---- gw: w(C) in su, sv (as b, d), sw (as a, b, d)
                    float e1 = F[o] + F[o - 1];
                    e1 = fmaf(LVpz[o], V0z[o], e1);
                    e1 = fmaf(LVpm[o], V0m[o], e1);
                    float e2 = G[o] + G[o - 1];
                    e2 = fmaf(LV0z[o], Vpz[o], e2);
                    e2 = fmaf(LV0m[o], Vpm[o], e2);
                    const float ex = fmaf(LW0z[o + 1], R[o], -LW0z[o - 1] * R[o - 1]);
                    const float ey = fmaf(LW0p[o], V0z[o] + Vpz[o], -LW0m[o] * (V0m[o] + Vpm[o]));
                    float t = keep(has_p, fmaf(tcx, ex, fmaf(tcy, ey, fmaf(-c2, e2, -d2 * LW0z[o] * Wpz[o]))));
                    t += keep(pu, c1p * e1);
                    t += keep(pw, d1p * LWpz[o] * fmaf(2.f, W0z[o], Wpz[o]));
                    t += keep(has_m, d1 * LW0z[o] * Wmz[o]);
                    t -= keep(mw, d2m * LWmz[o] * fmaf(2.f, W0z[o], Wmz[o]));
                    rw[c] = t;
                }
            };
            if (K >= 3 && K <= nz - 2)
                body(std::false_type{});
            else
                body(std::true_type{});

            if (valid) {
                const long long o = g.origin + (long long)K * g.pk + (long long)J * g.pj + I0;
                float bu[NA], bv[NA], bw[NA];
                if (accumulate) {
                    adj_ldv<NA>(gu + o, bu);
                    adj_ldv<NA>(gv + o, bv);
                    adj_ldv<NA>(gw + o, bw);
                } else if (add_lambda) {   // the raw sensitivities of level K
                    const float* q = P0 + r * L::BW + c0;
                    adj_ldv<NA>(q + 3 * L::FIELD, bu);
                    adj_ldv<NA>(q + 4 * L::FIELD, bv);
                    adj_ldv<NA>(q + 5 * L::FIELD, bw);
                } else {
#pragma unroll
                    for (int c = 0; c < NA; ++c) bu[c] = bv[c] = bw[c] = 0.f;
                }
#pragma unroll
                for (int c = 0; c < NA; ++c) {
                    bu[c] = fmaf(alpha, ru[c], bu[c]);
                    bv[c] = fmaf(alpha, rv[c], bv[c]);
                    bw[c] = fmaf(alpha, rw[c], bw[c]);
                }
                adj_stv<NA>(gu + o, bu);
                adj_stv<NA>(gv + o, bv);
                adj_stv<NA>(gw + o, bw);
            }
        }
#if PW_ADJ_SPLIT_ARRIVE
        // this warp is done with plane lp-1 (level K-1); the last warp to say
        // so refills its slot with plane lp-1+S
        __syncwarp();
        if (lane == 0 && ok && lp >= 1) {
            const int s = (lp - 1) % S;
            if (atom_add_acq_rel_cta(&cnt[s], 1u) == (uint32_t)(TY - 1)) {
                cnt[s] = 0;
                const int p = lp - 1 + S;
                if (p < np) {
                    fence_proxy_async_smem();
                    issue(p);
                    atomicMax(const_cast<int*>(&abort_flag[1]), p + 1);
                }
            }
        }
        if (abort_flag[0]) {
            aborted = true;
            break;
        }
#else
        __syncthreads();
        if (abort_flag[0]) {
            aborted = true;
            break;
        }
        // level K-1 is no longer needed: refill its slot
        if (tid == 0 && lp >= 1 && issued < np) {
            fence_proxy_async_smem();
            issue(issued);
            ++issued;
        }
#endif
    }
#if PW_ADJ_SPLIT_ARRIVE
    // every warp has left the march (each wait is bounded): an abort by any
    // warp is visible, and only the last S planes issued can be in flight
    __syncthreads();
    aborted = abort_flag[0] != 0;
    if (aborted && tid == 0) {
        report_error(err, DEV_TIMEOUT_TMA_WAIT);
        const int hi = abort_flag[1];
        for (int p = max(hi - S, 0); p < hi; ++p) mbar_wait_bounded(&bars[p % S], (p / S) & 1, kDrainLimitNs);
    }
    (void)waited;
#else
    if (aborted && tid == 0) {
        report_error(err, DEV_TIMEOUT_TMA_WAIT);
        for (int p = waited; p < issued; ++p)
            if (!mbar_wait_bounded(&bars[p % S], (p / S) & 1, kDrainLimitNs)) break;
    }
#endif
}

// Instantiated launch shapes (cells per thread, rows per CTA, ring slots;
// levels k-1, k, k+1 resident, the rest in flight).  Measured on GB300 with
// the automatic k segments, Gcell/s at 512^2 / 1024^2 / 2048^2 x 64:
//   4 cells: 4 rows 85.4 / 99.3 / 105.3, 5 rows 82.4 / 97.8 / 103.3,
//            6 rows 93.9 / 113.8 / 121.3 (two CTAs of 6 warps per SM);
//   2 cells: 4 rows 90.1 / 105.9 / 111.7, 5 rows 90.2 / 103.4 / 110.1,
//            6 rows 84.5 / 98.7 / 104.0, 8 rows 82.4 / 95.1 / 102.5;
// 3 slots (no plane in flight beyond k+1) lose a third; 5 slots (two planes
// in flight) gain nothing (4 x 4: 88.4 against 90.6, 2 x 8: 87.8 against
// 86.3, 2 x 6: 91.0 against 90.8 at 512^2), so the march does not wait on
// its planes' DRAM latency.  Two cells a
// thread halve the registers (96 against 165-182) and double the warps per
// SM, but that gains little: the gather is not bound by latency alone.
#define PW_ADJ_CONFIGS(X) X(4, 5, 4) X(4, 4, 4) X(4, 6, 4) X(2, 4, 4) X(2, 5, 4) X(2, 6, 4) X(2, 8, 4) X(2, 8, 3)

// The automatic shape (the fastest measured).
#ifndef PW_ADJ_NA
#define PW_ADJ_NA 4
#endif
#ifndef PW_ADJ_TY
#define PW_ADJ_TY 6
#endif
#ifndef PW_ADJ_S
#define PW_ADJ_S 4
#endif

AdjConfig adjoint_default_config() { return AdjConfig{PW_ADJ_NA, PW_ADJ_TY, PW_ADJ_S, 0}; }

bool adjoint_config_supported(const AdjConfig& c) {
#define PW_AS(NA_, TY_, S_) \
    if (c.na == NA_ && c.ty == TY_ && c.stages == S_) return true;
    PW_ADJ_CONFIGS(PW_AS)
#undef PW_AS
    return false;
}

int adjoint_blocks_per_sm(const AdjConfig& c) {
    int n = 0;
#define PW_AO(NA_, TY_, S_)                                                                                 \
    if (c.na == NA_ && c.ty == TY_ && c.stages == S_) {                                                    \
        auto kern = adjoint_vec_kernel<NA_, TY_, S_>;                                                      \
        using L = AdjLayout<NA_, TY_, S_>;                                                                 \
        if (set_smem_attr_once(kern, (int)L::SMEM) != cudaSuccess) return 0;                               \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 32 * TY_, L::SMEM) != cudaSuccess) return 0; \
        return n;                                                                                          \
    }
    PW_ADJ_CONFIGS(PW_AO)
#undef PW_AO
    return 0;
}

template <int NA, int TY, int S>
static cudaError_t launch_adj_inst(const GridDev& g, int ox, const AdjMaps& m, float* gu, float* gv, float* gw,
                                   float alpha, int accumulate, int add_lambda, const CoefDev& cf, int nseg, int* err,
                                   cudaStream_t s) {
    using L = AdjLayout<NA, TY, S>;
    auto kern = adjoint_vec_kernel<NA, TY, S>;
    cudaError_t e = set_smem_attr_once(kern, (int)L::SMEM);
    if (e != cudaSuccess) return e;
    nseg = std::max(nseg, (g.nz + L::CTZ_LEVELS - 3) / (L::CTZ_LEVELS - 2));   // segments within the table
    dim3 grid((g.nx + L::TX - 1) / L::TX, (g.ny + TY - 1) / TY, nseg);
    kern<<<grid, dim3(32, TY), L::SMEM, s>>>(m, gu, gv, gw, g, ox, nseg, cf, alpha, accumulate, add_lambda, err);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_tma(const GridDev& g, int ox, const CUtensorMap* maps6, float* gu, float* gv, float* gw,
                               float alpha, int accumulate, int add_lambda, const CoefDev& cf, int nseg, int* err,
                               const AdjConfig& c, cudaStream_t s) {
    AdjMaps m;
    for (int f = 0; f < 6; ++f) m.m[f] = maps6[f];
#define PW_AD(NA_, TY_, S_)                                                                                   \
    if (c.na == NA_ && c.ty == TY_ && c.stages == S_)                                                         \
        return launch_adj_inst<NA_, TY_, S_>(g, ox, m, gu, gv, gw, alpha, accumulate, add_lambda, cf, nseg, err, s);
    PW_ADJ_CONFIGS(PW_AD)
#undef PW_AD
    return cudaErrorInvalidConfiguration;
}

cudaError_t launch_adjoint(const GridDev& g, const float* u, const float* v, const float* w, const float* lu,
                           const float* lv, const float* lw, float* gu, float* gv, float* gw, float alpha,
                           int accumulate, int add_lambda, int periodic, const CoefDev& cf, int num_sms,
                           cudaStream_t s) {
    AdjArgs a{u, v, w, lu, lv, lw, gu, gv, gw, alpha, accumulate, add_lambda, periodic};
    const int hh = periodic ? 0 : 1;
    const long long total = (long long)(g.nx + 2 * hh) * (g.ny + 2 * hh) * g.nz;
    const int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > (long long)num_sms * 16) blocks = (long long)num_sms * 16;
    if (blocks < 1) blocks = 1;
    adjoint_gather_kernel<<<(unsigned)blocks, threads, 0, s>>>(g, a, cf);
    return cudaGetLastError();
}

}  // namespace pw
