// PW stencil kernels (Sec. 2.2; per-cell arithmetic shape Sec. 4), templated
// on the storage type T and on what the epilogue does with the source terms:
//   MODE_TEND: store su, sv, sw;
//   MODE_STEP: store the forward-Euler update q + dt*s of u, v, w, together
//              with the periodic images of the boundary cells in the lateral
//              halo, so the next step reads a complete halo.
// Instantiated by pw_tend.cu (MODE_TEND) and pw_step.cu (MODE_STEP).
#pragma once

#include "pw_device.cuh"
#include "pw_internal.h"

namespace pw {

enum { MODE_TEND = 0, MODE_STEP = 1 };

// Debug bounds build (PW_DEBUG_BOUNDS=1): every global store of the k-march
// and two-step kernels first checks that its cells lie where the kernel may
// write (layout_cells_ok: levels 1..nz, the interior for source terms and
// state, the lateral halo for periodic images, never row padding); a store
// that does not is skipped and recorded in the status word (DEV_OOB_STORE,
// reported by pw_sync).  Nothing is asserted, so a caught store never traps.
// (PW_DEBUG_BOUNDS defaults to 0 in pw_internal.h.)
// false (and the store is to be skipped) when the debug build catches it
__device__ __forceinline__ bool dbg_store(const GridDev& g, long long o, int n, bool interior_only, int* err) {
    if constexpr (PW_DEBUG_BOUNDS) {
        if (!layout_cells_ok(g, o, n, interior_only)) {
            if (err) atomicCAS(err, DEV_OK, DEV_OOB_STORE);
            return false;
        }
    }
    return true;
}

// Writes the three outputs of one cell or one row vector of N cells, plus the
// periodic images (MODE_STEP) when the cells lie near the lateral boundary.  o = offset of (k, j, i0); cells i0..i0+n-1.
template <typename T, int MODE>
struct Epilogue;

template <typename T>
struct Epilogue<T, MODE_TEND> {
    static __device__ __forceinline__ void store1(T* o0, T* o1, T* o2, long long o, float a, float b, float c,
                                                  const GridDev&, int, int) {
        o0[o] = Store<T>::from_f(a);
        o1[o] = Store<T>::from_f(b);
        o2[o] = Store<T>::from_f(c);
    }
    // one field's row vector of N cells
    template <int N>
    static __device__ __forceinline__ void store_field(T* of, long long o, const float (&a)[N], const GridDev& g, int,
                                                       int, int* err = nullptr) {
        if (dbg_store(g, o, N, true, err)) storev<N>(of + o, a);
    }
};

// Periodic images of a step's output cells in a lateral halo of any depth
// H = g.halo (H <= nx and H <= ny, which the grid check enforces): cell
// i <= H also goes to i + nx, cell i > nx - H to i - nx, and likewise in y,
// corners included.
struct StepImages {
    // one cell (j, i) at offset o, values already in the storage type
    template <typename T>
    static __device__ __forceinline__ void cell(T* o0, T* o1, T* o2, long long o, T ta, T tb, T tc,
                                                const GridDev& g, int j, int i) {
        auto put = [&](long long p) {
            o0[p] = ta;
            o1[p] = tb;
            o2[p] = tc;
        };
        const int H = g.halo;
        const long long dxp = (i <= H) ? (long long)g.nx : 0;             // image at i + nx
        const long long dxm = (i > g.nx - H) ? -(long long)g.nx : 0;      // image at i - nx
        const long long dyp = (j <= H) ? (long long)g.ny * g.pj : 0;
        const long long dym = (j > g.ny - H) ? -(long long)g.ny * g.pj : 0;
        if (dxp) put(o + dxp);
        if (dxm) put(o + dxm);
        if (dyp) {
            put(o + dyp);
            if (dxp) put(o + dyp + dxp);
            if (dxm) put(o + dyp + dxm);
        }
        if (dym) {
            put(o + dym);
            if (dxp) put(o + dym + dxp);
            if (dxm) put(o + dym + dxm);
        }
    }
    // one field's vector of N cells (j, i0..i0+N-1), i0 = 1 mod N, nx = 0 mod N
    template <typename T, int N>
    static __device__ __forceinline__ void vec1(T* of, long long o, const float (&a)[N], const GridDev& g, int j,
                                                int i0, int* err = nullptr) {
        const int H = g.halo;
        const bool west = (i0 <= H), east = (i0 + N - 1 > g.nx - H);
        const long long dyp = (j <= H) ? (long long)g.ny * g.pj : 0;
        const long long dym = (j > g.ny - H) ? -(long long)g.ny * g.pj : 0;
        if (!west && !east && !dyp && !dym) return;
        const long long shifts[3] = {0, dyp, dym};
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            if (s > 0 && shifts[s] == 0) continue;
            const long long p = o + shifts[s];
            if (s > 0 && dbg_store(g, p, N, false, err)) storev<N>(of + p, a);   // the row image
#pragma unroll
            for (int q = 0; q < N; ++q) {
                const int i = i0 + q;
                if (west && i <= H && dbg_store(g, p + q + g.nx, 1, false, err))
                    of[p + q + g.nx] = Store<T>::from_f(a[q]);   // i -> i + nx
                if (east && i > g.nx - H && dbg_store(g, p + q - g.nx, 1, false, err))
                    of[p + q - g.nx] = Store<T>::from_f(a[q]);   // i -> i - nx
            }
        }
    }
};

// MODE_STEP: the generic kernel's single cells get their images for any halo
// depth; the k-march's row vectors get those of a one-cell halo only (kept
// lean: the register count sets how many CTAs an SM holds), and the host
// refreshes deeper halos with the halo kernel after such a pass.
template <typename T>
struct Epilogue<T, MODE_STEP> {
    // one cell (j, i) at offset o
    static __device__ __forceinline__ void store1(T* o0, T* o1, T* o2, long long o, float a, float b, float c,
                                                  const GridDev& g, int j, int i) {
        const T ta = Store<T>::from_f(a), tb = Store<T>::from_f(b), tc = Store<T>::from_f(c);
        o0[o] = ta;
        o1[o] = tb;
        o2[o] = tc;
        StepImages::cell<T>(o0, o1, o2, o, ta, tb, tc, g, j, i);
    }
    // one field's vector of N cells (j, i0..i0+N-1), i0 = 1 mod N, nx = 0 mod N
    template <int N>
    static __device__ __forceinline__ void store_field(T* of, long long o, const float (&a)[N], const GridDev& g,
                                                       int j, int i0, int* err = nullptr) {
        if (dbg_store(g, o, N, true, err)) storev<N>(of + o, a);
        if (g.halo != 1) return;   // deeper halos are refreshed by the halo kernel
        const bool west = (i0 == 1), east = (i0 + N - 1 == g.nx);
        // most row vectors touch no boundary: one test, the same at every level
        if (!(west | east | (j == 1) | (j == g.ny))) return;
        const long long dyp = (j == 1) ? (long long)g.ny * g.pj : 0;
        const long long dym = (j == g.ny) ? -(long long)g.ny * g.pj : 0;
        const long long shifts[3] = {0, dyp, dym};
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            if (s > 0 && shifts[s] == 0) continue;
            const long long p = o + shifts[s];
            if (s > 0 && dbg_store(g, p, N, false, err)) storev<N>(of + p, a);   // the row image
            if (west && dbg_store(g, p + g.nx, 1, false, err))
                of[p + g.nx] = Store<T>::from_f(a[0]);                  // cell i = 1 -> i = nx+1
            if (east && dbg_store(g, p + (N - 1) - g.nx, 1, false, err))
                of[p + (N - 1) - g.nx] = Store<T>::from_f(a[N - 1]);    // cell i = nx -> i = 0
        }
    }
};

// ---------------------------------------------------------------------------
// Generic kernel: one thread per cell, plain loads, any layout and alignment.
template <typename T, bool SCALED, int MODE>
__global__ void generic_kernel(const GridDev g, const T* __restrict__ u, const T* __restrict__ v,
                               const T* __restrict__ w, T* __restrict__ o0, T* __restrict__ o1, T* __restrict__ o2,
                               const Scales sc, const CoefDev cf, const float dt) {
    const long long nx = g.nx, ny = g.ny, nz = g.nz;
    const long long total = nx * ny * nz;
    const int nzp2 = g.nz + 2;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = 1 + (int)(idx % nx);
        const int j = 1 + (int)((idx / nx) % ny);
        const int k = 1 + (int)(idx / (nx * ny));
        const long long c = g.origin + k * g.pk + j * g.pj + i;
        auto at = [&](const T* f, int dk, int dj, int di, float s) {
            float x = Store<T>::to_f(f[c + dk * g.pk + dj * g.pj + di]);
            return SCALED ? x * s : x;
        };
        auto U = [&](int dk, int dj, int di) { return at(u, dk, dj, di, sc.in[0]); };
        auto V = [&](int dk, int dj, int di) { return at(v, dk, dj, di, sc.in[1]); };
        auto W = [&](int dk, int dj, int di) { return at(w, dk, dj, di, sc.in[2]); };
        float ru = 0.f, rv = 0.f, rw = 0.f;
        if (k >= 2) {
            const float tz1 = cf.tz[k], tz2 = cf.tz[nzp2 + k];
            const bool top = k < g.nz;
            ru = cf.tcx * (U(0, 0, -1) * (U(0, 0, 0) + U(0, 0, -1)) - U(0, 0, 1) * (U(0, 0, 0) + U(0, 0, 1))) +
                 cf.tcy * (U(0, -1, 0) * (V(0, -1, 0) + V(0, -1, 1)) - U(0, 1, 0) * (V(0, 0, 0) + V(0, 0, 1))) +
                 tz1 * (U(-1, 0, 0) * (W(-1, 0, 0) + W(-1, 0, 1)));
            rv = cf.tcx * (V(0, 0, -1) * (U(0, 0, -1) + U(0, 1, -1)) - V(0, 0, 1) * (U(0, 0, 0) + U(0, 1, 0))) +
                 cf.tcy * (V(0, -1, 0) * (V(0, 0, 0) + V(0, -1, 0)) - V(0, 1, 0) * (V(0, 0, 0) + V(0, 1, 0))) +
                 tz1 * (V(-1, 0, 0) * (W(-1, 0, 0) + W(-1, 1, 0)));
            if (top) {
                ru -= tz2 * (U(1, 0, 0) * (W(0, 0, 0) + W(0, 0, 1)));
                rv -= tz2 * (V(1, 0, 0) * (W(0, 0, 0) + W(0, 1, 0)));
                const float td1 = cf.tz[2 * nzp2 + k], td2 = cf.tz[3 * nzp2 + k];
                rw = cf.tcx * (W(0, 0, -1) * (U(0, 0, -1) + U(1, 0, -1)) - W(0, 0, 1) * (U(0, 0, 0) + U(1, 0, 0))) +
                     cf.tcy * (W(0, -1, 0) * (V(0, -1, 0) + V(1, -1, 0)) - W(0, 1, 0) * (V(0, 0, 0) + V(1, 0, 0))) +
                     (td1 * (W(-1, 0, 0) * (W(0, 0, 0) + W(-1, 0, 0))) - td2 * (W(1, 0, 0) * (W(0, 0, 0) + W(1, 0, 0))));
            }
        }
        if (MODE == MODE_STEP) {
            ru = fmaf(dt, ru, U(0, 0, 0));
            rv = fmaf(dt, rv, V(0, 0, 0));
            rw = fmaf(dt, rw, W(0, 0, 0));
        }
        if (SCALED) {
            ru *= sc.out[0];
            rv *= sc.out[1];
            rw *= sc.out[2];
        }
        Epilogue<T, MODE>::store1(o0, o1, o2, c, ru, rv, rw, g, j, i);
    }
}

template <typename T, int MODE>
static cudaError_t launch_generic_mode(const GridDev& g, const void* u, const void* v, const void* w, void* o0,
                                       void* o1, void* o2, const Scales& sc, bool scaled, const CoefDev& cf,
                                       float dt, int num_sms, cudaStream_t s) {
    const long long total = (long long)g.nx * g.ny * g.nz;
    const int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    const long long cap = (long long)num_sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (scaled)
        generic_kernel<T, true, MODE><<<(unsigned)blocks, threads, 0, s>>>(
            g, (const T*)u, (const T*)v, (const T*)w, (T*)o0, (T*)o1, (T*)o2, sc, cf, dt);
    else
        generic_kernel<T, false, MODE><<<(unsigned)blocks, threads, 0, s>>>(
            g, (const T*)u, (const T*)v, (const T*)w, (T*)o0, (T*)o1, (T*)o2, sc, cf, dt);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Arithmetic on the values a k-march thread works with: V = float (one cell)
// or V = float2 (a cell and the cell one row further, computed together with
// the packed FP32x2 instructions of the sm_100 family).  Every operation is
// rounded exactly like its scalar counterpart (fmaf, IEEE add and multiply),
// so both forms give the same bits; none is contracted.
template <typename V>
struct VOps;
template <>
struct VOps<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
    static __device__ __forceinline__ float neg(float a) { return -a; }
    static __device__ __forceinline__ float splat(float a) { return a; }
    static __device__ __forceinline__ float zero() { return 0.f; }
    static __device__ __forceinline__ float sel(bool p, float a, float b) { return p ? a : b; }
    static __device__ __forceinline__ float shfl_up(float x, int w) { return __shfl_up_sync(0xffffffffu, x, 1, w); }
    static __device__ __forceinline__ float shfl_down(float x, int w) {
        return __shfl_down_sync(0xffffffffu, x, 1, w);
    }
};
template <>
struct VOps<float2> {
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
    static __device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }
    static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ float2 sel(bool p, float2 a, float2 b) { return p ? a : b; }
    static __device__ __forceinline__ float2 shfl_up(float2 x, int w) {
        return make_float2(__shfl_up_sync(0xffffffffu, x.x, 1, w), __shfl_up_sync(0xffffffffu, x.y, 1, w));
    }
    static __device__ __forceinline__ float2 shfl_down(float2 x, int w) {
        return make_float2(__shfl_down_sync(0xffffffffu, x.x, 1, w), __shfl_down_sync(0xffffffffu, x.y, 1, w));
    }
};

// ---------------------------------------------------------------------------
// One level of a k-march for the NC consecutive cells of one thread (shared
// by every k-march kernel: single step, two-step temporal blocking, batch).
//
// MarchRegs is what a thread carries from level kk to kk+1: the level-kk rows
// it loaded as level kk+1 on the previous step, and the lower vertical flux
// products of level kk, u(kk-1)*(w(kk-1,i) + w(kk-1,i+1)) and its v and w
// counterparts.  Both factors of each product are known one level earlier
// (the level's own values and its upper pair sums), so the product is formed
// there and carried instead of the two factors: the same operation on the
// same operands, three carried arrays instead of six.
template <int NC, typename V = float>
struct MarchRegs {
    V u0[NC], v0[NC], vs[NC], w0[NC];   // level kk: u, v, w in row r; vs = v in row r-1
    V pdu[NC], pdv[NC], pdw[NC];        // lower vertical flux products of level kk
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            pdu[c] = pdv[c] = pdw[c] = VOps<V>::zero();
            u0[c] = v0[c] = vs[c] = w0[c] = VOps<V>::zero();
        }
    }
};

enum { F_U = 0, F_V = 1, F_W = 2 };

// x neighbours of a thread's row vector by warp shuffles: the value at x = -1
// (m) and x = NC (p) come from the adjacent lanes, the row's two edge lanes
// read theirs from the halo columns (edge(f, up, dr): the value beyond the
// row's first lane for lane 0, beyond its last lane for lane LX-1).
template <int NC, int LX, typename V, class Edge>
struct NbrShfl {
    const Edge& edge;
    const int xl;
    __device__ __forceinline__ V m(int f, int up, int dr, const V (&x)[NC]) const {
        return VOps<V>::sel(xl == 0, edge(f, up, dr), VOps<V>::shfl_up(x[NC - 1], LX));
    }
    __device__ __forceinline__ V p(int f, int up, int dr, const V (&x)[NC]) const {
        return VOps<V>::sel(xl == LX - 1, edge(f, up, dr), VOps<V>::shfl_down(x[0], LX));
    }
};

// x neighbours when a thread's 2*NP consecutive cells are packed as NP pairs
// (cell q, cell q + NP): the pair one cell to the left of pair 0 is
// (x = -1, cell NP - 1) and the pair one to the right of pair NP-1 is
// (cell NP, x = 2*NP), so each takes one value loaded from the staged row
// (ld(f, up, dr, side): side 0 the value at x = -1, side 1 at x = 2*NP) and
// one of the thread's own.
template <int NP, class Ld>
struct NbrPairs {
    const Ld& ld;
    __device__ __forceinline__ float2 m(int f, int up, int dr, const float2 (&x)[NP]) const {
        return make_float2(ld(f, up, dr, 0), x[NP - 1].x);
    }
    __device__ __forceinline__ float2 p(int f, int up, int dr, const float2 (&x)[NP]) const {
        return make_float2(x[0].y, ld(f, up, dr, 1));
    }
};

// Per-level vertical coefficients of the three outputs, storage scales folded
// in (FoldedCoef): lower tzc1*kz_u, tzc1*kz_v; upper -(tzc2*kz_u), -(tzc2*kz_v),
// tzd1*kz_w, -(tzd2*kz_w).
// ZCoefLdg reads the coefficient arrays every level; ZCoefTab reads a table of
// the same products that the CTA computed once (zcoef_fill), each value
// stored twice so that a 16-byte shared load gives two ready FP32x2 operands.
struct ZCoefLdg {
    const FoldedCoef& k;
    const int nzp2;
    template <typename V>
    __device__ __forceinline__ void lower(int kk, V& tz1u, V& tz1v) const {
        const float t1 = __ldg(k.tz + kk);
        tz1u = VOps<V>::splat(t1 * k.kz[0]);
        tz1v = VOps<V>::splat(t1 * k.kz[1]);
    }
    template <typename V>
    __device__ __forceinline__ void upper(int kk, V& ntz2u, V& ntz2v, V& td1w, V& ntd2w) const {
        const float t2 = __ldg(k.tz + nzp2 + kk);
        const float d1 = __ldg(k.tz + 2 * nzp2 + kk);
        const float d2 = __ldg(k.tz + 3 * nzp2 + kk);
        ntz2u = VOps<V>::splat(-(t2 * k.kz[0]));
        ntz2v = VOps<V>::splat(-(t2 * k.kz[1]));
        td1w = VOps<V>::splat(d1 * k.kz[2]);
        ntd2w = VOps<V>::splat(-(d2 * k.kz[2]));
    }
};

struct ZCoefTab {
    const float4* tab;   // 3 float4 per level, level `base` first
    int base;
    static __device__ __forceinline__ void get(const float4& a, float& x, float& y) {
        x = a.x;
        y = a.z;
    }
    static __device__ __forceinline__ void get(const float4& a, float2& x, float2& y) {
        x = make_float2(a.x, a.y);
        y = make_float2(a.z, a.w);
    }
    template <typename V>
    __device__ __forceinline__ void lower(int kk, V& tz1u, V& tz1v) const {
        get(tab[3 * (kk - base)], tz1u, tz1v);
    }
    template <typename V>
    __device__ __forceinline__ void upper(int kk, V& ntz2u, V& ntz2v, V& td1w, V& ntd2w) const {
        get(tab[3 * (kk - base) + 1], ntz2u, ntz2v);
        get(tab[3 * (kk - base) + 2], td1w, ntd2w);
    }
};

// Levels lo..hi of the ZCoefTab table (entry 0 = level lo), computed by all
// `nthreads` threads of the CTA (the caller then synchronises the CTA).
__device__ __forceinline__ void zcoef_fill(float4* tab, const FoldedCoef& k, const int nzp2, const int lo,
                                           const int hi, const int tid, const int nthreads) {
    for (int e = tid; e < 3 * (hi - lo + 1); e += nthreads) {
        const int kk = lo + e / 3, part = e - 3 * (e / 3);
        float a, b;
        if (part == 0) {
            const float t1 = __ldg(k.tz + kk);
            a = t1 * k.kz[0];
            b = t1 * k.kz[1];
        } else if (part == 1) {
            const float t2 = __ldg(k.tz + nzp2 + kk);
            a = -(t2 * k.kz[0]);
            b = -(t2 * k.kz[1]);
        } else {
            const float d1 = __ldg(k.tz + 2 * nzp2 + kk), d2 = __ldg(k.tz + 3 * nzp2 + kk);
            a = d1 * k.kz[2];
            b = -(d2 * k.kz[2]);
        }
        tab[e] = make_float4(a, a, b, b);
    }
}

// Source terms (Sec. 2.2) of level kk, handed to `out` one field at a time,
// then the roll of `st` to level kk+1.  The data sources are abstract:
//   row(f, up, dr, o)  the thread's NC values of field f (F_U, F_V, F_W) in
//                      row r+dr of level kk+up (up = 0 or 1)
//   nbr.m / nbr.p      the value one cell beyond the row vector on the left
//                      (x = -1) / right (x = NC) (NbrShfl, NbrPairs)
//   zc                 the per-level vertical coefficients (ZCoefLdg, ZCoefTab)
//   out(f, s, q)       the source term s of field f and the field's level-kk
//                      values q
// first:   kk is the first level of the march (its rows are loaded here)
// have_up: level kk+1 exists (kk < nz): the upper vertical fluxes and sw
// compute: evaluate the source terms (else they are zero: k = 1, or a level
//          that only primes the carried state)
// The fields go one after the other (su, then sv, then sw, each handed out
// as soon as it is complete, and each lower flux product of the next level
// formed as soon as its pair sum has had its last use), so that few values
// are live at once.  Pair sums along x are shared by neighbouring cells.
// Every form of the k-march runs this one sequence of operations, so they
// agree bit for bit.
//
// pdx(f, p, store): where the lower flux products live between levels: a
// no-op when they stay in st's registers (PdRegs), else a copy of field f's
// products from (store = false) or to (store = true) shared memory, done just
// before their use and just after they are formed.
struct PdRegs {
    template <class A>
    __device__ __forceinline__ void operator()(int, A&, bool) const {}
};

template <int NC, typename V, class Row, class Nbr, class ZC, class Out, class Pd = PdRegs>
__device__ __forceinline__ void march_level_core(MarchRegs<NC, V>& st, const Row& row, const Nbr& nbr, const ZC& zc,
                                                 const Out& out, const bool first, const bool have_up,
                                                 const bool compute, const FoldedCoef& k, const int kk,
                                                 const Pd& pdx = Pd{}) {
    using O = VOps<V>;
    if (first) {
        row(F_U, 0, 0, st.u0);
        row(F_V, 0, 0, st.v0);
        row(F_V, 0, -1, st.vs);
        row(F_W, 0, 0, st.w0);
    }
    V W[NC + 2];   // w of level kk, x = -1..NC
    W[0] = nbr.m(F_W, 0, 0, st.w0);
    W[NC + 1] = nbr.p(F_W, 0, 0, st.w0);
#pragma unroll
    for (int c = 0; c < NC; ++c) W[c + 1] = st.w0[c];
    // upper vertical pair sum of su at level kk = its lower one at kk+1
    V pzu_n[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) pzu_n[c] = O::add(W[c + 1], W[c + 2]);   // w(k,i) + w(k,i+1)
    // level kk+1 rows (upper terms; carried into the next step)
    V uu[NC], vu[NC], vus[NC], wu[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) uu[c] = vu[c] = vus[c] = wu[c] = O::zero();
    if (have_up) row(F_U, 1, 0, uu);

    V r[NC];   // the source term of the field in hand
    if (compute) {
        // per output field: x, y and lower vertical coefficients (storage scales folded in)
        const V kxu = O::splat(k.kx[0]), kxv = O::splat(k.kx[1]), kxw = O::splat(k.kx[2]);
        const V kyu = O::splat(k.ky[0]), kyv = O::splat(k.ky[1]), kyw = O::splat(k.ky[2]);
        V tz1u, tz1v, ntz2u = O::zero(), ntz2v = O::zero(), td1w = O::zero(), ntd2w = O::zero();
        zc.lower(kk, tz1u, tz1v);
        if (have_up) zc.upper(kk, ntz2u, ntz2v, td1w, ntd2w);

        // ---- su
        V U[NC + 2], Vv[NC + 2];   // x = -1..NC
        V VS[NC + 1];              // x = 0..NC
        U[0] = nbr.m(F_U, 0, 0, st.u0);
        U[NC + 1] = nbr.p(F_U, 0, 0, st.u0);
        Vv[0] = nbr.m(F_V, 0, 0, st.v0);
        Vv[NC + 1] = nbr.p(F_V, 0, 0, st.v0);
        VS[NC] = nbr.p(F_V, 0, -1, st.vs);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            U[c + 1] = st.u0[c];
            Vv[c + 1] = st.v0[c];
            VS[c] = st.vs[c];
        }
        V un[NC];
        row(F_U, 0, 1, un);
        {
            V us[NC];
            row(F_U, 0, -1, us);
            // pair sums along x shared by neighbouring cells: index c is the
            // pair (x = c-1, c)
            V pxu[NC + 1], pxv[NC], pys[NC];
#pragma unroll
            for (int c = 0; c < NC + 1; ++c) pxu[c] = O::add(U[c], U[c + 1]);   // u(i-1) + u(i)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                pxv[c] = O::add(Vv[c + 1], Vv[c + 2]);   // v(j,i) + v(j,i+1)
                pys[c] = O::add(VS[c], VS[c + 1]);       // v(j-1,i) + v(j-1,i+1)
            }
            pdx(F_U, st.pdu, false);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                V x = O::mul(kxu, O::fma(O::neg(U[c + 2]), pxu[c + 1], O::mul(U[c], pxu[c])));
                x = O::fma(kyu, O::fma(O::neg(un[c]), pxv[c], O::mul(us[c], pys[c])), x);
                r[c] = O::fma(tz1u, st.pdu[c], x);
                if (have_up) r[c] = O::fma(ntz2u, O::mul(uu[c], pzu_n[c]), r[c]);
            }
        }
        out(F_U, r, st.u0);
#pragma unroll
        for (int c = 0; c < NC; ++c) st.pdu[c] = O::mul(st.u0[c], pzu_n[c]);   // u(k) * (w(k,i) + w(k,i+1))
        pdx(F_U, st.pdu, true);

        // ---- sv
        V wn[NC];
        row(F_W, 0, 1, wn);
        V pzv_n[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) pzv_n[c] = O::add(st.w0[c], wn[c]);   // w(k,j) + w(k,j+1)
        if (have_up) row(F_V, 1, 0, vu);
        {
            V vn[NC];
            row(F_V, 0, 1, vn);
            V UN[NC + 1], qx[NC + 1];   // x = -1..NC-1
            UN[0] = nbr.m(F_U, 0, 1, un);
#pragma unroll
            for (int c = 0; c < NC; ++c) UN[c + 1] = un[c];
#pragma unroll
            for (int c = 0; c < NC + 1; ++c) qx[c] = O::add(U[c], UN[c]);   // u(j,i-1) + u(j+1,i-1)
            pdx(F_V, st.pdv, false);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                V y = O::mul(kxv, O::fma(O::neg(Vv[c + 2]), qx[c + 1], O::mul(Vv[c], qx[c])));
                y = O::fma(kyv,
                           O::fma(O::neg(vn[c]), O::add(Vv[c + 1], vn[c]),
                                  O::mul(st.vs[c], O::add(Vv[c + 1], st.vs[c]))),
                           y);
                r[c] = O::fma(tz1v, st.pdv[c], y);
                if (have_up) r[c] = O::fma(ntz2v, O::mul(vu[c], pzv_n[c]), r[c]);
            }
        }
        out(F_V, r, st.v0);
#pragma unroll
        for (int c = 0; c < NC; ++c) st.pdv[c] = O::mul(st.v0[c], pzv_n[c]);   // v(k) * (w(k,j) + w(k,j+1))
        pdx(F_V, st.pdv, true);

        // ---- sw (zero at the lid)
        if (have_up) {
            row(F_V, 1, -1, vus);
            row(F_W, 1, 0, wu);
        }
        V pzw_n[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            pzw_n[c] = O::add(st.w0[c], wu[c]);   // w(k) + w(k+1)
            r[c] = O::zero();
        }
        if (have_up) {
            V ws[NC];
            row(F_W, 0, -1, ws);
            V UU[NC + 1], rx[NC + 1];   // x = -1..NC-1
            UU[0] = nbr.m(F_U, 1, 0, uu);
#pragma unroll
            for (int c = 0; c < NC; ++c) UU[c + 1] = uu[c];
#pragma unroll
            for (int c = 0; c < NC + 1; ++c) rx[c] = O::add(U[c], UU[c]);   // u(k,i-1) + u(k+1,i-1)
            pdx(F_W, st.pdw, false);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                V z = O::mul(kxw, O::fma(O::neg(W[c + 2]), rx[c + 1], O::mul(W[c], rx[c])));
                z = O::fma(kyw, O::fma(O::neg(wn[c]), O::add(Vv[c + 1], vu[c]), O::mul(ws[c], O::add(st.vs[c], vus[c]))),
                           z);
                z = O::fma(td1w, st.pdw[c], z);
                r[c] = O::fma(ntd2w, O::mul(wu[c], pzw_n[c]), z);
            }
        }
        out(F_W, r, st.w0);
#pragma unroll
        for (int c = 0; c < NC; ++c) st.pdw[c] = O::mul(st.w0[c], pzw_n[c]);   // w(k) * (w(k) + w(k+1))
        pdx(F_W, st.pdw, true);
    } else {
        // no source terms at this level: zeros out, and the rows and flux
        // products of level kk+1
        V wn[NC];
        row(F_W, 0, 1, wn);
        if (have_up) {
            row(F_V, 1, 0, vu);
            row(F_V, 1, -1, vus);
            row(F_W, 1, 0, wu);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) r[c] = O::zero();
        out(F_U, r, st.u0);
        out(F_V, r, st.v0);
        out(F_W, r, st.w0);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            st.pdu[c] = O::mul(st.u0[c], pzu_n[c]);
            st.pdv[c] = O::mul(st.v0[c], O::add(st.w0[c], wn[c]));
            st.pdw[c] = O::mul(st.w0[c], O::add(st.w0[c], wu[c]));
        }
        pdx(F_U, st.pdu, true);
        pdx(F_V, st.pdv, true);
        pdx(F_W, st.pdw, true);
    }

    // roll: level kk+1 becomes level kk
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        st.u0[c] = uu[c];
        st.v0[c] = vu[c];
        st.vs[c] = vus[c];
        st.w0[c] = wu[c];
    }
}

// The k-march level with x neighbours by warp shuffles (LX lanes per row) and
// the vertical coefficients read each level (the two-step kernel's stages):
// out(ru, rv, rw, u, v, w) receives the three source terms together.
template <int NC, int LX, typename V, class Row, class Edge, class Out>
__device__ __forceinline__ void march_level(MarchRegs<NC, V>& st, const Row& row, const Edge& edge, const Out& out,
                                            const int xl, const bool first, const bool have_up, const bool compute,
                                            const FoldedCoef& k, const int kk, const int nzp2) {
    const NbrShfl<NC, LX, V, Edge> nbr{edge, xl};
    const ZCoefLdg zc{k, nzp2};
    V ru[NC], rv[NC];
    auto out3 = [&](int f, const V (&r)[NC], const V (&)[NC]) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (f == F_U) ru[c] = r[c];
            if (f == F_V) rv[c] = r[c];
        }
        if (f == F_W) out(ru, rv, r, st.u0, st.v0, st.w0);
    };
    march_level_core<NC, V>(st, row, nbr, zc, out3, first, have_up, compute, k, kk);
}

// ---------------------------------------------------------------------------
// TMA k-march.
//
// A tile is NC*LX interior columns by TY*RP rows and one k segment; the CTA
// marches up the column one level at a time.  Level planes of u, v, w (the
// tile plus a one-cell halo, widened in x to the 16-byte TMA granule) arrive
// in a ring of S shared-memory slots by 3D TMA box copies that one thread
// issues, each slot completing on its own mbarrier; S-1 planes are in flight
// ahead of the level being computed, so every input element is read from HBM
// once and the copy engine, not the warps, keeps bytes in flight.
//
// LX lanes cover one row (LX = 32: one warp per row; LX = 16 or 8: two or
// four rows per warp, for narrow tiles).  A thread computes NC consecutive cells along x,
// in one row (RP = 1) or in two adjacent rows (RP = 2: a cell and the cell
// below it form one float2, and the arithmetic runs on the packed FP32x2
// instructions, half the instructions for the same operations).
// Shared-memory rows are read as 16-byte (FP32) or 8-byte (16-bit) vectors; x
// neighbours come from the adjacent lanes by warp shuffles (the two tile-edge
// lanes of a row read theirs from the halo columns); y neighbours from the
// rows above and below.  Registers carry from one level to the next: the
// level-k+1 rows the upper terms read (they are the level-k rows of the next
// step), the level-(k-1) values at the cell (a rolling window in z), and the
// three vertical pair sums of the upper fluxes, which are the lower pair sums
// of the next level.  Pair sums along x are shared by neighbouring cells of a
// thread.  Outputs go straight from registers to HBM as full vectors.
//
// Ring bookkeeping is global to the CTA: the n-th plane a CTA ever issues
// goes to slot n % S and completes phase (n / S) & 1 of that slot's mbarrier,
// so a persistent CTA can march tile after tile without re-initialising.
// Build-time knob of the k-march kernel: PW_TMA_MAX_MINB caps the resident
// CTAs per SM the register budget of the 4-cell shapes is sized for.  On
// GB300 a cap of 2 (the compiler's own choice, about 128 registers) was the
// fastest for every 4-cell shape; caps of 4 to 6 made them slower, and the
// 8-row ones spill.
#ifndef PW_TMA_MAX_MINB
#define PW_TMA_MAX_MINB 2
#endif
// Register target of the 8-cells-a-thread shapes (8 x 1 or 4 x 2).
#ifndef PW_TMA_REGS8
#define PW_TMA_REGS8 168
#endif
// How a plane slot is handed back to the copy engine after a level:
// 1 = each warp counts itself out on the slot (an acquire-release atomic) and
//     the last one refills it, so warps may drift up to S-1 levels apart;
// 0 = a CTA barrier after every level, then one thread refills.
// On GB300 the barrier was a little faster (BF16 16x8x4x8: 303 against 291
// Gcell/s; FP32 32x4x4x4: 270 against 265), so 0.
#ifndef PW_MARCH_SPLIT_ARRIVE
#define PW_MARCH_SPLIT_ARRIVE 0
#endif
// Levels per iteration of the k-march loop (2: the carried rows of one level
// are renamed rather than moved into place for the next).
#ifndef PW_MARCH_UNROLL
#define PW_MARCH_UNROLL 1
#endif
#ifndef PW_MARCH_UNROLL_XP
#define PW_MARCH_UNROLL_XP 2
#endif
// Steady levels with their facts (not first, computing, level kk+1 exists)
// as compile-time constants (0: the same runtime tests as other levels).
#ifndef PW_MARCH_FAST
#define PW_MARCH_FAST 1
#endif
// x-pair form: one CTA barrier per pair of steady levels instead of per level.
#ifndef PW_MARCH_PAIR_SYNC
#define PW_MARCH_PAIR_SYNC 1
#endif
// x-pair form: the lower flux products kept in shared memory between levels
// (fewer registers a thread) instead of registers.
// (BF16 378 -> 386, FP16 374 -> 382 Gcell/s at 2048^2 x 64: 128 registers,
// four CTAs per SM instead of three)
#ifndef PW_MARCH_PD_SMEM
#define PW_MARCH_PD_SMEM 1
#endif
// Register target of the x-pair shapes with 8 cells a thread and the flux
// products in shared memory (128: four CTAs of 4 warps per SM, no spills).
#ifndef PW_TMA_REGS_XP
#define PW_TMA_REGS_XP 128
#endif
// x-pair form: staged rows read through explicit 32-bit shared addresses
// (with two levels per iteration: BF16 384 against 376 Gcell/s at 2048^2 x 64).
#ifndef PW_MARCH_LDS_ASM
#define PW_MARCH_LDS_ASM 1
#endif

template <typename T, int LX, int TY, int S, int NC = 4, int RP = 1, int XP = 0>
struct TmaLayout {
    static constexpr int TX = NC * LX;
    static constexpr int RPW = 32 / LX;                // thread rows per warp
    static constexpr int WARPS = TY / (RPW * RP);
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int PADX = 16 / (int)sizeof(T);   // elements in one 16-byte granule
    static constexpr int BW = TX + 2 * PADX;           // box width
    static constexpr int ROWS = TY + 2;
    static constexpr int FIELD_RAW = BW * ROWS;
    static constexpr int FIELD_BYTES = ((FIELD_RAW * (int)sizeof(T) + 127) / 128) * 128;
    static constexpr int FIELD = FIELD_BYTES / (int)sizeof(T);
    static constexpr int STAGE = 3 * FIELD;
    static constexpr uint32_t TX_BYTES = 3u * FIELD_RAW * (uint32_t)sizeof(T);
    // packed FP32x2 forms read the per-level vertical coefficients from a
    // table in shared memory (ZCoefTab), CTAB_LEVELS levels at a time
    static constexpr bool PACKED = (RP == 2 || XP == 1);
    static constexpr bool CTAB = PACKED;
    static constexpr int CTAB_LEVELS = 128;
    static constexpr size_t CTAB_BYTES = CTAB ? (size_t)CTAB_LEVELS * 3 * sizeof(float4) : 0;
    // x-pair form with PW_MARCH_PD_SMEM: the lower flux products of every
    // thread (3 fields x NC/2 pairs) in shared memory between levels
    static constexpr bool PD_SMEM = XP == 1 && PW_MARCH_PD_SMEM;
    static constexpr size_t PD_BYTES = PD_SMEM ? (size_t)3 * (NC / 2) * THREADS * sizeof(float2) : 0;
    // The plane ring, then the mbarriers and flags, then the table and the
    // flux products.  A kernel that marches tiles of two shapes through one
    // ring gives both views the larger ring region (sb), so that the
    // mbarriers sit at one address.
    static constexpr size_t RING_BYTES = (size_t)S * STAGE * sizeof(T);
    static constexpr size_t ctab_off(size_t sb) {
        return ((sb + S * sizeof(uint64_t) + 16 + 4 * S + 15) / 16) * 16;
    }
    static constexpr size_t smem_bytes(size_t sb) { return ctab_off(sb) + CTAB_BYTES + PD_BYTES; }
    static constexpr size_t CTAB_OFF = ctab_off(RING_BYTES);
    static constexpr size_t PD_OFF = CTAB_OFF + CTAB_BYTES;
    static constexpr size_t SMEM = smem_bytes(RING_BYTES);
    static_assert(LX == 32 || LX == 16 || LX == 8, "LX must be 8, 16 or 32");
    static_assert(NC == 4 || NC == 8, "4 or 8 cells per thread");
    static_assert(BW <= 256, "a TMA box is at most 256 elements wide");
    static_assert(TY % (RPW * RP) == 0, "TY must be a multiple of the rows per warp");
    static_assert(RP == 1 || RP == 2, "one or two rows per thread");
    static_assert(XP == 0 || (RP == 1 && sizeof(T) == 2), "x pairs: one row per thread, 16-bit storage");
};

// Resident CTAs per SM the register budget is sized for: what shared memory
// and the thread limit allow, at most PW_TMA_MAX_MINB for 4 cells a thread;
// 8 cells a thread (8 x 1 or 4 x 2) get PW_TMA_REGS8 = 168 registers, which
// measured best on GB300 (16 lanes x 8 cells x 4 rows: 269 -> 295 Gcell/s for
// BF16 against the compiler's 210 registers, as more CTAs per SM hide more
// latency; 128 spills and 200 leaves 2 CTAs per SM, both slower).
template <typename T, int LX, int TY, int S, int NC = 4, int RP = 1, int XP = 0>
constexpr int tma_min_blocks() {
    using L = TmaLayout<T, LX, TY, S, NC, RP, XP>;
    constexpr int by_smem = (int)((227u * 1024u) / L::SMEM);
    constexpr int by_threads = 2048 / L::THREADS;
    constexpr int by_regs = (L::PD_SMEM && NC == 8)
                                ? 65536 / (L::THREADS * PW_TMA_REGS_XP)
                                : (NC * RP == 8 ? 65536 / (L::THREADS * PW_TMA_REGS8) : PW_TMA_MAX_MINB);
    constexpr int m0 = by_smem < by_threads ? by_smem : by_threads;
    constexpr int m = m0 < by_regs ? m0 : by_regs;
    return m < 1 ? 1 : m;
}

// Shared memory of a k-march CTA: the plane ring, one mbarrier per slot, the
// flags and one release counter per slot.
template <typename T, int LX, int TY, int S, int NC = 4, int RP = 1, int XP = 0>
struct MarchSmem {
    using L = TmaLayout<T, LX, TY, S, NC, RP, XP>;
    T* stages;
    uint64_t* bars;
    volatile int* flag;   // [0] abort, [1] work item broadcast, [2] planes issued (highest + 1)
    uint32_t* cnt;        // warps done with each slot's plane
    float4* ctab;         // vertical coefficient table (L::CTAB)
    float4* pd;           // lower flux products (L::PD_SMEM)
    // sb: bytes of the ring region (L::RING_BYTES, or more when the CTA also
    // marches another shape through the same ring)
    __device__ __forceinline__ explicit MarchSmem(unsigned char* raw, size_t sb = L::RING_BYTES) {
        pd = reinterpret_cast<float4*>(raw + L::ctab_off(sb) + L::CTAB_BYTES);
        stages = reinterpret_cast<T*>(raw);
        bars = reinterpret_cast<uint64_t*>(raw + sb);
        flag = reinterpret_cast<volatile int*>(bars + S);
        cnt = reinterpret_cast<uint32_t*>(bars + S) + 4;
        ctab = reinterpret_cast<float4*>(raw + L::ctab_off(sb));
    }
    // one thread, then a CTA barrier
    __device__ __forceinline__ void init(int tid) {
        if (tid == 0) {
            for (int s = 0; s < S; ++s) {
                mbar_init(&bars[s], 1);
                cnt[s] = 0;
            }
            flag[0] = 0;
            fence_mbar_init();
        }
        __syncthreads();
    }
};

// The thread's NC consecutive 16-bit values at p (aligned to NC elements) as
// NC/2 FP32 pairs (value q, value q + NC/2): the pairing of the x-pair form.
// (FP16: the conversion selects the half of the word itself; BF16: the half
// is moved into the upper 16 bits of an FP32 word, which is exact)
template <typename T>
__device__ __forceinline__ float lo_f(uint32_t w) {
    if constexpr (std::is_same<T, __half>::value)
        return __low2float(*reinterpret_cast<const __half2*>(&w));
    else
        return __uint_as_float(w << 16);
}
template <typename T>
__device__ __forceinline__ float hi_f(uint32_t w) {
    if constexpr (std::is_same<T, __half>::value)
        return __high2float(*reinterpret_cast<const __half2*>(&w));
    else
        return __uint_as_float(w & 0xffff0000u);
}
template <int NC, typename T>
__device__ __forceinline__ void unpack_pairs(const uint32_t (&w)[NC / 2], float2 (&o)[NC / 2]) {
    constexpr int NP = NC / 2;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        // value q sits in word q/2, value q + NP in word (q + NP)/2, the same half
        const uint32_t a = w[q / 2], b = w[(q + NP) / 2];
        o[q] = (q & 1) ? make_float2(hi_f<T>(a), hi_f<T>(b)) : make_float2(lo_f<T>(a), lo_f<T>(b));
    }
}
template <int NC, typename T>
__device__ __forceinline__ void load_pairs(const T* p, float2 (&o)[NC / 2]) {
    static_assert(sizeof(T) == 2 && (NC == 4 || NC == 8), "16-bit storage, 4 or 8 values");
    uint32_t w[NC / 2];
    if constexpr (NC == 8) {
        const uint4 t = *reinterpret_cast<const uint4*>(p);
        w[0] = t.x; w[1] = t.y; w[2] = t.z; w[3] = t.w;
    } else {
        const uint2 t = *reinterpret_cast<const uint2*>(p);
        w[0] = t.x; w[1] = t.y;
    }
    unpack_pairs<NC, T>(w, o);
}
// The same from a 32-bit shared-memory address.
template <int NC, typename T>
__device__ __forceinline__ void load_pairs_sa(uint32_t a, float2 (&o)[NC / 2]) {
    static_assert(sizeof(T) == 2 && (NC == 4 || NC == 8), "16-bit storage, 4 or 8 values");
    uint32_t w[NC / 2];
    if constexpr (NC == 8) {
        const uint4 t = lds_u128(a);
        w[0] = t.x; w[1] = t.y; w[2] = t.z; w[3] = t.w;
    } else {
        const uint2 t = lds_u64(a);
        w[0] = t.x; w[1] = t.y;
    }
    unpack_pairs<NC, T>(w, o);
}

// March one tile: columns bx, rows by, output levels kb..ke of grid g.
// `ring` counts the planes this CTA issued before; it is advanced by the
// planes of this tile.  Returns false if a wait timed out (the error is
// recorded and the copies in flight are drained).
//
// Per-thread forms: RP = 1, XP = 0: NC cells of one row, scalar FP32;
// RP = 2: the same NC cells in two adjacent rows, each cell paired with the
// cell below it (packed FP32x2); XP = 1 (16-bit storage): NC cells of one row
// packed as NC/2 pairs (cell q, cell q + NC/2), so that a staged row unpacks
// straight into FP32x2 operands and the x neighbours beyond the vector come
// from the staged row itself.
template <typename T, int LX, int TY, int S, int MODE, int NC = 4, int RP = 1, int XP = 0>
__device__ __forceinline__ bool march_tile(const MarchSmem<T, LX, TY, S, NC, RP, XP>& sm, const CUtensorMap* tm_u,
                                           const CUtensorMap* tm_v, const CUtensorMap* tm_w, T* __restrict__ o0,
                                           T* __restrict__ o1, T* __restrict__ o2, const GridDev& g, const int ox,
                                           const FoldedCoef& kc, const float dt, const int bx, const int by,
                                           const int kb, const int ke, uint32_t& ring, int* __restrict__ err) {
    using L = TmaLayout<T, LX, TY, S, NC, RP, XP>;
    using V = typename std::conditional<L::PACKED, float2, float>::type;
    constexpr int NV = XP ? NC / 2 : NC;   // values of type V per row vector
    constexpr int BW = L::BW;
    constexpr int PADX = L::PADX;
    constexpr int FU = 0, FV = L::FIELD, FW = 2 * L::FIELD;
    T* const stages = sm.stages;
    uint64_t* const bars = sm.bars;
    volatile int* const abort_flag = sm.flag;

    const int lane = threadIdx.x, warp = threadIdx.y;
    const int tid = warp * 32 + lane;
    const int xl = lane % LX;                          // lane within the row
    const int row = RP * (warp * L::RPW + lane / LX);  // first of the thread's RP rows, 0 .. TY-RP
    const int nz = g.nz;
    const int pb = max(kb - 1, 1);
    const int pe = min(ke + 1, nz);
    const int np = pe - pb + 1;
    const uint32_t base = ring;
    ring += (uint32_t)np;

    const int X0 = ox + 1 + L::TX * bx - PADX;
    const int Y0 = TY * by + g.halo - 1;

    auto issue = [&](int p) {   // plane pb+p into slot (base+p) % S
        const uint32_t n = base + (uint32_t)p;
        const int s = (int)(n % S);
        T* dst = stages + s * L::STAGE;
        mbar_arrive_expect_tx(&bars[s], L::TX_BYTES);
        tma_load_3d(dst + FU, tm_u, X0, Y0, pb + p, &bars[s]);
        tma_load_3d(dst + FV, tm_v, X0, Y0, pb + p, &bars[s]);
        tma_load_3d(dst + FW, tm_w, X0, Y0, pb + p, &bars[s]);
    };
    auto slot = [&](int p) { return (int)((base + (uint32_t)p) % S); };
    auto parity = [&](int p) { return (uint32_t)(((base + (uint32_t)p) / S) & 1u); };

    int issued = 0;
    if (tid == 0) {
        prefetch_tensormap(tm_u);
        prefetch_tensormap(tm_v);
        prefetch_tensormap(tm_w);
        for (; issued < S && issued < np; ++issued) issue(issued);
        sm.flag[2] = issued;
    }
    // vertical coefficients of the tile's first CTAB_LEVELS levels (the
    // previous tile of a persistent CTA is done with the table: every thread
    // has passed its last level's barrier)
    int tbase = pb;
    if constexpr (L::CTAB) {
        zcoef_fill(sm.ctab, kc, nz + 2, pb, min(ke, pb + L::CTAB_LEVELS - 1), tid, L::THREADS);
        __syncthreads();
    }

    const int r = row + 1;
    const int c0 = NC * xl + PADX;
    // tile-edge neighbour column: the row's first lane needs x = -1, its last
    // lane x = TX; the other lanes read the last lane's address (a broadcast)
    const int ce = (xl == 0) ? PADX - 1 : L::TX + PADX;
    const int j = TY * by + 1 + row;
    const int i0 = 1 + L::TX * bx + NC * xl;
    const bool valid = (j <= g.ny) && (i0 <= g.nx);
    const bool valid2 = (j + 1 <= g.ny) && (i0 <= g.nx);   // the second row (RP = 2)
    const long long row_off = g.origin + (long long)j * g.pj + i0;
    // the arithmetic runs on stored values, the storage scales folded into the
    // coefficients kc
    const int nzp2 = nz + 2;
    const unsigned FULL = 0xffffffffu;
    auto ld = [&](const T* p, float (&o)[NC]) { loadv<NC>(p, o); };
    auto ld1 = [&](const T* p) { return Store<T>::to_f(*p); };

    MarchRegs<NV, V> st;
    st.zero();
    int waited = 0;   // planes 0..waited-1 are known complete
    int lp = 0;       // plane index of the level being marched

    // the staged planes of level kk (up = 0) and kk+1 (up = 1); with RP = 2
    // each value pairs row r+dr (x) with row r+dr+1 (y)
    auto rowp = [&](int f, int up, int dr) {
        return stages + slot(lp + up) * L::STAGE + f * L::FIELD + (r + dr) * BW + c0;
    };
    // x-pair form with PW_MARCH_LDS_ASM: 32-bit shared addresses, the
    // thread's part added once, each load's constant part foldable into the
    // load instruction's immediate offset
    const uint32_t tsa = smem_u32(stages) + (uint32_t)((r * BW + c0) * (int)sizeof(T));
    auto rowsa = [&](int f, int up, int dr) {
        return tsa + (uint32_t)(slot(lp + up) * (L::STAGE * (int)sizeof(T))) +
               (uint32_t)((f * L::FIELD + dr * BW) * (int)sizeof(T));
    };
    auto rowld = [&](int f, int up, int dr, V (&o)[NV]) {
        const T* P = rowp(f, up, dr);
        if constexpr (XP && PW_MARCH_LDS_ASM) {
            load_pairs_sa<NC, T>(rowsa(f, up, dr), o);
        } else if constexpr (XP) {
            load_pairs<NC>(P, o);
        } else if constexpr (RP == 1) {
            ld(P, o);
        } else {
            float a[NC], b[NC];
            ld(P, a);
            ld(P + BW, b);
#pragma unroll
            for (int q = 0; q < NC; ++q) o[q] = make_float2(a[q], b[q]);
        }
    };
    auto edgeld = [&](int f, int up, int dr) -> V {   // (not used by the x-pair form)
        const T* P = stages + slot(lp + up) * L::STAGE + f * L::FIELD + (r + dr) * BW + ce;
        if constexpr (XP)
            return VOps<V>::zero();
        else if constexpr (RP == 1)
            return ld1(P);
        else
            return make_float2(ld1(P), ld1(P + BW));
    };
    // x-pair form: the values just beyond the thread's vector, x = -1 (side 0)
    // and x = NC (side 1), read from the staged row
    auto nbrld = [&](int f, int up, int dr, int side) -> float {
        if constexpr (XP && PW_MARCH_LDS_ASM) {
            const uint32_t x = lds_u16(rowsa(f, up, dr) + (side ? NC * (int)sizeof(T) : -(int)sizeof(T)));
            return lo_f<T>(x);
        } else {
            const T* P = rowp(f, up, dr);
            return ld1(side ? P + NC : P - 1);
        }
    };

    // One level of the march.  Returns false on abort.  FAST: a level that is
    // neither the tile's first nor the top of the grid (its rows come from the
    // last level, it computes, and level kk+1 exists), with those facts
    // compile-time constants.
    auto level = [&](const int kk, auto fast, auto sync) -> bool {
        constexpr bool FAST = decltype(fast)::value;
        constexpr bool SYNC = decltype(sync)::value;   // end the level with the CTA barrier
        lp = kk - pb;
        if constexpr (L::CTAB) {
            if (lp > 0 && lp % L::CTAB_LEVELS == 0) {
                __syncthreads();   // every warp is done with the table's last level
                tbase = kk;
                zcoef_fill(sm.ctab, kc, nzp2, kk, min(ke, kk + L::CTAB_LEVELS - 1), tid, L::THREADS);
                __syncthreads();
            }
        }
        bool ok = true;
        if (!FAST && lp == 0) ok = mbar_wait_bounded(&bars[slot(0)], parity(0), kWaitLimitNs);
        const bool have_up = FAST || (kk + 1 <= pe);
        if (ok && have_up) ok = mbar_wait_bounded(&bars[slot(lp + 1)], parity(lp + 1), kWaitLimitNs);
        ok = __all_sync(FULL, ok);
        if (!ok) *abort_flag = 1;
        if (ok) {
            waited = lp + (have_up ? 2 : 1);
            // the value of cell c (0..NC-1) in row `half` of the thread's vector
            auto cellv = [&](const V (&x)[NV], const int c, const int half) -> float {
                if constexpr (XP)
                    return c < NV ? x[c].x : x[c - NV].y;
                else if constexpr (RP == 1)
                    return x[c];
                else
                    return half ? x[c].y : x[c].x;
            };
            // one field's outputs: row `half` of each V (its source terms, or
            // with MODE_STEP the new state q + dt*s)
            auto outf = [&](const int f, const V (&rr)[NV], const V (&q)[NV]) {
                if (!FAST && kk < kb) return;
                T* const of = f == F_U ? o0 : (f == F_V ? o1 : o2);
                auto field_row = [&](const int half) {
                    float a[NC];
#pragma unroll
                    for (int c = 0; c < NC; ++c)   // at kk = 1 the source terms are 0
                        a[c] = MODE == MODE_STEP ? fmaf(dt, cellv(rr, c, half), cellv(q, c, half))
                                                 : cellv(rr, c, half);
                    const long long o = row_off + (long long)half * g.pj + (long long)kk * g.pk;
                    if constexpr (MODE == MODE_TEND && NC == 8) {
                        // nx = 4 mod 8: the row's last vector holds 4 cells of
                        // the grid (the other 4 were computed from halo and
                        // padding columns and are not stored)
                        if (i0 + NC - 1 > g.nx) {
                            const float h4[4] = {a[0], a[1], a[2], a[3]};
                            if (dbg_store(g, o, 4, true, err)) storev<4>(of + o, h4);
                            return;
                        }
                    }
                    Epilogue<T, MODE>::template store_field<NC>(of, o, a, g, j + half, i0, err);
                };
                if (valid) field_row(0);
                if (RP == 2 && valid2) field_row(1);
            };
            // the same for the two-step kernel's three-field interface
            auto out = [&](const V (&ru)[NV], const V (&rv)[NV], const V (&rw)[NV], const V (&u0)[NV],
                           const V (&v0)[NV], const V (&w0)[NV]) {
                outf(F_U, ru, u0);
                outf(F_V, rv, v0);
                outf(F_W, rw, w0);
            };
            const bool first = !FAST && lp == 0, compute = FAST || ((kk >= kb) && (kk >= 2));
            if constexpr (L::CTAB) {
                const ZCoefTab zc{sm.ctab, tbase};
                if constexpr (XP && L::PD_SMEM) {
                    // thread tid's pairs 2m, 2m+1 of field f at float4 (f*NV/2 + m)*THREADS + tid
                    auto pdx = [&](int f, V (&p)[NV], bool store) {
#pragma unroll
                        for (int m = 0; m < NV / 2; ++m) {
                            float4* a = sm.pd + (f * (NV / 2) + m) * L::THREADS + tid;
                            if (store) {
                                *a = make_float4(p[2 * m].x, p[2 * m].y, p[2 * m + 1].x, p[2 * m + 1].y);
                            } else {
                                const float4 t = *a;
                                p[2 * m] = make_float2(t.x, t.y);
                                p[2 * m + 1] = make_float2(t.z, t.w);
                            }
                        }
                    };
                    const NbrPairs<NV, decltype(nbrld)> nbr{nbrld};
                    march_level_core<NV, V>(st, rowld, nbr, zc, outf, first, have_up, compute, kc, kk, pdx);
                } else if constexpr (XP) {
                    const NbrPairs<NV, decltype(nbrld)> nbr{nbrld};
                    march_level_core<NV, V>(st, rowld, nbr, zc, outf, first, have_up, compute, kc, kk);
                } else {
                    const NbrShfl<NV, LX, V, decltype(edgeld)> nbr{edgeld, xl};
                    march_level_core<NV, V>(st, rowld, nbr, zc, outf, first, have_up, compute, kc, kk);
                }
            } else {
                march_level<NV, LX>(st, rowld, edgeld, out, xl, first, have_up, compute, kc, kk, nzp2);
            }
        }
#if PW_MARCH_SPLIT_ARRIVE
        // this warp is done with the plane of level kk; the last warp to say
        // so refills its slot with plane lp + S (the counter is reset before
        // the refill's arrive, whose release the next users acquire)
        __syncwarp();
        if (lane == 0 && ok) {
            const int s = slot(lp);
            if (atom_add_acq_rel_cta(&sm.cnt[s], 1u) == (uint32_t)(L::WARPS - 1)) {
                sm.cnt[s] = 0;
                if (lp + S < np) {
                    fence_proxy_async_smem();
                    issue(lp + S);
                    atomicMax(const_cast<int*>(&sm.flag[2]), lp + S + 1);
                }
            }
        }
        return !*abort_flag;
#else
        if constexpr (!SYNC) {
            return true;   // the planes of level kk are released at the next barrier
        } else {
            __syncthreads();
            if (*abort_flag) return false;
            // every plane up to lp is free: refill the slots of those not yet
            // refilled (one after a level with its own barrier, two after a
            // pair of levels)
            if (tid == 0) {
                for (; issued < np && issued <= lp + S; ++issued) {
                    fence_proxy_async_smem();
                    issue(issued);   // plane `issued` into the slot of plane issued - S
                }
            }
            return true;
        }
#endif
    };

    // The tile's first level (rows loaded, maybe only priming), then the
    // steady levels, then the top level of the grid if the tile reaches it.
    // Steady levels kk > pb always compute (kk >= kb, kk >= 2) and, below the
    // top, always have level kk+1.  The x-pair form takes two steady levels
    // per iteration (PW_MARCH_UNROLL_XP), so the carried rows change places
    // by register renaming rather than moves.
    // With PW_MARCH_PAIR_SYNC the x-pair form's two levels of an iteration
    // share one CTA barrier: after the second, the planes of both are free.
    using Fast = std::integral_constant<bool, PW_MARCH_FAST != 0>;
    using Gen = std::integral_constant<bool, false>;
    using Sync = std::integral_constant<bool, true>;
    using NoSync = std::integral_constant<bool, false>;   // (ignored with PW_MARCH_SPLIT_ARRIVE)
    // (One loop holding one general and one steady-pair body, smaller code,
    // measured slower: BF16 380 against 382, steps 322 against 345.)
    const int kfast = (ke == nz) ? ke - 1 : ke;
    bool aborted = !level(pb, Gen{}, Sync{});
    int kk = pb + 1;
    if constexpr (XP && PW_MARCH_PAIR_SYNC) {
        for (; kk + 1 <= kfast && !aborted; kk += 2)
            if (!level(kk, Fast{}, NoSync{}) || !level(kk + 1, Fast{}, Sync{})) aborted = true;
    } else {
        constexpr int kUnroll = XP ? PW_MARCH_UNROLL_XP : PW_MARCH_UNROLL;
#pragma unroll kUnroll
        for (; kk <= kfast && !aborted; ++kk)
            if (!level(kk, Fast{}, Sync{})) aborted = true;
    }
    for (; kk <= ke && !aborted; ++kk)
        if (!level(kk, Gen{}, Sync{})) aborted = true;

#if PW_MARCH_SPLIT_ARRIVE
    // every warp has left the march (each wait is bounded): the ring is free
    // for the next tile, and an abort by any warp is visible
    __syncthreads();
    aborted = *abort_flag != 0;
    if (aborted && tid == 0) {
        report_error(err, DEV_TIMEOUT_TMA_WAIT);
        // let the copies still in flight land before the CTA's smem is released:
        // planes issued are below flag[2], and only the last S of them can be
        // outstanding (a slot is refilled only after all warps consumed it)
        const int hi = sm.flag[2];
        for (int p = max(hi - S, 0); p < hi; ++p) mbar_wait_bounded(&bars[slot(p)], parity(p), kDrainLimitNs);
    }
    (void)waited;
    (void)issued;
#else
    if (aborted && tid == 0) {
        report_error(err, DEV_TIMEOUT_TMA_WAIT);
        // let the copies still in flight land before the CTA's smem is released
        for (int p = waited; p < issued; ++p)
            if (!mbar_wait_bounded(&bars[slot(p)], parity(p), kDrainLimitNs)) break;
    }
#endif
    (void)tbase;
    return !aborted;
}

// One grid, one tile per CTA: blockIdx = (tile column, tile row, k segment).
template <typename T, int LX, int TY, int S, int MODE, int NC, int RP, int XP>
__global__ void __launch_bounds__(TmaLayout<T, LX, TY, S, NC, RP, XP>::THREADS,
                                  (tma_min_blocks<T, LX, TY, S, NC, RP, XP>()))
    tma_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_v,
               const __grid_constant__ CUtensorMap tm_w, T* __restrict__ o0, T* __restrict__ o1,
               T* __restrict__ o2, const GridDev g, const int ox, const int nseg, const int seg0, const FoldedCoef kc,
               const float dt, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MarchSmem<T, LX, TY, S, NC, RP, XP> sm(smem_raw);
    const int bz = seg0 + blockIdx.z;
    const int kb = 1 + (int)(((long long)bz * g.nz) / nseg);
    const int ke = (int)(((long long)(bz + 1) * g.nz) / nseg);
    if (ke < kb) return;   // empty k segment (the host never launches one)
    sm.init(threadIdx.y * 32 + threadIdx.x);
    uint32_t ring = 0;
    march_tile<T, LX, TY, S, MODE, NC, RP, XP>(sm, &tm_u, &tm_v, &tm_w, o0, o1, o2, g, ox, kc, dt, blockIdx.x,
                                               blockIdx.y, kb, ke, ring, err);
}

// Instantiated single-grid launch shapes: (lanes per row, rows, stages, cells
// per thread along x, rows per thread, x pairs).  8 cells per thread, the
// packed two-row form and the x-pair form are instantiated for 16-bit
// storage only (8 cells: one 16-byte shared-memory access per row vector; two
// rows and x pairs: the 16-bit values unpack straight into FP32x2 operands,
// where FP32 rows would need register moves).
#define PW_TMA_CONFIGS(X) X(32, 4, 4, 4, 1, 0) X(32, 8, 3, 4, 1, 0) X(32, 8, 4, 4, 1, 0) X(32, 8, 6, 4, 1, 0) \
    X(32, 16, 3, 4, 1, 0) X(16, 4, 4, 4, 1, 0) X(16, 8, 4, 4, 1, 0) X(16, 4, 4, 8, 1, 0) X(16, 8, 4, 8, 1, 0)   \
    X(32, 8, 4, 4, 2, 0) X(32, 16, 4, 4, 2, 0) X(16, 8, 4, 4, 2, 0)                                            \
    X(16, 4, 4, 8, 1, 1) X(16, 8, 4, 8, 1, 1) X(16, 16, 4, 8, 1, 1) X(32, 4, 4, 4, 1, 1) X(32, 8, 4, 4, 1, 1)   \
    X(16, 8, 4, 4, 1, 1) X(8, 8, 4, 8, 1, 1) X(8, 16, 4, 8, 1, 1) X(8, 16, 4, 4, 1, 0) X(32, 16, 4, 4, 1, 0)      \
    X(16, 16, 4, 4, 1, 0)

template <typename T, int NC, int RP, int XP = 0>
constexpr bool nc_ok() { return (NC == 4 && RP == 1 && XP == 0) || sizeof(T) == 2; }

template <typename T, int LX, int TY, int S, int MODE, int NC, int RP, int XP>
static cudaError_t launch_tma_inst(const GridDev& g, int ox, const CUtensorMap* maps, void* o0, void* o1,
                                   void* o2, const Scales& sc, const CoefDev& cf, float dt, int* err, int nseg,
                                   int seg0, int seg_count, cudaStream_t s) {
  if constexpr (!nc_ok<T, NC, RP, XP>()) {
    return cudaErrorInvalidConfiguration;
  } else {
    using L = TmaLayout<T, LX, TY, S, NC, RP, XP>;
    auto kern = tma_kernel<T, LX, TY, S, MODE, NC, RP, XP>;
    cudaError_t e = set_smem_attr_once(kern, (int)L::SMEM);
    if (e != cudaSuccess) return e;
    if (seg_count <= 0) seg_count = nseg - seg0;
    dim3 grid((g.nx + L::TX - 1) / L::TX, (g.ny + TY - 1) / TY, seg_count);
    dim3 block(32, L::WARPS);
    kern<<<grid, block, L::SMEM, s>>>(maps[0], maps[1], maps[2], (T*)o0, (T*)o1, (T*)o2, g, ox, nseg, seg0,
                                      fold_coef(cf, sc), dt, err);
    return cudaGetLastError();
  }
}

template <typename T, int MODE>
static cudaError_t launch_tma_mode(const GridDev& g, int ox, const CUtensorMap* maps, void* o0, void* o1, void* o2,
                                   const Scales& sc, const CoefDev& cf, float dt, int* err,
                                   const TmaConfig& c, cudaStream_t s) {
#define PW_DISPATCH(LX_, TY_, S_, NC_, RP_, XP_)                                                        \
    if (c.lx == LX_ && c.ty == TY_ && c.stages == S_ && c.nc == NC_ && c.rp == RP_ && c.xp == XP_)      \
        return launch_tma_inst<T, LX_, TY_, S_, MODE, NC_, RP_, XP_>(g, ox, maps, o0, o1, o2, sc, cf, dt, err, \
                                                                     c.nseg, c.seg0, c.seg_count, s);
    PW_TMA_CONFIGS(PW_DISPATCH)
#undef PW_DISPATCH
    return cudaErrorInvalidConfiguration;
}

}  // namespace pw
