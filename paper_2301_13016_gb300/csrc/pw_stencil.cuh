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
    template <int N>
    static __device__ __forceinline__ void storevec(T* o0, T* o1, T* o2, long long o, const float (&a)[N],
                                                    const float (&b)[N], const float (&c)[N], const GridDev&, int,
                                                    int) {
        storev<N>(o0 + o, a);
        storev<N>(o1 + o, b);
        storev<N>(o2 + o, c);
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
    // a vector of N cells (j, i0..i0+N-1), i0 = 1 mod N, nx = 0 mod N
    template <typename T, int N>
    static __device__ __forceinline__ void vec(T* o0, T* o1, T* o2, long long o, const float (&a)[N],
                                               const float (&b)[N], const float (&c)[N], const GridDev& g, int j,
                                               int i0) {
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
            if (s > 0) {   // the row image
                storev<N>(o0 + p, a);
                storev<N>(o1 + p, b);
                storev<N>(o2 + p, c);
            }
#pragma unroll
            for (int q = 0; q < N; ++q) {
                const int i = i0 + q;
                auto put = [&](long long x) {
                    o0[x] = Store<T>::from_f(a[q]);
                    o1[x] = Store<T>::from_f(b[q]);
                    o2[x] = Store<T>::from_f(c[q]);
                };
                if (west && i <= H) put(p + q + g.nx);           // i -> i + nx
                if (east && i > g.nx - H) put(p + q - g.nx);     // i -> i - nx
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
    // a vector of N cells (j, i0..i0+N-1), i0 = 1 mod N, nx = 0 mod N
    template <int N>
    static __device__ __forceinline__ void storevec(T* o0, T* o1, T* o2, long long o, const float (&a)[N],
                                                    const float (&b)[N], const float (&c)[N], const GridDev& g, int j,
                                                    int i0) {
        storev<N>(o0 + o, a);
        storev<N>(o1 + o, b);
        storev<N>(o2 + o, c);
        if (g.halo != 1) return;   // deeper halos are refreshed by the halo kernel
        const bool west = (i0 == 1), east = (i0 + N - 1 == g.nx);
        // most row vectors touch no boundary: one test, the same at every level
        if (!(west | east | (j == 1) | (j == g.ny))) return;
        const long long dyp = (j == 1) ? (long long)g.ny * g.pj : 0;
        const long long dym = (j == g.ny) ? -(long long)g.ny * g.pj : 0;
        auto cell = [&](long long p, int q) {
            o0[p] = Store<T>::from_f(a[q]);
            o1[p] = Store<T>::from_f(b[q]);
            o2[p] = Store<T>::from_f(c[q]);
        };
        const long long shifts[3] = {0, dyp, dym};
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            if (s > 0 && shifts[s] == 0) continue;
            const long long p = o + shifts[s];
            if (s > 0) {   // the row image
                storev<N>(o0 + p, a);
                storev<N>(o1 + p, b);
                storev<N>(o2 + p, c);
            }
            if (west) cell(p + g.nx, 0);                   // cell i = 1 -> i = nx+1
            if (east) cell(p + (N - 1) - g.nx, N - 1);     // cell i = nx -> i = 0
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

// Source terms (Sec. 2.2) of level kk, handed to `out`, then the roll of `st`
// to level kk+1.  The data source is abstract:
//   row(f, up, dr, o)  the thread's NC values of field f (F_U, F_V, F_W) in
//                      row r+dr of level kk+up (up = 0 or 1)
//   edge(f, up, dr)    the x neighbour beyond the row's ends: x = -1 for the
//                      row's first lane, x = NC*LX for its last lane
//   out(ru, rv, rw, u, v, w)   the source terms and the level-kk values
// first:   kk is the first level of the march (its rows are loaded here)
// have_up: level kk+1 exists (kk < nz): the upper vertical fluxes and sw
// compute: evaluate the source terms (else they are zero: k = 1, or a level
//          that only primes the carried state)
// x neighbours within a row come from the adjacent lanes by warp shuffles
// (LX lanes per row).  Pair sums along x are shared by neighbouring cells.
template <int NC, int LX, typename V, class Row, class Edge, class Out>
__device__ __forceinline__ void march_level(MarchRegs<NC, V>& st, const Row& row, const Edge& edge, const Out& out,
                                            const int xl, const bool first, const bool have_up, const bool compute,
                                            const FoldedCoef& k, const int kk, const int nzp2) {
    using O = VOps<V>;
    // x-neighbours of a row vector: value at x = -1 (m) and x = NC (p)
    auto nbr_m = [&](const V (&x)[NC], V e) { return O::sel(xl == 0, e, O::shfl_up(x[NC - 1], LX)); };
    auto nbr_p = [&](const V (&x)[NC], V e) { return O::sel(xl == LX - 1, e, O::shfl_down(x[0], LX)); };
    if (first) {
        row(F_U, 0, 0, st.u0);
        row(F_V, 0, 0, st.v0);
        row(F_V, 0, -1, st.vs);
        row(F_W, 0, 0, st.w0);
    }
    V wn[NC];
    row(F_W, 0, 1, wn);
    const V ew = edge(F_W, 0, 0);
    V W[NC + 2];   // x = -1..NC
    W[0] = nbr_m(st.w0, ew);
    W[NC + 1] = nbr_p(st.w0, ew);
#pragma unroll
    for (int c = 0; c < NC; ++c) W[c + 1] = st.w0[c];

    // level kk+1 rows (upper terms; carried into the next step)
    V uu[NC], vu[NC], vus[NC], wu[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) uu[c] = vu[c] = vus[c] = wu[c] = O::zero();
    V euu = O::zero();
    if (have_up) {
        row(F_U, 1, 0, uu);
        row(F_V, 1, 0, vu);
        row(F_V, 1, -1, vus);
        row(F_W, 1, 0, wu);
        euu = edge(F_U, 1, 0);
    }
    // upper vertical pair sums of level kk = lower ones of level kk+1
    V pzu_n[NC], pzv_n[NC], pzw_n[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        pzu_n[c] = O::add(W[c + 1], W[c + 2]);   // w(k,i) + w(k,i+1)
        pzv_n[c] = O::add(st.w0[c], wn[c]);      // w(k,j) + w(k,j+1)
        pzw_n[c] = O::add(st.w0[c], wu[c]);      // w(k) + w(k+1)
    }

    V ru[NC], rv[NC], rw[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) ru[c] = rv[c] = rw[c] = O::zero();
    if (compute) {
        // per output field: x, y and lower vertical coefficients (storage scales folded in)
        const V kxu = O::splat(k.kx[0]), kxv = O::splat(k.kx[1]), kxw = O::splat(k.kx[2]);
        const V kyu = O::splat(k.ky[0]), kyv = O::splat(k.ky[1]), kyw = O::splat(k.ky[2]);
        V us[NC], un[NC], vn[NC], ws[NC];
        row(F_U, 0, -1, us);
        row(F_U, 0, 1, un);
        row(F_V, 0, 1, vn);
        row(F_W, 0, -1, ws);
        const V eu = edge(F_U, 0, 0);
        const V ev = edge(F_V, 0, 0);
        const V eun = edge(F_U, 0, 1);
        const V evs = edge(F_V, 0, -1);
        V U[NC + 2], Vv[NC + 2];   // x = -1..NC
        V UN[NC + 1], UU[NC + 1];  // x = -1..NC-1
        V VS[NC + 1];              // x = 0..NC
        U[0] = nbr_m(st.u0, eu);
        U[NC + 1] = nbr_p(st.u0, eu);
        Vv[0] = nbr_m(st.v0, ev);
        Vv[NC + 1] = nbr_p(st.v0, ev);
        UN[0] = nbr_m(un, eun);
        UU[0] = nbr_m(uu, euu);
        VS[NC] = nbr_p(st.vs, evs);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            U[c + 1] = st.u0[c];
            Vv[c + 1] = st.v0[c];
            UN[c + 1] = un[c];
            UU[c + 1] = uu[c];
            VS[c] = st.vs[c];
        }

        // pair sums along x shared by neighbouring cells: index c is the
        // pair (x = c-1, c)
        V pxu[NC + 1], qx[NC + 1], rx[NC + 1], pxv[NC], pys[NC];
#pragma unroll
        for (int c = 0; c < NC + 1; ++c) {
            pxu[c] = O::add(U[c], U[c + 1]);   // u(i-1) + u(i)
            qx[c] = O::add(U[c], UN[c]);       // u(j,i-1) + u(j+1,i-1)
            rx[c] = O::add(U[c], UU[c]);       // u(k,i-1) + u(k+1,i-1)
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            pxv[c] = O::add(Vv[c + 1], Vv[c + 2]);   // v(j,i) + v(j,i+1)
            pys[c] = O::add(VS[c], VS[c + 1]);       // v(j-1,i) + v(j-1,i+1)
        }
        const float t1 = __ldg(k.tz + kk);
        const V tz1u = O::splat(t1 * k.kz[0]), tz1v = O::splat(t1 * k.kz[1]);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            // su
            V x = O::mul(kxu, O::fma(O::neg(U[c + 2]), pxu[c + 1], O::mul(U[c], pxu[c])));
            x = O::fma(kyu, O::fma(O::neg(un[c]), pxv[c], O::mul(us[c], pys[c])), x);
            ru[c] = O::fma(tz1u, st.pdu[c], x);
            // sv
            V y = O::mul(kxv, O::fma(O::neg(Vv[c + 2]), qx[c + 1], O::mul(Vv[c], qx[c])));
            y = O::fma(kyv,
                       O::fma(O::neg(vn[c]), O::add(Vv[c + 1], vn[c]), O::mul(st.vs[c], O::add(Vv[c + 1], st.vs[c]))),
                       y);
            rv[c] = O::fma(tz1v, st.pdv[c], y);
        }
        if (have_up) {   // kk < nz: upper vertical fluxes and sw
            const float t2 = __ldg(k.tz + nzp2 + kk);
            const float d1 = __ldg(k.tz + 2 * nzp2 + kk);
            const float d2 = __ldg(k.tz + 3 * nzp2 + kk);
            const V ntz2u = O::splat(-(t2 * k.kz[0])), ntz2v = O::splat(-(t2 * k.kz[1]));
            const V td1w = O::splat(d1 * k.kz[2]), ntd2w = O::splat(-(d2 * k.kz[2]));
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                ru[c] = O::fma(ntz2u, O::mul(uu[c], pzu_n[c]), ru[c]);
                rv[c] = O::fma(ntz2v, O::mul(vu[c], pzv_n[c]), rv[c]);
                V z = O::mul(kxw, O::fma(O::neg(W[c + 2]), rx[c + 1], O::mul(W[c], rx[c])));
                z = O::fma(kyw, O::fma(O::neg(wn[c]), O::add(Vv[c + 1], vu[c]), O::mul(ws[c], O::add(st.vs[c], vus[c]))),
                           z);
                z = O::fma(td1w, st.pdw[c], z);
                rw[c] = O::fma(ntd2w, O::mul(wu[c], pzw_n[c]), z);
            }
        }
    }

    out(ru, rv, rw, st.u0, st.v0, st.w0);

    // roll: the lower flux products of level kk+1, then level kk+1 becomes level kk
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        st.pdu[c] = O::mul(st.u0[c], pzu_n[c]);   // u(k) * (w(k,i) + w(k,i+1))
        st.pdv[c] = O::mul(st.v0[c], pzv_n[c]);   // v(k) * (w(k,j) + w(k,j+1))
        st.pdw[c] = O::mul(st.w0[c], pzw_n[c]);   // w(k) * (w(k) + w(k+1))
        st.u0[c] = uu[c];
        st.v0[c] = vu[c];
        st.vs[c] = vus[c];
        st.w0[c] = wu[c];
    }
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
// LX lanes cover one row (LX = 32: one warp per row; LX = 16: two rows per
// warp, for narrow grids).  A thread computes NC consecutive cells along x,
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
template <typename T, int LX, int TY, int S, int NC = 4, int RP = 1>
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
    static constexpr size_t SMEM = (size_t)S * STAGE * sizeof(T) + S * sizeof(uint64_t) + 16 + 4 * S;
    static_assert(LX == 32 || LX == 16, "LX must be 16 or 32");
    static_assert(NC == 4 || NC == 8, "4 or 8 cells per thread");
    static_assert(BW <= 256, "a TMA box is at most 256 elements wide");
    static_assert(TY % (RPW * RP) == 0, "TY must be a multiple of the rows per warp");
    static_assert(RP == 1 || RP == 2, "one or two rows per thread");
};

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

// Resident CTAs per SM the register budget is sized for: what shared memory
// and the thread limit allow, at most PW_TMA_MAX_MINB for 4 cells a thread;
// 8 cells a thread (8 x 1 or 4 x 2) get PW_TMA_REGS8 = 168 registers, which
// measured best on GB300 (16 lanes x 8 cells x 4 rows: 269 -> 295 Gcell/s for
// BF16 against the compiler's 210 registers, as more CTAs per SM hide more
// latency; 128 spills and 200 leaves 2 CTAs per SM, both slower).
template <typename T, int LX, int TY, int S, int NC = 4, int RP = 1>
constexpr int tma_min_blocks() {
    using L = TmaLayout<T, LX, TY, S, NC, RP>;
    constexpr int by_smem = (int)((227u * 1024u) / L::SMEM);
    constexpr int by_threads = 2048 / L::THREADS;
    constexpr int by_regs = NC * RP == 8 ? 65536 / (L::THREADS * PW_TMA_REGS8) : PW_TMA_MAX_MINB;
    constexpr int m0 = by_smem < by_threads ? by_smem : by_threads;
    constexpr int m = m0 < by_regs ? m0 : by_regs;
    return m < 1 ? 1 : m;
}

// Shared memory of a k-march CTA: the plane ring, one mbarrier per slot, the
// flags and one release counter per slot.
template <typename T, int LX, int TY, int S, int NC = 4, int RP = 1>
struct MarchSmem {
    using L = TmaLayout<T, LX, TY, S, NC, RP>;
    T* stages;
    uint64_t* bars;
    volatile int* flag;   // [0] abort, [1] work item broadcast, [2] planes issued (highest + 1)
    uint32_t* cnt;        // warps done with each slot's plane
    __device__ __forceinline__ MarchSmem(unsigned char* raw) {
        stages = reinterpret_cast<T*>(raw);
        bars = reinterpret_cast<uint64_t*>(raw + (size_t)S * L::STAGE * sizeof(T));
        flag = reinterpret_cast<volatile int*>(bars + S);
        cnt = reinterpret_cast<uint32_t*>(bars + S) + 4;
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

// March one tile: columns bx, rows by, output levels kb..ke of grid g.
// `ring` counts the planes this CTA issued before; it is advanced by the
// planes of this tile.  Returns false if a wait timed out (the error is
// recorded and the copies in flight are drained).
template <typename T, int LX, int TY, int S, int MODE, int NC = 4, int RP = 1>
__device__ __forceinline__ bool march_tile(const MarchSmem<T, LX, TY, S, NC, RP>& sm, const CUtensorMap* tm_u,
                                           const CUtensorMap* tm_v, const CUtensorMap* tm_w, T* __restrict__ o0,
                                           T* __restrict__ o1, T* __restrict__ o2, const GridDev& g, const int ox,
                                           const FoldedCoef& kc, const float dt, const int bx, const int by,
                                           const int kb, const int ke, uint32_t& ring, int* __restrict__ err) {
    using L = TmaLayout<T, LX, TY, S, NC, RP>;
    using V = typename std::conditional<RP == 1, float, float2>::type;
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

    MarchRegs<NC, V> st;
    st.zero();
    int waited = 0;   // planes 0..waited-1 are known complete
    int lp = 0;       // plane index of the level being marched

    // the staged planes of level kk (up = 0) and kk+1 (up = 1); with RP = 2
    // each value pairs row r+dr (x) with row r+dr+1 (y)
    auto rowld = [&](int f, int up, int dr, V (&o)[NC]) {
        const T* P = stages + slot(lp + up) * L::STAGE + f * L::FIELD + (r + dr) * BW + c0;
        if constexpr (RP == 1) {
            ld(P, o);
        } else {
            float a[NC], b[NC];
            ld(P, a);
            ld(P + BW, b);
#pragma unroll
            for (int q = 0; q < NC; ++q) o[q] = make_float2(a[q], b[q]);
        }
    };
    auto edgeld = [&](int f, int up, int dr) -> V {
        const T* P = stages + slot(lp + up) * L::STAGE + f * L::FIELD + (r + dr) * BW + ce;
        if constexpr (RP == 1)
            return ld1(P);
        else
            return make_float2(ld1(P), ld1(P + BW));
    };

    // One level of the march.  Returns false on abort.
    auto level = [&](const int kk) -> bool {
        lp = kk - pb;
        bool ok = true;
        if (lp == 0) ok = mbar_wait_bounded(&bars[slot(0)], parity(0), kWaitLimitNs);
        const bool have_up = (kk + 1 <= pe);
        if (ok && have_up) ok = mbar_wait_bounded(&bars[slot(lp + 1)], parity(lp + 1), kWaitLimitNs);
        ok = __all_sync(FULL, ok);
        if (!ok) *abort_flag = 1;
        if (ok) {
            waited = lp + (have_up ? 2 : 1);
            // one row of outputs (values of row `half` of each V)
            auto out_row = [&](const V (&ru)[NC], const V (&rv)[NC], const V (&rw)[NC], const V (&u0)[NC],
                               const V (&v0)[NC], const V (&w0)[NC], const int half) {
                auto comp = [&](const V& x) -> float {
                    if constexpr (RP == 1)
                        return x;
                    else
                        return half ? x.y : x.x;
                };
                float a[NC], b[NC], d[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (MODE == MODE_STEP) {   // at kk = 1 the source terms are 0
                        a[c] = fmaf(dt, comp(ru[c]), comp(u0[c]));
                        b[c] = fmaf(dt, comp(rv[c]), comp(v0[c]));
                        d[c] = fmaf(dt, comp(rw[c]), comp(w0[c]));
                    } else {
                        a[c] = comp(ru[c]);
                        b[c] = comp(rv[c]);
                        d[c] = comp(rw[c]);
                    }
                }
                Epilogue<T, MODE>::template storevec<NC>(o0, o1, o2,
                                                         row_off + (long long)half * g.pj + (long long)kk * g.pk, a,
                                                         b, d, g, j + half, i0);
            };
            auto out = [&](const V (&ru)[NC], const V (&rv)[NC], const V (&rw)[NC], const V (&u0)[NC],
                           const V (&v0)[NC], const V (&w0)[NC]) {
                if (kk < kb) return;
                if (valid) out_row(ru, rv, rw, u0, v0, w0, 0);
                if (RP == 2 && valid2) out_row(ru, rv, rw, u0, v0, w0, 1);
            };
            march_level<NC, LX>(st, rowld, edgeld, out, xl, lp == 0, have_up, (kk >= kb) && (kk >= 2), kc, kk,
                                nzp2);
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
        __syncthreads();
        if (*abort_flag) return false;
        if (tid == 0 && issued < np) {
            fence_proxy_async_smem();
            issue(issued);   // plane lp + S into the slot level kk just released
            ++issued;
        }
        return true;
#endif
    };

    // One level per loop iteration.  (Two or three per iteration, so that the
    // carried rows rotate by register renaming instead of moves, cost
    // registers and CTAs per SM and measured 15-25 % slower on GB300; reloading
    // the level's rows from the staged plane instead of carrying them gained
    // nothing either.)
    bool aborted = false;
    for (int kk = pb; kk <= ke && !aborted; ++kk)
        if (!level(kk)) aborted = true;

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
    return !aborted;
}

// One grid, one tile per CTA: blockIdx = (tile column, tile row, k segment).
template <typename T, int LX, int TY, int S, int MODE, int NC, int RP>
__global__ void __launch_bounds__(TmaLayout<T, LX, TY, S, NC, RP>::THREADS,
                                  (tma_min_blocks<T, LX, TY, S, NC, RP>()))
    tma_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_v,
               const __grid_constant__ CUtensorMap tm_w, T* __restrict__ o0, T* __restrict__ o1,
               T* __restrict__ o2, const GridDev g, const int ox, const int nseg, const int seg0, const FoldedCoef kc,
               const float dt, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MarchSmem<T, LX, TY, S, NC, RP> sm(smem_raw);
    const int bz = seg0 + blockIdx.z;
    const int kb = 1 + (int)(((long long)bz * g.nz) / nseg);
    const int ke = (int)(((long long)(bz + 1) * g.nz) / nseg);
    if (ke < kb) return;   // empty k segment (the host never launches one)
    sm.init(threadIdx.y * 32 + threadIdx.x);
    uint32_t ring = 0;
    march_tile<T, LX, TY, S, MODE, NC, RP>(sm, &tm_u, &tm_v, &tm_w, o0, o1, o2, g, ox, kc, dt,
                                                   blockIdx.x, blockIdx.y, kb, ke, ring, err);
}

// Instantiated single-grid launch shapes: (lanes per row, rows, stages, cells
// per thread along x, rows per thread).  8 cells per thread and the packed
// two-row form are instantiated for 16-bit storage only (8 cells: one
// 16-byte shared-memory access per row vector; two rows: the 16-bit values
// unpack straight into row pairs, where FP32 rows would need register moves).
#define PW_TMA_CONFIGS(X) X(32, 4, 4, 4, 1) X(32, 8, 3, 4, 1) X(32, 8, 4, 4, 1) X(32, 8, 6, 4, 1) \
    X(32, 16, 3, 4, 1) X(16, 4, 4, 4, 1) X(16, 8, 4, 4, 1) X(16, 4, 4, 8, 1) X(16, 8, 4, 8, 1)        \
    X(32, 8, 4, 4, 2) X(32, 16, 4, 4, 2) X(16, 8, 4, 4, 2)

template <typename T, int NC, int RP>
constexpr bool nc_ok() { return (NC == 4 && RP == 1) || sizeof(T) == 2; }

template <typename T, int LX, int TY, int S, int MODE, int NC, int RP>
static cudaError_t launch_tma_inst(const GridDev& g, int ox, const CUtensorMap* maps, void* o0, void* o1,
                                   void* o2, const Scales& sc, const CoefDev& cf, float dt, int* err, int nseg,
                                   int seg0, int seg_count, cudaStream_t s) {
  if constexpr (!nc_ok<T, NC, RP>()) {
    return cudaErrorInvalidConfiguration;
  } else {
    using L = TmaLayout<T, LX, TY, S, NC, RP>;
    auto kern = tma_kernel<T, LX, TY, S, MODE, NC, RP>;
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
#define PW_DISPATCH(LX_, TY_, S_, NC_, RP_)                                                                   \
    if (c.lx == LX_ && c.ty == TY_ && c.stages == S_ && c.nc == NC_ && c.rp == RP_)                           \
        return launch_tma_inst<T, LX_, TY_, S_, MODE, NC_, RP_>(g, ox, maps, o0, o1, o2, sc, cf, dt, err, c.nseg, \
                                                                c.seg0, c.seg_count, s);
    PW_TMA_CONFIGS(PW_DISPATCH)
#undef PW_DISPATCH
    return cudaErrorInvalidConfiguration;
}

}  // namespace pw
