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

// MODE_STEP writes, with each cell, its periodic images in the lateral halo
// of depth H = g.halo (H <= nx and H <= ny, which the grid check enforces):
// cell i <= H also goes to i + nx, cell i > nx - H to i - nx, and likewise in
// y, corners included, so the next step reads a complete halo.
template <typename T>
struct Epilogue<T, MODE_STEP> {
    // one cell (j, i) at offset o
    static __device__ __forceinline__ void store1(T* o0, T* o1, T* o2, long long o, float a, float b, float c,
                                                  const GridDev& g, int j, int i) {
        const T ta = Store<T>::from_f(a), tb = Store<T>::from_f(b), tc = Store<T>::from_f(c);
        auto put = [&](long long p) {
            o0[p] = ta;
            o1[p] = tb;
            o2[p] = tc;
        };
        put(o);
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
    template <int N>
    static __device__ __forceinline__ void storevec(T* o0, T* o1, T* o2, long long o, const float (&a)[N],
                                                    const float (&b)[N], const float (&c)[N], const GridDev& g, int j,
                                                    int i0) {
        storev<N>(o0 + o, a);
        storev<N>(o1 + o, b);
        storev<N>(o2 + o, c);
        const int H = g.halo;
        const bool west = (i0 <= H), east = (i0 + N - 1 > g.nx - H);
        const long long dyp = (j <= H) ? (long long)g.ny * g.pj : 0;
        const long long dym = (j > g.ny - H) ? -(long long)g.ny * g.pj : 0;
        if (!west && !east && !dyp && !dym) return;
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
#pragma unroll
            for (int q = 0; q < N; ++q) {
                if (west && i0 + q <= H) cell(p + q + g.nx, q);          // i -> i + nx
                if (east && i0 + q > g.nx - H) cell(p + q - g.nx, q);    // i -> i - nx
            }
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
// One level of a k-march for the NC consecutive cells of one thread (shared
// by every k-march kernel: single step, two-step temporal blocking, batch).
//
// MarchRegs is what a thread carries from level kk to kk+1: the level-kk rows
// it loaded as level kk+1 on the previous step, the level kk-1 values at its
// cells (a rolling window in z) and the three vertical pair sums of the upper
// fluxes, which are the lower pair sums of the next level.
template <int NC>
struct MarchRegs {
    float u0[NC], v0[NC], vs[NC], w0[NC];   // level kk: u, v, w in row r; vs = v in row r-1
    float ud[NC], vd[NC], wd[NC];           // level kk-1 at the cells
    float pzu[NC], pzv[NC], pzw[NC];        // lower vertical pair sums of level kk
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            ud[c] = vd[c] = wd[c] = pzu[c] = pzv[c] = pzw[c] = 0.f;
            u0[c] = v0[c] = vs[c] = w0[c] = 0.f;
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
template <int NC, int LX, class Row, class Edge, class Out>
__device__ __forceinline__ void march_level(MarchRegs<NC>& st, const Row& row, const Edge& edge, const Out& out,
                                            const int xl, const bool first, const bool have_up, const bool compute,
                                            const float tcx, const float tcy, const float* __restrict__ tz,
                                            const int kk, const int nzp2) {
    const unsigned FULL = 0xffffffffu;
    // x-neighbours of a row vector: value at x = -1 (m) and x = NC (p)
    auto nbr_m = [&](const float (&x)[NC], float e) {
        float m = __shfl_up_sync(FULL, x[NC - 1], 1, LX);
        return xl == 0 ? e : m;
    };
    auto nbr_p = [&](const float (&x)[NC], float e) {
        float p = __shfl_down_sync(FULL, x[0], 1, LX);
        return xl == LX - 1 ? e : p;
    };
    if (first) {
        row(F_U, 0, 0, st.u0);
        row(F_V, 0, 0, st.v0);
        row(F_V, 0, -1, st.vs);
        row(F_W, 0, 0, st.w0);
    }
    float wn[NC];
    row(F_W, 0, 1, wn);
    const float ew = edge(F_W, 0, 0);
    float W[NC + 2];   // x = -1..NC
    W[0] = nbr_m(st.w0, ew);
    W[NC + 1] = nbr_p(st.w0, ew);
#pragma unroll
    for (int c = 0; c < NC; ++c) W[c + 1] = st.w0[c];

    // level kk+1 rows (upper terms; carried into the next step)
    float uu[NC], vu[NC], vus[NC], wu[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) uu[c] = vu[c] = vus[c] = wu[c] = 0.f;
    float euu = 0.f;
    if (have_up) {
        row(F_U, 1, 0, uu);
        row(F_V, 1, 0, vu);
        row(F_V, 1, -1, vus);
        row(F_W, 1, 0, wu);
        euu = edge(F_U, 1, 0);
    }
    // upper vertical pair sums of level kk = lower ones of level kk+1
    float pzu_n[NC], pzv_n[NC], pzw_n[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        pzu_n[c] = W[c + 1] + W[c + 2];    // w(k,i) + w(k,i+1)
        pzv_n[c] = st.w0[c] + wn[c];       // w(k,j) + w(k,j+1)
        pzw_n[c] = st.w0[c] + wu[c];       // w(k) + w(k+1)
    }

    float ru[NC], rv[NC], rw[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) ru[c] = rv[c] = rw[c] = 0.f;
    if (compute) {
        float us[NC], un[NC], vn[NC], ws[NC];
        row(F_U, 0, -1, us);
        row(F_U, 0, 1, un);
        row(F_V, 0, 1, vn);
        row(F_W, 0, -1, ws);
        const float eu = edge(F_U, 0, 0);
        const float ev = edge(F_V, 0, 0);
        const float eun = edge(F_U, 0, 1);
        const float evs = edge(F_V, 0, -1);
        float U[NC + 2], V[NC + 2];    // x = -1..NC
        float UN[NC + 1], UU[NC + 1];  // x = -1..NC-1
        float VS[NC + 1];              // x = 0..NC
        U[0] = nbr_m(st.u0, eu);
        U[NC + 1] = nbr_p(st.u0, eu);
        V[0] = nbr_m(st.v0, ev);
        V[NC + 1] = nbr_p(st.v0, ev);
        UN[0] = nbr_m(un, eun);
        UU[0] = nbr_m(uu, euu);
        VS[NC] = nbr_p(st.vs, evs);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            U[c + 1] = st.u0[c];
            V[c + 1] = st.v0[c];
            UN[c + 1] = un[c];
            UU[c + 1] = uu[c];
            VS[c] = st.vs[c];
        }

        // pair sums along x shared by neighbouring cells: index c is the
        // pair (x = c-1, c)
        float pxu[NC + 1], qx[NC + 1], rx[NC + 1], pxv[NC], pys[NC];
#pragma unroll
        for (int c = 0; c < NC + 1; ++c) {
            pxu[c] = U[c] + U[c + 1];     // u(i-1) + u(i)
            qx[c] = U[c] + UN[c];         // u(j,i-1) + u(j+1,i-1)
            rx[c] = U[c] + UU[c];         // u(k,i-1) + u(k+1,i-1)
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            pxv[c] = V[c + 1] + V[c + 2];  // v(j,i) + v(j,i+1)
            pys[c] = VS[c] + VS[c + 1];    // v(j-1,i) + v(j-1,i+1)
        }
        const float tz1 = __ldg(tz + kk);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            // su
            float x = tcx * fmaf(-U[c + 2], pxu[c + 1], U[c] * pxu[c]);
            x = fmaf(tcy, fmaf(-un[c], pxv[c], us[c] * pys[c]), x);
            ru[c] = fmaf(tz1, st.ud[c] * st.pzu[c], x);
            // sv
            float y = tcx * fmaf(-V[c + 2], qx[c + 1], V[c] * qx[c]);
            y = fmaf(tcy, fmaf(-vn[c], V[c + 1] + vn[c], st.vs[c] * (V[c + 1] + st.vs[c])), y);
            rv[c] = fmaf(tz1, st.vd[c] * st.pzv[c], y);
        }
        if (have_up) {   // kk < nz: upper vertical fluxes and sw
            const float tz2 = __ldg(tz + nzp2 + kk);
            const float td1 = __ldg(tz + 2 * nzp2 + kk);
            const float td2 = __ldg(tz + 3 * nzp2 + kk);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                ru[c] = fmaf(-tz2, uu[c] * pzu_n[c], ru[c]);
                rv[c] = fmaf(-tz2, vu[c] * pzv_n[c], rv[c]);
                float z = tcx * fmaf(-W[c + 2], rx[c + 1], W[c] * rx[c]);
                z = fmaf(tcy, fmaf(-wn[c], V[c + 1] + vu[c], ws[c] * (st.vs[c] + vus[c])), z);
                z = fmaf(td1, st.wd[c] * st.pzw[c], z);
                rw[c] = fmaf(-td2, wu[c] * pzw_n[c], z);
            }
        }
    }

    out(ru, rv, rw, st.u0, st.v0, st.w0);

    // roll: level kk becomes level k-1, level kk+1 becomes level kk
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        st.ud[c] = st.u0[c];
        st.vd[c] = st.v0[c];
        st.wd[c] = st.w0[c];
        st.pzu[c] = pzu_n[c];
        st.pzv[c] = pzv_n[c];
        st.pzw[c] = pzw_n[c];
        st.u0[c] = uu[c];
        st.v0[c] = vu[c];
        st.vs[c] = vus[c];
        st.w0[c] = wu[c];
    }
}

// ---------------------------------------------------------------------------
// TMA k-march.
//
// A tile is TX = 4*LX interior columns by TY rows and one k segment; the CTA
// marches up the column one level at a time.  Level planes of u, v, w (the
// tile plus a one-cell halo, widened in x to the 16-byte TMA granule) arrive
// in a ring of S shared-memory slots by 3D TMA box copies that one thread
// issues, each slot completing on its own mbarrier; S-1 planes are in flight
// ahead of the level being computed, so every input element is read from HBM
// once and the copy engine, not the warps, keeps bytes in flight.
//
// LX lanes cover one row (LX = 32: one warp per row; LX = 16: two rows per
// warp, for narrow grids).  A thread computes 4 consecutive cells along x.
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
template <typename T, int LX, int TY, int S, int NC = 4>
struct TmaLayout {
    static constexpr int TX = NC * LX;
    static constexpr int RPW = 32 / LX;                // rows per warp
    static constexpr int WARPS = TY / RPW;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int PADX = 16 / (int)sizeof(T);   // elements in one 16-byte granule
    static constexpr int BW = TX + 2 * PADX;           // box width
    static constexpr int ROWS = TY + 2;
    static constexpr int FIELD_RAW = BW * ROWS;
    static constexpr int FIELD_BYTES = ((FIELD_RAW * (int)sizeof(T) + 127) / 128) * 128;
    static constexpr int FIELD = FIELD_BYTES / (int)sizeof(T);
    static constexpr int STAGE = 3 * FIELD;
    static constexpr uint32_t TX_BYTES = 3u * FIELD_RAW * (uint32_t)sizeof(T);
    static constexpr size_t SMEM = (size_t)S * STAGE * sizeof(T) + S * sizeof(uint64_t) + 16;
    static_assert(LX == 32 || LX == 16, "LX must be 16 or 32");
    static_assert(NC == 4 || NC == 8, "4 or 8 cells per thread");
    static_assert(BW <= 256, "a TMA box is at most 256 elements wide");
    static_assert(TY % RPW == 0, "TY must be a multiple of the rows per warp");
};

// Build-time knob of the k-march kernel: PW_TMA_MAX_MINB caps the resident
// CTAs per SM the register budget is sized for (a cap of 3 made the 8-row
// shapes spill; 2 does not).
#ifndef PW_TMA_MAX_MINB
#define PW_TMA_MAX_MINB 2
#endif

// Resident CTAs per SM the register budget is sized for: what shared memory
// and the thread limit allow, at most PW_TMA_MAX_MINB.
template <typename T, int LX, int TY, int S, int NC = 4>
constexpr int tma_min_blocks() {
    using L = TmaLayout<T, LX, TY, S, NC>;
    constexpr int by_smem = (int)((227u * 1024u) / L::SMEM);
    constexpr int by_threads = 2048 / L::THREADS;
    constexpr int m = by_smem < by_threads ? by_smem : by_threads;
    return m < 1 ? 1 : (m > PW_TMA_MAX_MINB ? PW_TMA_MAX_MINB : m);
}

// Shared memory of a k-march CTA: the plane ring, one mbarrier per slot, and
// the abort flag / work-item word.
template <typename T, int LX, int TY, int S, int NC = 4>
struct MarchSmem {
    using L = TmaLayout<T, LX, TY, S, NC>;
    T* stages;
    uint64_t* bars;
    volatile int* flag;   // flag[0]: abort, flag[1]: work item broadcast
    __device__ __forceinline__ MarchSmem(unsigned char* raw) {
        stages = reinterpret_cast<T*>(raw);
        bars = reinterpret_cast<uint64_t*>(raw + (size_t)S * L::STAGE * sizeof(T));
        flag = reinterpret_cast<volatile int*>(bars + S);
    }
    // one thread, then a CTA barrier
    __device__ __forceinline__ void init(int tid) {
        if (tid == 0) {
            for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
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
template <typename T, int LX, int TY, int S, bool SCALED, int MODE, int NC = 4>
__device__ __forceinline__ bool march_tile(const MarchSmem<T, LX, TY, S, NC>& sm, const CUtensorMap* tm_u,
                                           const CUtensorMap* tm_v, const CUtensorMap* tm_w, T* __restrict__ o0,
                                           T* __restrict__ o1, T* __restrict__ o2, const GridDev& g, const int ox,
                                           const Scales& sc, const CoefDev& cf, const float dt, const int bx,
                                           const int by, const int kb, const int ke, uint32_t& ring,
                                           int* __restrict__ err) {
    using L = TmaLayout<T, LX, TY, S, NC>;
    constexpr int BW = L::BW;
    constexpr int PADX = L::PADX;
    constexpr int FU = 0, FV = L::FIELD, FW = 2 * L::FIELD;
    T* const stages = sm.stages;
    uint64_t* const bars = sm.bars;
    volatile int* const abort_flag = sm.flag;

    const int lane = threadIdx.x, warp = threadIdx.y;
    const int tid = warp * 32 + lane;
    const int xl = lane % LX;                          // lane within the row
    const int row = warp * L::RPW + lane / LX;         // 0 .. TY-1
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
    }

    const int r = row + 1;
    const int c0 = NC * xl + PADX;
    // tile-edge neighbour column: the row's first lane needs x = -1, its last
    // lane x = TX; the other lanes read the last lane's address (a broadcast)
    const int ce = (xl == 0) ? PADX - 1 : L::TX + PADX;
    const int j = TY * by + 1 + row;
    const int i0 = 1 + L::TX * bx + NC * xl;
    const bool valid = (j <= g.ny) && (i0 <= g.nx);
    const long long row_off = g.origin + (long long)j * g.pj + i0;
    const float tcx = cf.tcx, tcy = cf.tcy;
    const int nzp2 = nz + 2;
    const unsigned FULL = 0xffffffffu;
    auto ld = [&](const T* p, float (&o)[NC], float s) {
        loadv<NC>(p, o);
        if (SCALED) {
#pragma unroll
            for (int q = 0; q < NC; ++q) o[q] *= s;
        }
    };
    auto ld1 = [&](const T* p, float s) {
        float x = Store<T>::to_f(*p);
        return SCALED ? x * s : x;
    };
    const float s_in[3] = {sc.in[0], sc.in[1], sc.in[2]};

    MarchRegs<NC> st;
    st.zero();
    int waited = 0;   // planes 0..waited-1 are known complete
    int lp = 0;       // plane index of the level being marched

    // the staged planes of level kk (up = 0) and kk+1 (up = 1)
    auto rowld = [&](int f, int up, int dr, float (&o)[NC]) {
        ld(stages + slot(lp + up) * L::STAGE + f * L::FIELD + (r + dr) * BW + c0, o, s_in[f]);
    };
    auto edgeld = [&](int f, int up, int dr) {
        return ld1(stages + slot(lp + up) * L::STAGE + f * L::FIELD + (r + dr) * BW + ce, s_in[f]);
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
            auto out = [&](const float (&ru)[NC], const float (&rv)[NC], const float (&rw)[NC],
                           const float (&u0)[NC], const float (&v0)[NC], const float (&w0)[NC]) {
                if (!(kk >= kb && valid)) return;
                float a[NC], b[NC], d[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (MODE == MODE_STEP) {   // at kk = 1 the source terms are 0
                        a[c] = fmaf(dt, ru[c], u0[c]);
                        b[c] = fmaf(dt, rv[c], v0[c]);
                        d[c] = fmaf(dt, rw[c], w0[c]);
                    } else {
                        a[c] = ru[c];
                        b[c] = rv[c];
                        d[c] = rw[c];
                    }
                    if (SCALED) {
                        a[c] *= sc.out[0];
                        b[c] *= sc.out[1];
                        d[c] *= sc.out[2];
                    }
                }
                Epilogue<T, MODE>::template storevec<NC>(o0, o1, o2, row_off + (long long)kk * g.pk, a, b, d, g, j,
                                                         i0);
            };
            march_level<NC, LX>(st, rowld, edgeld, out, xl, lp == 0, have_up, (kk >= kb) && (kk >= 2), tcx, tcy,
                                cf.tz, kk, nzp2);
        }
        __syncthreads();
        if (*abort_flag) return false;
        if (tid == 0 && issued < np) {
            fence_proxy_async_smem();
            issue(issued);   // plane lp + S into the slot level kk just released
            ++issued;
        }
        return true;
    };

    bool aborted = false;
    for (int kk = pb; kk <= ke && !aborted; ++kk)
        if (!level(kk)) aborted = true;

    if (aborted && tid == 0) {
        report_error(err, DEV_TIMEOUT_TMA_WAIT);
        // let the copies still in flight land before the CTA's smem is released
        for (int p = waited; p < issued; ++p)
            if (!mbar_wait_bounded(&bars[slot(p)], parity(p), kDrainLimitNs)) break;
    }
    return !aborted;
}

// One grid, one tile per CTA: blockIdx = (tile column, tile row, k segment).
template <typename T, int LX, int TY, int S, bool SCALED, int MODE, int NC>
__global__ void __launch_bounds__(TmaLayout<T, LX, TY, S, NC>::THREADS, (tma_min_blocks<T, LX, TY, S, NC>()))
    tma_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_v,
               const __grid_constant__ CUtensorMap tm_w, T* __restrict__ o0, T* __restrict__ o1,
               T* __restrict__ o2, const GridDev g, const int ox, const int nseg, const int seg0, const Scales sc,
               const CoefDev cf, const float dt, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MarchSmem<T, LX, TY, S, NC> sm(smem_raw);
    const int bz = seg0 + blockIdx.z;
    const int kb = 1 + (int)(((long long)bz * g.nz) / nseg);
    const int ke = (int)(((long long)(bz + 1) * g.nz) / nseg);
    if (ke < kb) return;   // empty k segment (the host never launches one)
    sm.init(threadIdx.y * 32 + threadIdx.x);
    uint32_t ring = 0;
    march_tile<T, LX, TY, S, SCALED, MODE, NC>(sm, &tm_u, &tm_v, &tm_w, o0, o1, o2, g, ox, sc, cf, dt, blockIdx.x,
                                               blockIdx.y, kb, ke, ring, err);
}

// Instantiated single-grid launch shapes: (lanes per row, rows, stages, cells
// per thread).  8 cells per thread is instantiated for 16-bit storage only
// (one 16-byte shared-memory access per row vector).
#define PW_TMA_CONFIGS(X) X(32, 4, 4, 4) X(32, 8, 3, 4) X(32, 8, 4, 4) X(32, 8, 6, 4) X(32, 16, 3, 4) \
    X(16, 4, 4, 4) X(16, 8, 4, 4) X(16, 4, 4, 8) X(16, 8, 4, 8)

template <typename T, int NC>
constexpr bool nc_ok() { return NC == 4 || sizeof(T) == 2; }

template <typename T, int LX, int TY, int S, bool SC, int MODE, int NC>
static cudaError_t launch_tma_inst(const GridDev& g, int ox, const CUtensorMap* maps, void* o0, void* o1,
                                   void* o2, const Scales& sc, const CoefDev& cf, float dt, int* err, int nseg,
                                   int seg0, int seg_count, cudaStream_t s) {
  if constexpr (!nc_ok<T, NC>()) {
    return cudaErrorInvalidConfiguration;
  } else {
    using L = TmaLayout<T, LX, TY, S, NC>;
    auto kern = tma_kernel<T, LX, TY, S, SC, MODE, NC>;
    cudaError_t e = set_smem_attr_once(kern, (int)L::SMEM);
    if (e != cudaSuccess) return e;
    if (seg_count <= 0) seg_count = nseg - seg0;
    dim3 grid((g.nx + L::TX - 1) / L::TX, (g.ny + TY - 1) / TY, seg_count);
    dim3 block(32, L::WARPS);
    kern<<<grid, block, L::SMEM, s>>>(maps[0], maps[1], maps[2], (T*)o0, (T*)o1, (T*)o2, g, ox, nseg, seg0, sc, cf,
                                      dt, err);
    return cudaGetLastError();
  }
}

template <typename T, int MODE>
static cudaError_t launch_tma_mode(const GridDev& g, int ox, const CUtensorMap* maps, void* o0, void* o1, void* o2,
                                   const Scales& sc, bool scaled, const CoefDev& cf, float dt, int* err,
                                   const TmaConfig& c, cudaStream_t s) {
#define PW_DISPATCH(LX_, TY_, S_, NC_)                                                                        \
    if (c.lx == LX_ && c.ty == TY_ && c.stages == S_ && c.nc == NC_)                                          \
        return scaled ? launch_tma_inst<T, LX_, TY_, S_, true, MODE, NC_>(g, ox, maps, o0, o1, o2, sc, cf, dt, err, \
                                                                          c.nseg, c.seg0, c.seg_count, s)     \
                      : launch_tma_inst<T, LX_, TY_, S_, false, MODE, NC_>(g, ox, maps, o0, o1, o2, sc, cf, dt,   \
                                                                           err, c.nseg, c.seg0, c.seg_count, s);
    PW_TMA_CONFIGS(PW_DISPATCH)
#undef PW_DISPATCH
    return cudaErrorInvalidConfiguration;
}

}  // namespace pw
