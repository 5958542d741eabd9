// PW advective source terms (Sec. 2.2; per-cell arithmetic shape Sec. 4):
// a generic per-cell kernel for any layout, and the TMA-staged k-march kernel.
#include "pw_device.cuh"
#include "pw_internal.h"

namespace pw {

// ---------------------------------------------------------------------------
// Generic kernel: one thread per output cell, plain loads, any layout and
// alignment.  The correctness fallback and the cross-check of the fast path.
template <typename T, bool SCALED>
__global__ void tend_generic_kernel(const GridDev g, const T* __restrict__ u, const T* __restrict__ v,
                                    const T* __restrict__ w, T* __restrict__ su, T* __restrict__ sv,
                                    T* __restrict__ sw, const Scales sc, const CoefDev cf) {
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
        if (SCALED) {
            ru *= sc.out[0];
            rv *= sc.out[1];
            rw *= sc.out[2];
        }
        su[c] = Store<T>::from_f(ru);
        sv[c] = Store<T>::from_f(rv);
        sw[c] = Store<T>::from_f(rw);
    }
}

template <typename T>
static cudaError_t launch_generic_t(const GridDev& g, const void* u, const void* v, const void* w, void* su,
                                    void* sv, void* sw, const Scales& sc, bool scaled, const CoefDev& cf,
                                    int num_sms, cudaStream_t s) {
    const long long total = (long long)g.nx * g.ny * g.nz;
    const int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    const long long cap = (long long)num_sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (scaled)
        tend_generic_kernel<T, true><<<(unsigned)blocks, threads, 0, s>>>(
            g, (const T*)u, (const T*)v, (const T*)w, (T*)su, (T*)sv, (T*)sw, sc, cf);
    else
        tend_generic_kernel<T, false><<<(unsigned)blocks, threads, 0, s>>>(
            g, (const T*)u, (const T*)v, (const T*)w, (T*)su, (T*)sv, (T*)sw, sc, cf);
    return cudaGetLastError();
}

cudaError_t launch_tend_generic(pw_dtype_t dt, const GridDev& g, const void* u, const void* v, const void* w,
                                void* su, void* sv, void* sw, const Scales& sc, bool scaled,
                                const CoefDev& cf, int num_sms, cudaStream_t s) {
    switch (dt) {
        case PW_F32: return launch_generic_t<float>(g, u, v, w, su, sv, sw, sc, scaled, cf, num_sms, s);
        case PW_BF16: return launch_generic_t<__nv_bfloat16>(g, u, v, w, su, sv, sw, sc, scaled, cf, num_sms, s);
        case PW_F16: return launch_generic_t<__half>(g, u, v, w, su, sv, sw, sc, scaled, cf, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// TMA k-march kernel.
//
// A CTA owns an x-y tile of 128 x TY interior columns and one k segment.  It
// marches up the column one level at a time.  Level planes of u, v, w (the
// tile plus a one-cell halo, widened in x to the 16-byte TMA granule) are
// brought into a ring of `S` shared-memory stages by 3D TMA box copies issued
// by one thread, each stage completing on its own mbarrier; S-1 planes are in
// flight ahead of the level being computed, so each input element is read
// from HBM once and the copy engine, not the warps, keeps bytes in flight.
//
// Thread (lane, ty) computes 4 consecutive cells along x of row ty: smem rows
// are read as 16-byte (FP32) or 8-byte (16-bit) vectors, x-neighbours come
// from the adjacent lanes by warp shuffles (the two tile-edge lanes read
// theirs from the halo columns in smem), y-neighbours from the rows above and
// below, and the values of level k-1 the scheme needs (u, v, w at the cell,
// w one cell east and one row north) are carried in registers from the
// previous step: a rolling window in z.  The level k+1 plane supplies the
// upper terms.  Outputs are written straight from registers as full vectors.
template <typename T, int TY, int S>
struct TmaLayout {
    static constexpr int TX = 128;
    static constexpr int PADX = 16 / (int)sizeof(T);   // elements in one 16-byte granule
    static constexpr int BW = TX + 2 * PADX;           // box width
    static constexpr int ROWS = TY + 2;
    static constexpr int FIELD_RAW = BW * ROWS;
    static constexpr int FIELD_BYTES = ((FIELD_RAW * (int)sizeof(T) + 127) / 128) * 128;
    static constexpr int FIELD = FIELD_BYTES / (int)sizeof(T);
    static constexpr int STAGE = 3 * FIELD;
    static constexpr uint32_t TX_BYTES = 3u * FIELD_RAW * (uint32_t)sizeof(T);
    static constexpr size_t SMEM = (size_t)S * STAGE * sizeof(T) + S * sizeof(uint64_t) + 16;
};

template <typename T, int TY, int S, bool SCALED>
__global__ void __launch_bounds__(32 * TY)
    tend_tma_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_v,
                    const __grid_constant__ CUtensorMap tm_w, T* __restrict__ su, T* __restrict__ sv,
                    T* __restrict__ sw, const GridDev g, const int ox, const int nseg, const Scales sc,
                    const CoefDev cf, int* __restrict__ err) {
    using L = TmaLayout<T, TY, S>;
    constexpr int BW = L::BW;
    constexpr int PADX = L::PADX;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* stages = reinterpret_cast<T*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)S * L::STAGE * sizeof(T));
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + S);

    const int lane = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 32 + lane;
    const int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
    const int nz = g.nz;
    const int kb = 1 + (int)(((long long)bz * nz) / nseg);
    const int ke = (int)(((long long)(bz + 1) * nz) / nseg);
    const int pb = max(kb - 1, 1);
    const int pe = min(ke + 1, nz);
    const int np = pe - pb + 1;
    if (ke < kb) return;   // empty k segment (the host never launches one)

    const int X0 = ox + 1 + L::TX * bx - PADX;
    const int Y0 = TY * by + g.halo - 1;

    auto issue = [&](int p) {   // plane pb+p into stage p % S
        const int s = p % S;
        T* dst = stages + s * L::STAGE;
        mbar_arrive_expect_tx(&bars[s], L::TX_BYTES);
        tma_load_3d(dst, &tm_u, X0, Y0, pb + p, &bars[s]);
        tma_load_3d(dst + L::FIELD, &tm_v, X0, Y0, pb + p, &bars[s]);
        tma_load_3d(dst + 2 * L::FIELD, &tm_w, X0, Y0, pb + p, &bars[s]);
    };

    int issued = 0;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        prefetch_tensormap(&tm_u);
        prefetch_tensormap(&tm_v);
        prefetch_tensormap(&tm_w);
        for (; issued < S && issued < np; ++issued) issue(issued);
    }

    const int r = ty + 1;
    const int c0 = 4 * lane + PADX;
    // tile-edge neighbour column: lane 0 needs x = -1, lane 31 needs x = 128;
    // the other lanes read lane 31's address (a broadcast, no bank conflict)
    const int ce = (lane == 0) ? PADX - 1 : L::TX + PADX;
    const int j = TY * by + 1 + ty;
    const int i0 = 1 + L::TX * bx + 4 * lane;
    const bool valid = (j <= g.ny) && (i0 <= g.nx);
    const long long row_off = g.origin + (long long)j * g.pj + i0;
    const float tcx = cf.tcx, tcy = cf.tcy;
    const int nzp2 = nz + 2;
    const unsigned FULL = 0xffffffffu;

    auto ld = [&](const T* p, float (&o)[4], float s) {
        load4(p, o);
        if (SCALED) {
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] *= s;
        }
    };
    auto ld1 = [&](const T* p, float s) {
        float x = Store<T>::to_f(*p);
        return SCALED ? x * s : x;
    };

    // level k-1 window
    float ud[4] = {0, 0, 0, 0}, vd[4] = {0, 0, 0, 0}, wd[5] = {0, 0, 0, 0, 0}, wdn[4] = {0, 0, 0, 0};
    int waited = 0;   // planes 0..waited-1 are known complete
    bool aborted = false;

    for (int kk = pb; kk <= ke; ++kk) {
        const int lp = kk - pb;
        bool ok = true;
        if (lp == 0) ok = mbar_wait_bounded(&bars[0], 0, kWaitLimitNs);
        const bool have_up = (kk + 1 <= pe);
        if (ok && have_up) ok = mbar_wait_bounded(&bars[(lp + 1) % S], ((lp + 1) / S) & 1, kWaitLimitNs);
        ok = __all_sync(FULL, ok);
        if (!ok) *abort_flag = 1;
        if (ok) {
            waited = lp + (have_up ? 2 : 1);
            const T* P = stages + (lp % S) * L::STAGE;   // level kk
            const T* PU = P, *PV = P + L::FIELD, *PW = P + 2 * L::FIELD;
            float u0[4], us[4], un[4], v0[4], vs[4], vn[4], w0[4], ws[4], wn[4];
            ld(PU + r * BW + c0, u0, sc.in[0]);
            ld(PV + r * BW + c0, v0, sc.in[1]);
            ld(PW + r * BW + c0, w0, sc.in[2]);
            ld(PW + (r + 1) * BW + c0, wn, sc.in[2]);
            const float ew = ld1(PW + r * BW + ce, sc.in[2]);
            float w0m = __shfl_up_sync(FULL, w0[3], 1);
            float w0p = __shfl_down_sync(FULL, w0[0], 1);
            if (lane == 0) w0m = ew;
            if (lane == 31) w0p = ew;

            if (kk >= kb && valid) {
                const long long o = row_off + (long long)kk * g.pk;
                if (kk == 1) {
                    const float z4[4] = {0.f, 0.f, 0.f, 0.f};
                    store4(su + o, z4);
                    store4(sv + o, z4);
                    store4(sw + o, z4);
                }
            }
            if (kk >= kb && kk >= 2) {
                ld(PU + (r - 1) * BW + c0, us, sc.in[0]);
                ld(PU + (r + 1) * BW + c0, un, sc.in[0]);
                ld(PV + (r - 1) * BW + c0, vs, sc.in[1]);
                ld(PV + (r + 1) * BW + c0, vn, sc.in[1]);
                ld(PW + (r - 1) * BW + c0, ws, sc.in[2]);
                const float eu = ld1(PU + r * BW + ce, sc.in[0]);
                const float ev = ld1(PV + r * BW + ce, sc.in[1]);
                const float eun = ld1(PU + (r + 1) * BW + ce, sc.in[0]);
                const float evs = ld1(PV + (r - 1) * BW + ce, sc.in[1]);
                float u0m = __shfl_up_sync(FULL, u0[3], 1);
                float u0p = __shfl_down_sync(FULL, u0[0], 1);
                float unm = __shfl_up_sync(FULL, un[3], 1);
                float v0m = __shfl_up_sync(FULL, v0[3], 1);
                float v0p = __shfl_down_sync(FULL, v0[0], 1);
                float vsp = __shfl_down_sync(FULL, vs[0], 1);
                if (lane == 0) { u0m = eu; unm = eun; v0m = ev; }
                if (lane == 31) { u0p = eu; v0p = ev; vsp = evs; }
                const float U[6] = {u0m, u0[0], u0[1], u0[2], u0[3], u0p};     // x = -1..4
                const float V[6] = {v0m, v0[0], v0[1], v0[2], v0[3], v0p};
                const float W[6] = {w0m, w0[0], w0[1], w0[2], w0[3], w0p};
                const float UN[5] = {unm, un[0], un[1], un[2], un[3]};          // x = -1..3
                const float VS[5] = {vs[0], vs[1], vs[2], vs[3], vsp};          // x = 0..4

                const float tz1 = __ldg(cf.tz + kk);
                const float tz2 = __ldg(cf.tz + nzp2 + kk);
                float ru[4], rv[4], rw[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    ru[c] = tcx * (U[c] * (U[c + 1] + U[c]) - U[c + 2] * (U[c + 1] + U[c + 2])) +
                            tcy * (us[c] * (VS[c] + VS[c + 1]) - un[c] * (V[c + 1] + V[c + 2])) +
                            tz1 * (ud[c] * (wd[c] + wd[c + 1]));
                    rv[c] = tcx * (V[c] * (U[c] + UN[c]) - V[c + 2] * (U[c + 1] + UN[c + 1])) +
                            tcy * (vs[c] * (V[c + 1] + vs[c]) - vn[c] * (V[c + 1] + vn[c])) +
                            tz1 * (vd[c] * (wd[c] + wdn[c]));
                    rw[c] = 0.f;
                }
                if (kk < nz) {   // upper terms from level kk+1
                    const T* Q = stages + ((lp + 1) % S) * L::STAGE;
                    const T* QU = Q, *QV = Q + L::FIELD, *QW = Q + 2 * L::FIELD;
                    float uu[4], vu[4], vus[4], wu[4];
                    ld(QU + r * BW + c0, uu, sc.in[0]);
                    ld(QV + r * BW + c0, vu, sc.in[1]);
                    ld(QV + (r - 1) * BW + c0, vus, sc.in[1]);
                    ld(QW + r * BW + c0, wu, sc.in[2]);
                    const float euu = ld1(QU + r * BW + ce, sc.in[0]);
                    float uum = __shfl_up_sync(FULL, uu[3], 1);
                    if (lane == 0) uum = euu;
                    const float UU[5] = {uum, uu[0], uu[1], uu[2], uu[3]};      // x = -1..3
                    const float td1 = __ldg(cf.tz + 2 * nzp2 + kk);
                    const float td2 = __ldg(cf.tz + 3 * nzp2 + kk);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        ru[c] -= tz2 * (uu[c] * (W[c + 1] + W[c + 2]));
                        rv[c] -= tz2 * (vu[c] * (W[c + 1] + wn[c]));
                        rw[c] = tcx * (W[c] * (U[c] + UU[c]) - W[c + 2] * (U[c + 1] + UU[c + 1])) +
                                tcy * (ws[c] * (vs[c] + vus[c]) - wn[c] * (V[c + 1] + vu[c])) +
                                (td1 * (wd[c] * (W[c + 1] + wd[c])) - td2 * (wu[c] * (W[c + 1] + wu[c])));
                    }
                }
                if (valid) {
                    if (SCALED) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            ru[c] *= sc.out[0];
                            rv[c] *= sc.out[1];
                            rw[c] *= sc.out[2];
                        }
                    }
                    const long long o = row_off + (long long)kk * g.pk;
                    store4(su + o, ru);
                    store4(sv + o, rv);
                    store4(sw + o, rw);
                }
            }
            // roll the window: level kk becomes level k-1 of the next step
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                ud[c] = u0[c];
                vd[c] = v0[c];
                wd[c] = w0[c];
                wdn[c] = wn[c];
            }
            wd[4] = w0p;
        }
        __syncthreads();
        if (*abort_flag) {
            aborted = true;
            break;
        }
        if (tid == 0 && issued < np) {
            fence_proxy_async_smem();
            issue(issued);   // plane lp + S into the stage level kk just released
            ++issued;
        }
    }

    if (aborted && tid == 0) {
        report_error(err, DEV_TIMEOUT_TMA_WAIT);
        // let the copies still in flight land before the CTA's smem is released
        for (int p = waited; p < issued; ++p)
            if (!mbar_wait_bounded(&bars[p % S], (p / S) & 1, kDrainLimitNs)) break;
    }
}

// Instantiated launch shapes: (ty, stages).
#define PW_TMA_CONFIGS(X) X(4, 4) X(8, 3) X(8, 4) X(8, 6) X(16, 3) X(16, 4)

template <typename T, int TY, int S, bool SC>
static cudaError_t launch_tma_inst(const GridDev& g, int ox, const CUtensorMap* maps, void* su, void* sv,
                                   void* sw, const Scales& sc, const CoefDev& cf, int* err, int nseg,
                                   cudaStream_t s) {
    using L = TmaLayout<T, TY, S>;
    auto kern = tend_tma_kernel<T, TY, S, SC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((g.nx + L::TX - 1) / L::TX, (g.ny + TY - 1) / TY, nseg);
    dim3 block(32, TY);
    kern<<<grid, block, L::SMEM, s>>>(maps[0], maps[1], maps[2], (T*)su, (T*)sv, (T*)sw, g, ox, nseg, sc, cf,
                                      err);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_tma_t(const GridDev& g, int ox, const CUtensorMap* maps, void* su, void* sv, void* sw,
                                const Scales& sc, bool scaled, const CoefDev& cf, int* err, const TmaConfig& c,
                                cudaStream_t s) {
#define PW_DISPATCH(TY_, S_)                                                                           \
    if (c.ty == TY_ && c.stages == S_)                                                                 \
        return scaled ? launch_tma_inst<T, TY_, S_, true>(g, ox, maps, su, sv, sw, sc, cf, err, c.nseg, s) \
                      : launch_tma_inst<T, TY_, S_, false>(g, ox, maps, su, sv, sw, sc, cf, err, c.nseg, s);
    PW_TMA_CONFIGS(PW_DISPATCH)
#undef PW_DISPATCH
    return cudaErrorInvalidConfiguration;
}

cudaError_t launch_tend_tma(pw_dtype_t dt, const GridDev& g, int ox, const CUtensorMap* maps, void* su, void* sv,
                            void* sw, const Scales& sc, bool scaled, const CoefDev& cf, int* err,
                            const TmaConfig& c, cudaStream_t s) {
    switch (dt) {
        case PW_F32: return launch_tma_t<float>(g, ox, maps, su, sv, sw, sc, scaled, cf, err, c, s);
        case PW_BF16: return launch_tma_t<__nv_bfloat16>(g, ox, maps, su, sv, sw, sc, scaled, cf, err, c, s);
        case PW_F16: return launch_tma_t<__half>(g, ox, maps, su, sv, sw, sc, scaled, cf, err, c, s);
    }
    return cudaErrorInvalidValue;
}

bool tma_config_supported(pw_dtype_t, const TmaConfig& c) {
#define PW_SUP(TY_, S_) \
    if (c.ty == TY_ && c.stages == S_) return true;
    PW_TMA_CONFIGS(PW_SUP)
#undef PW_SUP
    return false;
}

template <typename T>
static size_t smem_t(const TmaConfig& c) {
#define PW_SM(TY_, S_) \
    if (c.ty == TY_ && c.stages == S_) return TmaLayout<T, TY_, S_>::SMEM;
    PW_TMA_CONFIGS(PW_SM)
#undef PW_SM
    return 0;
}

size_t tma_smem_bytes(pw_dtype_t dt, const TmaConfig& c) {
    switch (dt) {
        case PW_F32: return smem_t<float>(c);
        case PW_BF16: return smem_t<__nv_bfloat16>(c);
        case PW_F16: return smem_t<__half>(c);
    }
    return 0;
}

template <typename T>
static int blocks_per_sm_t(const TmaConfig& c) {
    int n = 0;
#define PW_OCC(TY_, S_)                                                                                \
    if (c.ty == TY_ && c.stages == S_) {                                                               \
        auto kern = tend_tma_kernel<T, TY_, S_, false>;                                                \
        using L = TmaLayout<T, TY_, S_>;                                                               \
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::SMEM) !=   \
            cudaSuccess)                                                                               \
            return 0;                                                                                  \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 32 * TY_, L::SMEM) != cudaSuccess) \
            return 0;                                                                                  \
        return n;                                                                                      \
    }
    PW_TMA_CONFIGS(PW_OCC)
#undef PW_OCC
    return 0;
}

int tma_blocks_per_sm(pw_dtype_t dt, const TmaConfig& c) {
    switch (dt) {
        case PW_F32: return blocks_per_sm_t<float>(c);
        case PW_BF16: return blocks_per_sm_t<__nv_bfloat16>(c);
        case PW_F16: return blocks_per_sm_t<__half>(c);
    }
    return 0;
}

int tma_box_width(pw_dtype_t dt) { return 128 + 2 * (16 / (int)dtype_size(dt)); }

}  // namespace pw
