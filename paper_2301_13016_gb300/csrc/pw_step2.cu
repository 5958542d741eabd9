// Two forward-Euler steps per pass (temporal blocking, T = 2) of the
// advection-only system q <- q + dt*s(q), s the PW source terms (Sec. 2.2):
//     q1 = q0 + dt*s(q0),   q2 = q1 + dt*s(q1),
// with one read of q0 and one write of q2 per pass, so the HBM bytes per
// cell-step are half those of a single-step pass.  The intermediate state q1
// never leaves shared memory and stays in FP32 whatever the storage type (so
// 16-bit storage rounds the state once per two steps instead of every step);
// with FP32 storage the result equals two single-step passes bit for bit
// (both run the same per-level arithmetic, march_level).
//
// Geometry.  s is a depth-1 stencil, so q2 on a tile needs q1 on the tile
// plus one cell all round, and that needs q0 on the tile plus two cells: the
// lateral halo must be at least 2 deep.  A CTA of TY warps (one warp per row,
// 32 lanes x 4 cells) computes q1 on a 128-column x TY-row tile and q2 on its
// inner 120 columns (lanes 1..30) and TY-2 rows (warps 1..TY-2); tiles
// overlap by the discarded border.  The q0 box is the q1 tile plus one cell,
// widened to 16-byte granules (4 columns each side, 136 in all); because an
// output tile starts at interior column 1 + 120*bx (16-byte aligned) and the
// box 7 columns earlier, every TMA x coordinate is a multiple of 16 bytes for
// FP32 and for 16-bit storage as long as interior rows start 16-byte aligned
// and at least 7 columns into their padded row.
//
// The march in z.  Iteration t computes q1 at level t from the staged q0
// planes t-1..t+1 (stage 1, all warps; q1 goes to a ring of three FP32
// planes in shared memory) and then q2 at level t-1 from q1 at t-2..t
// (stage 2, warps 1..TY-2).  Each stage carries its own rolling state in
// registers (MarchRegs), so stage 2 reads only planes t-1 and t of the ring;
// with three ring planes the write of q1(t+1) never meets a read still in
// flight, and one CTA barrier per level suffices.  A k segment [kb, ke] of q2
// needs q1 on [kb-1, ke+1] and q0 planes [kb-2, ke+2] (clipped to 1..nz).
#include "pw_stencil.cuh"

namespace pw {

template <typename T, int TY, int S>
struct Tb2Layout {
    static constexpr int NC = 4;
    static constexpr int TX = 128;        // q1 columns per tile (32 lanes x 4 cells)
    static constexpr int OX = 120;        // q2 columns per tile (lanes 1..30)
    static constexpr int OY = TY - 2;     // q2 rows per tile (warps 1..TY-2)
    static constexpr int PADL = 4;        // box columns left of the q1 tile
    static constexpr int BW = TX + 8;     // box width
    static constexpr int ROWS = TY + 2;
    static constexpr int THREADS = 32 * TY;
    static constexpr int FIELD_RAW = BW * ROWS;
    static constexpr int FIELD_BYTES = ((FIELD_RAW * (int)sizeof(T) + 127) / 128) * 128;
    static constexpr int FIELD = FIELD_BYTES / (int)sizeof(T);
    static constexpr int STAGE = 3 * FIELD;
    static constexpr uint32_t TX_BYTES = 3u * FIELD_RAW * (uint32_t)sizeof(T);
    static constexpr int NQ = 3;          // q1 planes in the ring
    static constexpr int QF = TY * TX;    // floats per field of a q1 plane
    static constexpr int QPLANE = 3 * QF;
    static constexpr size_t STAGE_BYTES = (size_t)S * STAGE * sizeof(T);
    static constexpr size_t SMEM = STAGE_BYTES + (size_t)NQ * QPLANE * sizeof(float) + S * sizeof(uint64_t) + 16;
    static_assert(BW <= 256, "a TMA box is at most 256 elements wide");
    static_assert((BW * (int)sizeof(T)) % 16 == 0, "box rows are whole 16-byte granules");
    static_assert((OX * (int)sizeof(T)) % 16 == 0, "tile origins stay 16-byte aligned");
    static_assert(TY >= 3, "at least one output row");
    static_assert(SMEM <= 227u * 1024u, "shared memory per CTA");
};

// MINB: resident CTAs per SM the register budget is sized for (1: up to 255
// registers a thread for 8 rows; 2: 128, with some state spilled to local
// memory).
template <typename T, int TY, int S, int MINB>
constexpr int tb2_min_blocks() {
    using L = Tb2Layout<T, TY, S>;
    constexpr int by_smem = (int)((227u * 1024u) / L::SMEM);
    constexpr int by_threads = 2048 / L::THREADS;
    constexpr int m = by_smem < by_threads ? by_smem : by_threads;
    return m < 1 ? 1 : (m > MINB ? MINB : m);
}

template <typename T, int TY, int S, int MINB>
__global__ void __launch_bounds__(Tb2Layout<T, TY, S>::THREADS, (tb2_min_blocks<T, TY, S, MINB>()))
    tb2_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_v,
               const __grid_constant__ CUtensorMap tm_w, T* __restrict__ o0, T* __restrict__ o1,
               T* __restrict__ o2, const GridDev g, const int ox, const int nseg, const FoldedCoef kc,
               const float dt, int* __restrict__ err) {
    using L = Tb2Layout<T, TY, S>;
    constexpr int NC = L::NC;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* const stages = reinterpret_cast<T*>(smem_raw);
    float* const q1 = reinterpret_cast<float*>(smem_raw + L::STAGE_BYTES);
    uint64_t* const bars = reinterpret_cast<uint64_t*>(q1 + L::NQ * L::QPLANE);
    volatile int* const abort_flag = reinterpret_cast<volatile int*>(bars + S);

    const int lane = threadIdx.x, row = threadIdx.y;   // one warp per tile row
    const int tid = row * 32 + lane;
    const int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
    const int nz = g.nz;
    const int kb = 1 + (int)(((long long)bz * nz) / nseg);
    const int ke = (int)(((long long)(bz + 1) * nz) / nseg);
    if (ke < kb) return;   // empty k segment (the host never launches one)
    const int kb1 = max(kb - 1, 1), ke1 = min(ke + 1, nz);   // q1 levels
    const int pb = max(kb1 - 1, 1), pe = min(ke1 + 1, nz);   // q0 planes
    const int np = pe - pb + 1;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    const int X0 = ox + 1 + L::OX * bx - NC - L::PADL;
    const int Y0 = L::OY * by + g.halo - 2;
    auto slot = [&](int p) { return p % S; };
    auto parity = [&](int p) { return (uint32_t)((p / S) & 1); };
    auto issue = [&](int p) {   // plane pb+p into slot p % S
        const int s = slot(p);
        T* dst = stages + s * L::STAGE;
        mbar_arrive_expect_tx(&bars[s], L::TX_BYTES);
        tma_load_3d(dst, &tm_u, X0, Y0, pb + p, &bars[s]);
        tma_load_3d(dst + L::FIELD, &tm_v, X0, Y0, pb + p, &bars[s]);
        tma_load_3d(dst + 2 * L::FIELD, &tm_w, X0, Y0, pb + p, &bars[s]);
    };
    int issued = 0;
    if (tid == 0) {
        prefetch_tensormap(&tm_u);
        prefetch_tensormap(&tm_v);
        prefetch_tensormap(&tm_w);
        for (; issued < S && issued < np; ++issued) issue(issued);
    }

    // stage 1: the thread's cells in the staged box
    const int r = row + 1;
    const int c0 = L::PADL + NC * lane;
    const int ce = (lane == 0) ? L::PADL - 1 : L::TX + L::PADL;
    // stage 2: output cells (j, i0..i0+3)
    const bool stage2 = (row >= 1) && (row <= TY - 2);   // warp-uniform
    const int j = L::OY * by + row;
    const int i0 = L::OX * bx + 1 + NC * (lane - 1);
    const bool valid = stage2 && lane >= 1 && lane <= 30 && j <= g.ny && i0 <= g.nx;
    const long long row_off = g.origin + (long long)j * g.pj + i0;
    // both stages run on stored values with the storage scales folded into the
    // coefficients kc (a step stores its state with the scale it read it with,
    // so q1 in shared memory is in stored units too)
    const int nzp2 = nz + 2;
    const unsigned FULL = 0xffffffffu;

    int lp = 0;   // plane index (from pb) of the stage-1 level
    auto rowld1 = [&](int f, int up, int dr, float (&o)[NC]) {
        loadv<NC>(stages + slot(lp + up) * L::STAGE + f * L::FIELD + (r + dr) * L::BW + c0, o);
    };
    auto edgeld1 = [&](int f, int up, int dr) {
        return Store<T>::to_f(stages[slot(lp + up) * L::STAGE + f * L::FIELD + (r + dr) * L::BW + ce]);
    };
    int m2 = 0;   // stage-2 level
    auto rowld2 = [&](int f, int up, int dr, float (&o)[NC]) {
        const float4 x = *reinterpret_cast<const float4*>(q1 + ((m2 + up) % L::NQ) * L::QPLANE + f * L::QF +
                                                          (row + dr) * L::TX + NC * lane);
        o[0] = x.x;
        o[1] = x.y;
        o[2] = x.z;
        o[3] = x.w;
    };
    // lanes 0 and 31 of stage 2 produce no output: their outer neighbours are unused
    auto edgeld2 = [&](int, int, int) { return 0.f; };

    MarchRegs<NC> st1, st2;
    st1.zero();
    st2.zero();
    int waited = 0;   // q0 planes 0..waited-1 are known complete
    bool aborted = false;

    for (int t = pb; t <= ke + 1; ++t) {
        if (t <= ke1) {   // stage 1: q1 at level t
            lp = t - pb;
            bool ok = true;
            if (lp == 0) ok = mbar_wait_bounded(&bars[slot(0)], parity(0), kWaitLimitNs);
            const bool have_up = (t + 1 <= pe);
            if (ok && have_up) ok = mbar_wait_bounded(&bars[slot(lp + 1)], parity(lp + 1), kWaitLimitNs);
            ok = __all_sync(FULL, ok);
            if (!ok) *abort_flag = 1;
            if (ok) {
                waited = lp + (have_up ? 2 : 1);
                auto out1 = [&](const float (&ru)[NC], const float (&rv)[NC], const float (&rw)[NC],
                                const float (&u0)[NC], const float (&v0)[NC], const float (&w0)[NC]) {
                    if (t < kb1) return;
                    float* Q = q1 + (t % L::NQ) * L::QPLANE + row * L::TX + NC * lane;
                    // at t = 1 the source terms are 0
                    *reinterpret_cast<float4*>(Q) = make_float4(fmaf(dt, ru[0], u0[0]), fmaf(dt, ru[1], u0[1]),
                                                                fmaf(dt, ru[2], u0[2]), fmaf(dt, ru[3], u0[3]));
                    *reinterpret_cast<float4*>(Q + L::QF) = make_float4(
                        fmaf(dt, rv[0], v0[0]), fmaf(dt, rv[1], v0[1]), fmaf(dt, rv[2], v0[2]), fmaf(dt, rv[3], v0[3]));
                    *reinterpret_cast<float4*>(Q + 2 * L::QF) = make_float4(
                        fmaf(dt, rw[0], w0[0]), fmaf(dt, rw[1], w0[1]), fmaf(dt, rw[2], w0[2]), fmaf(dt, rw[3], w0[3]));
                };
                march_level<NC, 32>(st1, rowld1, edgeld1, out1, lane, lp == 0, have_up, (t >= kb1) && (t >= 2), kc,
                                    t, nzp2);
            }
        }
        __syncthreads();   // q1(t) visible; the q0 slot of plane t is free
        if (*abort_flag) {
            aborted = true;
            break;
        }
        if (tid == 0 && t <= ke1 && issued < np) {
            fence_proxy_async_smem();
            issue(issued);
            ++issued;
        }
        const int m = t - 1;
        if (stage2 && m >= kb1) {   // stage 2: q2 at level m
            m2 = m;
            auto out2 = [&](const float (&ru)[NC], const float (&rv)[NC], const float (&rw)[NC],
                            const float (&u1)[NC], const float (&v1)[NC], const float (&w1)[NC]) {
                if (!(m >= kb && valid)) return;
                float a[NC], b[NC], d[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    a[c] = fmaf(dt, ru[c], u1[c]);
                    b[c] = fmaf(dt, rv[c], v1[c]);
                    d[c] = fmaf(dt, rw[c], w1[c]);
                }
                const long long o = row_off + (long long)m * g.pk;
                if (dbg_store(g, o, NC, true, err)) {
                    storev<NC>(o0 + o, a);
                    storev<NC>(o1 + o, b);
                    storev<NC>(o2 + o, d);
                }
                StepImages::vec1<T, NC>(o0, o, a, g, j, i0, err);
                StepImages::vec1<T, NC>(o1, o, b, g, j, i0, err);
                StepImages::vec1<T, NC>(o2, o, d, g, j, i0, err);
            };
            march_level<NC, 32>(st2, rowld2, edgeld2, out2, lane, m == kb1, m + 1 <= ke1, (m >= kb) && (m >= 2), kc,
                                m, nzp2);
        }
    }

    if (aborted && tid == 0) {
        report_error(err, DEV_TIMEOUT_TMA_WAIT);
        // let the copies still in flight land before the CTA's smem is released
        for (int p = waited; p < issued; ++p)
            if (!mbar_wait_bounded(&bars[slot(p)], parity(p), kDrainLimitNs)) break;
    }
}

// Instantiated (rows per CTA, stages, register budget in resident CTAs).
#define PW_TB2_CONFIGS(X) X(8, 3, 1) X(8, 3, 2) X(8, 4, 1) X(12, 3, 1) X(16, 3, 1) X(16, 4, 1)

template <typename T, int TY, int S, int MINB>
static cudaError_t launch_tb2_inst(const GridDev& g, int ox, const CUtensorMap* maps, void* o0, void* o1, void* o2,
                                   const Scales& sc, const CoefDev& cf, float dt, int* err, int nseg,
                                   cudaStream_t s) {
    using L = Tb2Layout<T, TY, S>;
    auto kern = tb2_kernel<T, TY, S, MINB>;
    cudaError_t e = set_smem_attr_once(kern, (int)L::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((g.nx + L::OX - 1) / L::OX, (g.ny + L::OY - 1) / L::OY, nseg);
    dim3 block(32, TY);
    kern<<<grid, block, L::SMEM, s>>>(maps[0], maps[1], maps[2], (T*)o0, (T*)o1, (T*)o2, g, ox, nseg,
                                      fold_coef(cf, sc), dt, err);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_tb2_t(const GridDev& g, int ox, const CUtensorMap* maps, void* o0, void* o1, void* o2,
                                const Scales& sc, const CoefDev& cf, float dt, int* err,
                                const Step2Config& c, cudaStream_t s) {
#define PW_DISPATCH(TY_, S_, M_)                                                                             \
    if (c.ty == TY_ && c.stages == S_ && c.minb == M_)                                                       \
        return launch_tb2_inst<T, TY_, S_, M_>(g, ox, maps, o0, o1, o2, sc, cf, dt, err, c.nseg, s);
    PW_TB2_CONFIGS(PW_DISPATCH)
#undef PW_DISPATCH
    return cudaErrorInvalidConfiguration;
}

template <typename T>
static size_t tb2_smem_t(const Step2Config& c) {
#define PW_SMEM(TY_, S_, M_) \
    if (c.ty == TY_ && c.stages == S_ && c.minb == M_) return Tb2Layout<T, TY_, S_>::SMEM;
    PW_TB2_CONFIGS(PW_SMEM)
#undef PW_SMEM
    return 0;
}

template <typename T>
static int tb2_blocks_t(const Step2Config& c) {
#define PW_OCC(TY_, S_, M_)                                                                                    \
    if (c.ty == TY_ && c.stages == S_ && c.minb == M_) {                                                       \
        auto kern = tb2_kernel<T, TY_, S_, M_>;                                                                  \
        if (set_smem_attr_once(kern, (int)Tb2Layout<T, TY_, S_>::SMEM) != cudaSuccess) return 0;               \
        int n = 0;                                                                                             \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 32 * TY_, Tb2Layout<T, TY_, S_>::SMEM) !=  \
            cudaSuccess)                                                                                       \
            return 0;                                                                                          \
        return n;                                                                                              \
    }
    PW_TB2_CONFIGS(PW_OCC)
#undef PW_OCC
    return 0;
}

bool step2_config_supported(const Step2Config& c) { return tb2_smem_t<float>(c) != 0; }

int step2_box_width() { return Tb2Layout<float, 8, 3>::BW; }

int step2_tile_cols() { return Tb2Layout<float, 8, 3>::OX; }

int step2_blocks_per_sm(pw_dtype_t dt, const Step2Config& c) {
    switch (dt) {
        case PW_F32: return tb2_blocks_t<float>(c);
        case PW_BF16: return tb2_blocks_t<__nv_bfloat16>(c);
        case PW_F16: return tb2_blocks_t<__half>(c);
    }
    return 0;
}

cudaError_t launch_step2_tma(pw_dtype_t dt, const GridDev& g, int ox, const CUtensorMap* maps, void* nu, void* nv,
                             void* nw, const Scales& sc, const CoefDev& cf, float tstep, int* err,
                             const Step2Config& c, cudaStream_t s) {
    switch (dt) {
        case PW_F32: return launch_tb2_t<float>(g, ox, maps, nu, nv, nw, sc, cf, tstep, err, c, s);
        case PW_BF16:
            return launch_tb2_t<__nv_bfloat16>(g, ox, maps, nu, nv, nw, sc, cf, tstep, err, c, s);
        case PW_F16: return launch_tb2_t<__half>(g, ox, maps, nu, nv, nw, sc, cf, tstep, err, c, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pw
