// PW advective source terms (Sec. 2.2; per-cell arithmetic shape Sec. 4):
// launchers of the generic and TMA k-march kernels in their tendency mode,
// and the launch-shape queries shared with the other modes.
#include "pw_stencil.cuh"

namespace pw {

cudaError_t launch_tend_generic(pw_dtype_t dt, const GridDev& g, const void* u, const void* v, const void* w,
                                void* su, void* sv, void* sw, const Scales& sc, bool scaled,
                                const CoefDev& cf, int num_sms, cudaStream_t s) {
    switch (dt) {
        case PW_F32:
            return launch_generic_mode<float, MODE_TEND>(g, u, v, w, su, sv, sw, sc, scaled, cf, 0.f, num_sms, s);
        case PW_BF16:
            return launch_generic_mode<__nv_bfloat16, MODE_TEND>(g, u, v, w, su, sv, sw, sc, scaled, cf, 0.f,
                                                                 num_sms, s);
        case PW_F16:
            return launch_generic_mode<__half, MODE_TEND>(g, u, v, w, su, sv, sw, sc, scaled, cf, 0.f, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_tend_tma(pw_dtype_t dt, const GridDev& g, int ox, const CUtensorMap* maps, void* su, void* sv,
                            void* sw, const Scales& sc, const CoefDev& cf, int* err,
                            const TmaConfig& c, cudaStream_t s) {
    switch (dt) {
        case PW_F32: return launch_tma_mode<float, MODE_TEND>(g, ox, maps, su, sv, sw, sc, cf, 0.f, err, c, s);
        case PW_BF16:
            return launch_tma_mode<__nv_bfloat16, MODE_TEND>(g, ox, maps, su, sv, sw, sc, cf, 0.f, err, c, s);
        case PW_F16: return launch_tma_mode<__half, MODE_TEND>(g, ox, maps, su, sv, sw, sc, cf, 0.f, err, c, s);
    }
    return cudaErrorInvalidValue;
}

bool tma_config_supported(pw_dtype_t dt, const TmaConfig& c) {
#define PW_SUP(LX_, TY_, S_, NC_, RP_, XP_)                                                       \
    if (c.lx == LX_ && c.ty == TY_ && c.stages == S_ && c.nc == NC_ && c.rp == RP_ && c.xp == XP_) \
        return (NC_ == 4 && RP_ == 1 && XP_ == 0) || dtype_size(dt) == 2;
    PW_TMA_CONFIGS(PW_SUP)
#undef PW_SUP
    return false;
}

template <typename T>
static size_t smem_t(const TmaConfig& c) {
#define PW_SM(LX_, TY_, S_, NC_, RP_, XP_)                                                            \
    if constexpr (nc_ok<T, NC_, RP_, XP_>())                                                           \
        if (c.lx == LX_ && c.ty == TY_ && c.stages == S_ && c.nc == NC_ && c.rp == RP_ && c.xp == XP_) \
            return TmaLayout<T, LX_, TY_, S_, NC_, RP_, XP_>::SMEM;
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
#define PW_OCC(LX_, TY_, S_, NC_, RP_, XP_)                                                           \
    if constexpr (nc_ok<T, NC_, RP_, XP_>())                                                           \
        if (c.lx == LX_ && c.ty == TY_ && c.stages == S_ && c.nc == NC_ && c.rp == RP_ && c.xp == XP_) { \
            auto kern = tma_kernel<T, LX_, TY_, S_, MODE_TEND, NC_, RP_, XP_>;                         \
            using L = TmaLayout<T, LX_, TY_, S_, NC_, RP_, XP_>;                                       \
            if (set_smem_attr_once(kern, (int)L::SMEM) != cudaSuccess) return 0;                       \
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, L::THREADS, L::SMEM) != cudaSuccess) \
                return 0;                                                                              \
            return n;                                                                                  \
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

int tma_box_width(pw_dtype_t dt, int lx, int nc) { return nc * lx + 2 * (16 / (int)dtype_size(dt)); }

}  // namespace pw
