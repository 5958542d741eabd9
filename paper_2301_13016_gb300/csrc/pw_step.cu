// Forward-Euler update q <- q + dt*s(q) of the advection-only system, fused
// with the PW source terms (Sec. 2.2: the scheme runs every model timestep):
// launchers of the generic and TMA k-march kernels in their step mode.  Each
// pass reads the state once and writes the next state once, including the
// periodic images of its boundary cells, so no separate halo pass is needed.
#include "pw_stencil.cuh"

namespace pw {

cudaError_t launch_step_generic(pw_dtype_t dt, const GridDev& g, const void* u, const void* v, const void* w,
                                void* nu, void* nv, void* nw, const Scales& sc, bool scaled, const CoefDev& cf,
                                float tstep, int num_sms, cudaStream_t s) {
    switch (dt) {
        case PW_F32:
            return launch_generic_mode<float, MODE_STEP>(g, u, v, w, nu, nv, nw, sc, scaled, cf, tstep, num_sms, s);
        case PW_BF16:
            return launch_generic_mode<__nv_bfloat16, MODE_STEP>(g, u, v, w, nu, nv, nw, sc, scaled, cf, tstep,
                                                                 num_sms, s);
        case PW_F16:
            return launch_generic_mode<__half, MODE_STEP>(g, u, v, w, nu, nv, nw, sc, scaled, cf, tstep, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_step_tma(pw_dtype_t dt, const GridDev& g, int ox, const CUtensorMap* maps, void* nu, void* nv,
                            void* nw, const Scales& sc, const CoefDev& cf, float tstep, int* err,
                            const TmaConfig& c, cudaStream_t s) {
    switch (dt) {
        case PW_F32:
            return launch_tma_mode<float, MODE_STEP>(g, ox, maps, nu, nv, nw, sc, cf, tstep, err, c, s);
        case PW_BF16:
            return launch_tma_mode<__nv_bfloat16, MODE_STEP>(g, ox, maps, nu, nv, nw, sc, cf, tstep, err, c,
                                                             s);
        case PW_F16:
            return launch_tma_mode<__half, MODE_STEP>(g, ox, maps, nu, nv, nw, sc, cf, tstep, err, c, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pw
