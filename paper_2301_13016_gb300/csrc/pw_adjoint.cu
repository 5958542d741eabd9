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
#include "pw_device.cuh"
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
