/*
 * CPU oracle for the Piacsek-Williams (PW) advection scheme (Sec. 2.2).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load this library.  It
 * shares no source, header, table or helper with the CUDA library; both sides
 * see only the same seeded inputs.
 *
 * Plain loop nests, written for a reader to check against the scheme by eye:
 * no blocking, no fusion, no reordering.  Built with -O2 -ffp-contract=off so
 * the single-precision variant evaluates exactly the expression order in
 * pw_oracle_body.h (no fused multiply-add).
 *
 * Entry points (all fields in the oracle's dense (nz+2, ny+2, nx+2) layout):
 *   pw_oracle_tendencies_f64 / _f32    source terms su, sv, sw       (Sec. 2.2, Sec. 4)
 *   pw_oracle_fill_halo_periodic_f64/_f32   lateral periodic halo swap
 *   pw_oracle_step_f64                 forward-Euler time steps q += dt*s(q)
 *   pw_oracle_adjoint_tendencies_f64   transpose of the linearised scheme
 *   pw_oracle_fold_halo_periodic_f64   transpose of the periodic halo swap
 *   pw_oracle_step_adjoint_f64         reverse sweep of the Euler rollout
 *   pw_oracle_abs_terms_f64            per-cell magnitude sum of the terms
 *                                      (running-error bounds)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define REAL double
#define FN(name) name##_f64
#include "pw_oracle_body.h"
#undef REAL
#undef FN
#undef IDX

#define REAL float
#define FN(name) name##_f32
#include "pw_oracle_body.h"
#undef REAL
#undef FN
#undef IDX

#define IDX(k, j, i) ((((size_t)(k)) * (size_t)(ny + 2) + (size_t)(j)) * (size_t)(nx + 2) + (size_t)(i))

void pw_oracle_tendencies_f64(int nx, int ny, int nz,
                              const double *u, const double *v, const double *w,
                              double tcx, double tcy,
                              const double *tzc1, const double *tzc2,
                              const double *tzd1, const double *tzd2,
                              double *su, double *sv, double *sw)
{
    tendencies_f64(nx, ny, nz, u, v, w, tcx, tcy, tzc1, tzc2, tzd1, tzd2, su, sv, sw);
}

void pw_oracle_tendencies_f32(int nx, int ny, int nz,
                              const float *u, const float *v, const float *w,
                              float tcx, float tcy,
                              const float *tzc1, const float *tzc2,
                              const float *tzd1, const float *tzd2,
                              float *su, float *sv, float *sw)
{
    tendencies_f32(nx, ny, nz, u, v, w, tcx, tcy, tzc1, tzc2, tzd1, tzd2, su, sv, sw);
}

void pw_oracle_fill_halo_periodic_f64(int nx, int ny, int nz, double *f)
{
    fill_halo_periodic_f64(nx, ny, nz, f);
}

void pw_oracle_fill_halo_periodic_f32(int nx, int ny, int nz, float *f)
{
    fill_halo_periodic_f32(nx, ny, nz, f);
}

/*
 * Forward-Euler time stepping of the advection-only system, q <- q + dt*s(q)
 * for q = (u, v, w), with doubly periodic lateral boundaries and the rigid
 * surface and lid (the source terms are zero there, so those levels keep
 * their values).  The halos of u, v, w are refilled from the interior before
 * every evaluation and once more at the end.  Returns 0, or -1 when scratch
 * memory cannot be allocated.
 */
int pw_oracle_step_f64(int nx, int ny, int nz, double *u, double *v, double *w,
                       double tcx, double tcy,
                       const double *tzc1, const double *tzc2,
                       const double *tzd1, const double *tzd2,
                       double dt, int nsteps)
{
    size_t n = (size_t)(nx + 2) * (size_t)(ny + 2) * (size_t)(nz + 2);
    double *su = (double *)calloc(n, sizeof(double));
    double *sv = (double *)calloc(n, sizeof(double));
    double *sw = (double *)calloc(n, sizeof(double));
    if (!su || !sv || !sw) {
        free(su); free(sv); free(sw);
        return -1;
    }
    for (int s = 0; s < nsteps; ++s) {
        fill_halo_periodic_f64(nx, ny, nz, u);
        fill_halo_periodic_f64(nx, ny, nz, v);
        fill_halo_periodic_f64(nx, ny, nz, w);
        tendencies_f64(nx, ny, nz, u, v, w, tcx, tcy, tzc1, tzc2, tzd1, tzd2, su, sv, sw);
        for (int k = 1; k <= nz; ++k)
            for (int j = 1; j <= ny; ++j)
                for (int i = 1; i <= nx; ++i) {
                    size_t c = IDX(k, j, i);
                    u[c] = u[c] + dt * su[c];
                    v[c] = v[c] + dt * sv[c];
                    w[c] = w[c] + dt * sw[c];
                }
    }
    fill_halo_periodic_f64(nx, ny, nz, u);
    fill_halo_periodic_f64(nx, ny, nz, v);
    fill_halo_periodic_f64(nx, ny, nz, w);
    free(su); free(sv); free(sw);
    return 0;
}

/*
 * Adjoint (transpose) of the scheme linearised about (u, v, w): given upstream
 * sensitivities lsu, lsv, lsw of a scalar with respect to su, sv, sw, adds
 * J(u,v,w)^T [lsu; lsv; lsw] into gu, gv, gw (full padded arrays, halo cells
 * included: the halo values are independent inputs of the scheme).
 *
 * Scatter form, one line per term of the forward scheme.  Every term has the
 * shape  c * a * (b + d)  and its transpose with upstream l adds
 * c*l*(b + d) to the slot of a, and c*l*a to the slots of b and d.  The
 * outputs the scheme fixes to zero (su, sv at k = 1, sw at k = 1 and nz) and
 * the vertical term dropped at the lid carry no sensitivity.
 */
#define TERM(c, l, ga, a, gb, b, gd, d)        \
    do {                                         \
        double cl_ = (c) * (l);                  \
        (ga) += cl_ * ((b) + (d));               \
        (gb) += cl_ * (a);                       \
        (gd) += cl_ * (a);                       \
    } while (0)

void pw_oracle_adjoint_tendencies_f64(int nx, int ny, int nz,
                                      const double *u, const double *v, const double *w,
                                      double tcx, double tcy,
                                      const double *tzc1, const double *tzc2,
                                      const double *tzd1, const double *tzd2,
                                      const double *lsu, const double *lsv, const double *lsw,
                                      double *gu, double *gv, double *gw)
{
    for (int k = 2; k <= nz; ++k) {
        for (int j = 1; j <= ny; ++j) {
            for (int i = 1; i <= nx; ++i) {
                size_t c = IDX(k, j, i);
                double l;

                /* su = tcx*[u(i-1)(u+u(i-1)) - u(i+1)(u+u(i+1))]
                      + tcy*[u(j-1)(v(j-1)+v(j-1,i+1)) - u(j+1)(v+v(i+1))]
                      + tzc1*u(k-1)(w(k-1)+w(k-1,i+1)) - tzc2*u(k+1)(w+w(i+1)) */
                l = lsu[c];
                TERM(tcx, l, gu[IDX(k, j, i - 1)], u[IDX(k, j, i - 1)],
                     gu[IDX(k, j, i)], u[IDX(k, j, i)], gu[IDX(k, j, i - 1)], u[IDX(k, j, i - 1)]);
                TERM(-tcx, l, gu[IDX(k, j, i + 1)], u[IDX(k, j, i + 1)],
                     gu[IDX(k, j, i)], u[IDX(k, j, i)], gu[IDX(k, j, i + 1)], u[IDX(k, j, i + 1)]);
                TERM(tcy, l, gu[IDX(k, j - 1, i)], u[IDX(k, j - 1, i)],
                     gv[IDX(k, j - 1, i)], v[IDX(k, j - 1, i)], gv[IDX(k, j - 1, i + 1)], v[IDX(k, j - 1, i + 1)]);
                TERM(-tcy, l, gu[IDX(k, j + 1, i)], u[IDX(k, j + 1, i)],
                     gv[IDX(k, j, i)], v[IDX(k, j, i)], gv[IDX(k, j, i + 1)], v[IDX(k, j, i + 1)]);
                TERM(tzc1[k], l, gu[IDX(k - 1, j, i)], u[IDX(k - 1, j, i)],
                     gw[IDX(k - 1, j, i)], w[IDX(k - 1, j, i)], gw[IDX(k - 1, j, i + 1)], w[IDX(k - 1, j, i + 1)]);
                if (k < nz)
                    TERM(-tzc2[k], l, gu[IDX(k + 1, j, i)], u[IDX(k + 1, j, i)],
                         gw[IDX(k, j, i)], w[IDX(k, j, i)], gw[IDX(k, j, i + 1)], w[IDX(k, j, i + 1)]);

                /* sv = tcx*[v(i-1)(u(i-1)+u(j+1,i-1)) - v(i+1)(u+u(j+1))]
                      + tcy*[v(j-1)(v+v(j-1)) - v(j+1)(v+v(j+1))]
                      + tzc1*v(k-1)(w(k-1)+w(k-1,j+1)) - tzc2*v(k+1)(w+w(j+1)) */
                l = lsv[c];
                TERM(tcx, l, gv[IDX(k, j, i - 1)], v[IDX(k, j, i - 1)],
                     gu[IDX(k, j, i - 1)], u[IDX(k, j, i - 1)], gu[IDX(k, j + 1, i - 1)], u[IDX(k, j + 1, i - 1)]);
                TERM(-tcx, l, gv[IDX(k, j, i + 1)], v[IDX(k, j, i + 1)],
                     gu[IDX(k, j, i)], u[IDX(k, j, i)], gu[IDX(k, j + 1, i)], u[IDX(k, j + 1, i)]);
                TERM(tcy, l, gv[IDX(k, j - 1, i)], v[IDX(k, j - 1, i)],
                     gv[IDX(k, j, i)], v[IDX(k, j, i)], gv[IDX(k, j - 1, i)], v[IDX(k, j - 1, i)]);
                TERM(-tcy, l, gv[IDX(k, j + 1, i)], v[IDX(k, j + 1, i)],
                     gv[IDX(k, j, i)], v[IDX(k, j, i)], gv[IDX(k, j + 1, i)], v[IDX(k, j + 1, i)]);
                TERM(tzc1[k], l, gv[IDX(k - 1, j, i)], v[IDX(k - 1, j, i)],
                     gw[IDX(k - 1, j, i)], w[IDX(k - 1, j, i)], gw[IDX(k - 1, j + 1, i)], w[IDX(k - 1, j + 1, i)]);
                if (k < nz)
                    TERM(-tzc2[k], l, gv[IDX(k + 1, j, i)], v[IDX(k + 1, j, i)],
                         gw[IDX(k, j, i)], w[IDX(k, j, i)], gw[IDX(k, j + 1, i)], w[IDX(k, j + 1, i)]);

                /* sw (k < nz) = tcx*[w(i-1)(u(i-1)+u(k+1,i-1)) - w(i+1)(u+u(k+1))]
                      + tcy*[w(j-1)(v(j-1)+v(k+1,j-1)) - w(j+1)(v+v(k+1))]
                      + tzd1*w(k-1)(w+w(k-1)) - tzd2*w(k+1)(w+w(k+1)) */
                if (k < nz) {
                    l = lsw[c];
                    TERM(tcx, l, gw[IDX(k, j, i - 1)], w[IDX(k, j, i - 1)],
                         gu[IDX(k, j, i - 1)], u[IDX(k, j, i - 1)], gu[IDX(k + 1, j, i - 1)], u[IDX(k + 1, j, i - 1)]);
                    TERM(-tcx, l, gw[IDX(k, j, i + 1)], w[IDX(k, j, i + 1)],
                         gu[IDX(k, j, i)], u[IDX(k, j, i)], gu[IDX(k + 1, j, i)], u[IDX(k + 1, j, i)]);
                    TERM(tcy, l, gw[IDX(k, j - 1, i)], w[IDX(k, j - 1, i)],
                         gv[IDX(k, j - 1, i)], v[IDX(k, j - 1, i)], gv[IDX(k + 1, j - 1, i)], v[IDX(k + 1, j - 1, i)]);
                    TERM(-tcy, l, gw[IDX(k, j + 1, i)], w[IDX(k, j + 1, i)],
                         gv[IDX(k, j, i)], v[IDX(k, j, i)], gv[IDX(k + 1, j, i)], v[IDX(k + 1, j, i)]);
                    TERM(tzd1[k], l, gw[IDX(k - 1, j, i)], w[IDX(k - 1, j, i)],
                         gw[IDX(k, j, i)], w[IDX(k, j, i)], gw[IDX(k - 1, j, i)], w[IDX(k - 1, j, i)]);
                    TERM(-tzd2[k], l, gw[IDX(k + 1, j, i)], w[IDX(k + 1, j, i)],
                         gw[IDX(k, j, i)], w[IDX(k, j, i)], gw[IDX(k + 1, j, i)], w[IDX(k + 1, j, i)]);
                }
            }
        }
    }
}

/*
 * Magnitude sum of the scheme's terms, for error bounds: for every output
 * cell, the sum over its terms  c * a * (b + d)  of  |c| * |a| * (|b| + |d|)
 * (zero where the scheme writes zero).  A perturbation of every input by a
 * relative amount <= e changes each output by at most about 2 e times this
 * sum (first order), and rounding the arithmetic perturbs it by a small
 * multiple of the unit roundoff times this sum: the running-error bound the
 * reduced-precision checks use.  Same term list and levels as the scheme.
 */
#define ABS3(c, a, b, d) (fabs(c) * fabs(a) * (fabs(b) + fabs(d)))

void pw_oracle_abs_terms_f64(int nx, int ny, int nz,
                             const double *u, const double *v, const double *w,
                             double tcx, double tcy,
                             const double *tzc1, const double *tzc2,
                             const double *tzd1, const double *tzd2,
                             double *au, double *av, double *aw)
{
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                size_t c = IDX(k, j, i);
                au[c] = 0; av[c] = 0; aw[c] = 0;
                if (k == 1) continue;
                au[c] = ABS3(tcx, u[IDX(k, j, i - 1)], u[IDX(k, j, i)], u[IDX(k, j, i - 1)])
                      + ABS3(tcx, u[IDX(k, j, i + 1)], u[IDX(k, j, i)], u[IDX(k, j, i + 1)])
                      + ABS3(tcy, u[IDX(k, j - 1, i)], v[IDX(k, j - 1, i)], v[IDX(k, j - 1, i + 1)])
                      + ABS3(tcy, u[IDX(k, j + 1, i)], v[IDX(k, j, i)], v[IDX(k, j, i + 1)])
                      + ABS3(tzc1[k], u[IDX(k - 1, j, i)], w[IDX(k - 1, j, i)], w[IDX(k - 1, j, i + 1)]);
                av[c] = ABS3(tcx, v[IDX(k, j, i - 1)], u[IDX(k, j, i - 1)], u[IDX(k, j + 1, i - 1)])
                      + ABS3(tcx, v[IDX(k, j, i + 1)], u[IDX(k, j, i)], u[IDX(k, j + 1, i)])
                      + ABS3(tcy, v[IDX(k, j - 1, i)], v[IDX(k, j, i)], v[IDX(k, j - 1, i)])
                      + ABS3(tcy, v[IDX(k, j + 1, i)], v[IDX(k, j, i)], v[IDX(k, j + 1, i)])
                      + ABS3(tzc1[k], v[IDX(k - 1, j, i)], w[IDX(k - 1, j, i)], w[IDX(k - 1, j + 1, i)]);
                if (k < nz) {
                    au[c] += ABS3(tzc2[k], u[IDX(k + 1, j, i)], w[IDX(k, j, i)], w[IDX(k, j, i + 1)]);
                    av[c] += ABS3(tzc2[k], v[IDX(k + 1, j, i)], w[IDX(k, j, i)], w[IDX(k, j + 1, i)]);
                    aw[c] = ABS3(tcx, w[IDX(k, j, i - 1)], u[IDX(k, j, i - 1)], u[IDX(k + 1, j, i - 1)])
                          + ABS3(tcx, w[IDX(k, j, i + 1)], u[IDX(k, j, i)], u[IDX(k + 1, j, i)])
                          + ABS3(tcy, w[IDX(k, j - 1, i)], v[IDX(k, j - 1, i)], v[IDX(k + 1, j - 1, i)])
                          + ABS3(tcy, w[IDX(k, j + 1, i)], v[IDX(k, j, i)], v[IDX(k + 1, j, i)])
                          + ABS3(tzd1[k], w[IDX(k - 1, j, i)], w[IDX(k, j, i)], w[IDX(k - 1, j, i)])
                          + ABS3(tzd2[k], w[IDX(k + 1, j, i)], w[IDX(k, j, i)], w[IDX(k + 1, j, i)]);
                }
            }
}

/*
 * Transpose of the periodic halo swap: every halo value was a copy of an
 * interior value, so its sensitivity is added to that interior cell and the
 * halo entry is cleared.  Undoes the y pass first, then the x pass (the
 * reverse of the forward order).  Levels k = 1..nz.
 */
void pw_oracle_fold_halo_periodic_f64(int nx, int ny, int nz, double *g)
{
    for (int k = 1; k <= nz; ++k) {
        for (int i = 0; i <= nx + 1; ++i) {
            g[IDX(k, 1, i)] += g[IDX(k, ny + 1, i)];
            g[IDX(k, ny + 1, i)] = 0;
            g[IDX(k, ny, i)] += g[IDX(k, 0, i)];
            g[IDX(k, 0, i)] = 0;
        }
        for (int j = 1; j <= ny; ++j) {
            g[IDX(k, j, 1)] += g[IDX(k, j, nx + 1)];
            g[IDX(k, j, nx + 1)] = 0;
            g[IDX(k, j, nx)] += g[IDX(k, j, 0)];
            g[IDX(k, j, 0)] = 0;
        }
    }
}

/*
 * Reverse sweep of nsteps forward-Euler steps started from (u0, v0, w0)
 * (interior values are the state; halos are ignored and refilled).  On entry
 * gu, gv, gw hold dL/dq at the final state (interior; halo entries ignored);
 * on return they hold dL/dq at the initial state (interior; halo zero).
 *
 * With x_{n+1} = x_n + dt * P s(F x_n)   (F: periodic fill, P: interior
 * restriction), the recursion is  g_n = g_{n+1} + dt * F^T J(F x_n)^T P^T g_{n+1}.
 * Every intermediate state is stored (no checkpointing): this is the plain
 * version the checkpointed device path is compared with.
 * Returns 0, or -1 when memory cannot be allocated.
 */
int pw_oracle_step_adjoint_f64(int nx, int ny, int nz,
                               const double *u0, const double *v0, const double *w0,
                               double tcx, double tcy,
                               const double *tzc1, const double *tzc2,
                               const double *tzd1, const double *tzd2,
                               double dt, int nsteps,
                               double *gu, double *gv, double *gw)
{
    size_t n = (size_t)(nx + 2) * (size_t)(ny + 2) * (size_t)(nz + 2);
    size_t nstates = (size_t)(nsteps > 0 ? nsteps : 1);
    double *states = (double *)malloc(3 * n * nstates * sizeof(double));
    double *lu = (double *)calloc(n, sizeof(double));
    double *lv = (double *)calloc(n, sizeof(double));
    double *lw = (double *)calloc(n, sizeof(double));
    double *hu = (double *)calloc(n, sizeof(double));
    double *hv = (double *)calloc(n, sizeof(double));
    double *hw = (double *)calloc(n, sizeof(double));
    if (!states || !lu || !lv || !lw || !hu || !hv || !hw) {
        free(states); free(lu); free(lv); free(lw); free(hu); free(hv); free(hw);
        return -1;
    }
    /* forward sweep: state n (halo filled) is kept in states[n] */
    memcpy(states + 0 * n, u0, n * sizeof(double));
    memcpy(states + 1 * n, v0, n * sizeof(double));
    memcpy(states + 2 * n, w0, n * sizeof(double));
    for (int s = 0; s < nsteps; ++s) {
        double *q = states + 3 * n * (size_t)s;
        fill_halo_periodic_f64(nx, ny, nz, q);
        fill_halo_periodic_f64(nx, ny, nz, q + n);
        fill_halo_periodic_f64(nx, ny, nz, q + 2 * n);
        if (s + 1 < nsteps) {
            double *qn = states + 3 * n * (size_t)(s + 1);
            memcpy(qn, q, 3 * n * sizeof(double));
            if (pw_oracle_step_f64(nx, ny, nz, qn, qn + n, qn + 2 * n, tcx, tcy,
                                   tzc1, tzc2, tzd1, tzd2, dt, 1) != 0) {
                free(states); free(lu); free(lv); free(lw); free(hu); free(hv); free(hw);
                return -1;
            }
        }
    }
    /* reverse sweep */
    for (int s = nsteps - 1; s >= 0; --s) {
        const double *q = states + 3 * n * (size_t)s;
        memset(lu, 0, n * sizeof(double));
        memset(lv, 0, n * sizeof(double));
        memset(lw, 0, n * sizeof(double));
        memset(hu, 0, n * sizeof(double));
        memset(hv, 0, n * sizeof(double));
        memset(hw, 0, n * sizeof(double));
        for (int k = 1; k <= nz; ++k)          /* P^T g_{n+1} */
            for (int j = 1; j <= ny; ++j)
                for (int i = 1; i <= nx; ++i) {
                    size_t c = IDX(k, j, i);
                    lu[c] = gu[c];
                    lv[c] = gv[c];
                    lw[c] = gw[c];
                }
        pw_oracle_adjoint_tendencies_f64(nx, ny, nz, q, q + n, q + 2 * n, tcx, tcy,
                                         tzc1, tzc2, tzd1, tzd2, lu, lv, lw, hu, hv, hw);
        pw_oracle_fold_halo_periodic_f64(nx, ny, nz, hu);   /* F^T */
        pw_oracle_fold_halo_periodic_f64(nx, ny, nz, hv);
        pw_oracle_fold_halo_periodic_f64(nx, ny, nz, hw);
        for (int k = 1; k <= nz; ++k)
            for (int j = 1; j <= ny; ++j)
                for (int i = 1; i <= nx; ++i) {
                    size_t c = IDX(k, j, i);
                    gu[c] = gu[c] + dt * hu[c];
                    gv[c] = gv[c] + dt * hv[c];
                    gw[c] = gw[c] + dt * hw[c];
                }
    }
    /* halo entries of the result are zero (the state is the interior) */
    for (int k = 0; k <= nz + 1; ++k)
        for (int j = 0; j <= ny + 1; ++j)
            for (int i = 0; i <= nx + 1; ++i)
                if (k == 0 || k == nz + 1 || j == 0 || j == ny + 1 || i == 0 || i == nx + 1) {
                    size_t c = IDX(k, j, i);
                    gu[c] = 0; gv[c] = 0; gw[c] = 0;
                }
    free(states); free(lu); free(lv); free(lw); free(hu); free(hv); free(hw);
    return 0;
}
