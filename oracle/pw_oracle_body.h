/*
 * Body of the CPU oracle, included twice by pw_oracle.c: once with REAL=double
 * (the reference) and once with REAL=float (the single-precision CPU result,
 * evaluated in the order written here).  TEST INFRASTRUCTURE ONLY: nothing in
 * the product path includes or links this file.
 *
 * Layout (the oracle's own, unrelated to the device library's): a field is a
 * dense C array of shape (nz+2, ny+2, nx+2) with one halo cell on every side;
 * element (k, j, i) sits at ((k*(ny+2) + j)*(nx+2) + i).  i is x, j is y,
 * k is z; interior i = 1..nx, j = 1..ny, k = 1..nz.  k = 1 is the surface and
 * k = nz the rigid lid.
 */

#define IDX(k, j, i) ((((size_t)(k)) * (size_t)(ny + 2) + (size_t)(j)) * (size_t)(nx + 2) + (size_t)(i))

/*
 * Piacsek-Williams advective source terms (Sec. 2.2: a depth-one stencil over
 * U, V and W producing one source term per field).  Per field and cell the
 * arithmetic has the shape Sec. 4 describes: six pair sums, six products of a
 * neighbour with a pair sum, the differences scaled by the grid coefficients,
 * and a final sum over the three directions.
 *
 * The index pattern is the PW scheme on an Arakawa-C grid: u(k,j,i) on the +x
 * face of cell (j,i), v on the +y face, w on the top face of layer k.  It is
 * the centred skew-symmetric form -1/2 [u.grad(q) + div(u q)] of the
 * momentum advection term for q = u, v, w.
 *
 * su, sv at k = 2..nz (no flux through the lid: the upper vertical term is
 * dropped at k = nz); sw at k = 2..nz-1.  su, sv at k = 1 and sw at k = 1, nz
 * are set to zero.  Halo cells of su, sv, sw are not written.  The z-halo
 * planes k = 0 and k = nz+1 of u, v, w are never read.
 */
static void FN(tendencies)(int nx, int ny, int nz,
                           const REAL *u, const REAL *v, const REAL *w,
                           REAL tcx, REAL tcy,
                           const REAL *tzc1, const REAL *tzc2,
                           const REAL *tzd1, const REAL *tzd2,
                           REAL *su, REAL *sv, REAL *sw)
{
    for (int k = 1; k <= nz; ++k) {
        for (int j = 1; j <= ny; ++j) {
            for (int i = 1; i <= nx; ++i) {
                size_t c = IDX(k, j, i);
                if (k == 1) {
                    su[c] = 0;
                    sv[c] = 0;
                    sw[c] = 0;
                    continue;
                }

                /* ---- su: x-momentum, at the +x face of cell (j,i) ---- */
                {
                    /* pair sums (advecting velocity on the faces of the u-volume) */
                    REAL ax_w = u[IDX(k, j, i)] + u[IDX(k, j, i - 1)];
                    REAL ax_e = u[IDX(k, j, i)] + u[IDX(k, j, i + 1)];
                    REAL ay_s = v[IDX(k, j - 1, i)] + v[IDX(k, j - 1, i + 1)];
                    REAL ay_n = v[IDX(k, j, i)] + v[IDX(k, j, i + 1)];
                    REAL az_b = w[IDX(k - 1, j, i)] + w[IDX(k - 1, j, i + 1)];
                    REAL az_t = w[IDX(k, j, i)] + w[IDX(k, j, i + 1)];
                    /* neighbour products */
                    REAL px_w = u[IDX(k, j, i - 1)] * ax_w;
                    REAL px_e = u[IDX(k, j, i + 1)] * ax_e;
                    REAL py_s = u[IDX(k, j - 1, i)] * ay_s;
                    REAL py_n = u[IDX(k, j + 1, i)] * ay_n;
                    REAL pz_b = u[IDX(k - 1, j, i)] * az_b;
                    REAL pz_t = (k < nz) ? u[IDX(k + 1, j, i)] * az_t : (REAL)0;
                    /* scaled differences and the reduction */
                    REAL tx = tcx * (px_w - px_e);
                    REAL ty = tcy * (py_s - py_n);
                    REAL tz = (k < nz) ? tzc1[k] * pz_b - tzc2[k] * pz_t : tzc1[k] * pz_b;
                    su[c] = tx + ty + tz;
                }

                /* ---- sv: y-momentum, at the +y face of cell (j,i) ---- */
                {
                    REAL ax_w = u[IDX(k, j, i - 1)] + u[IDX(k, j + 1, i - 1)];
                    REAL ax_e = u[IDX(k, j, i)] + u[IDX(k, j + 1, i)];
                    REAL ay_s = v[IDX(k, j, i)] + v[IDX(k, j - 1, i)];
                    REAL ay_n = v[IDX(k, j, i)] + v[IDX(k, j + 1, i)];
                    REAL az_b = w[IDX(k - 1, j, i)] + w[IDX(k - 1, j + 1, i)];
                    REAL az_t = w[IDX(k, j, i)] + w[IDX(k, j + 1, i)];
                    REAL px_w = v[IDX(k, j, i - 1)] * ax_w;
                    REAL px_e = v[IDX(k, j, i + 1)] * ax_e;
                    REAL py_s = v[IDX(k, j - 1, i)] * ay_s;
                    REAL py_n = v[IDX(k, j + 1, i)] * ay_n;
                    REAL pz_b = v[IDX(k - 1, j, i)] * az_b;
                    REAL pz_t = (k < nz) ? v[IDX(k + 1, j, i)] * az_t : (REAL)0;
                    REAL tx = tcx * (px_w - px_e);
                    REAL ty = tcy * (py_s - py_n);
                    REAL tz = (k < nz) ? tzc1[k] * pz_b - tzc2[k] * pz_t : tzc1[k] * pz_b;
                    sv[c] = tx + ty + tz;
                }

                /* ---- sw: z-momentum, at the top face of layer k ---- */
                if (k < nz) {
                    REAL ax_w = u[IDX(k, j, i - 1)] + u[IDX(k + 1, j, i - 1)];
                    REAL ax_e = u[IDX(k, j, i)] + u[IDX(k + 1, j, i)];
                    REAL ay_s = v[IDX(k, j - 1, i)] + v[IDX(k + 1, j - 1, i)];
                    REAL ay_n = v[IDX(k, j, i)] + v[IDX(k + 1, j, i)];
                    REAL az_b = w[IDX(k, j, i)] + w[IDX(k - 1, j, i)];
                    REAL az_t = w[IDX(k, j, i)] + w[IDX(k + 1, j, i)];
                    REAL px_w = w[IDX(k, j, i - 1)] * ax_w;
                    REAL px_e = w[IDX(k, j, i + 1)] * ax_e;
                    REAL py_s = w[IDX(k, j - 1, i)] * ay_s;
                    REAL py_n = w[IDX(k, j + 1, i)] * ay_n;
                    REAL pz_b = w[IDX(k - 1, j, i)] * az_b;
                    REAL pz_t = w[IDX(k + 1, j, i)] * az_t;
                    REAL tx = tcx * (px_w - px_e);
                    REAL ty = tcy * (py_s - py_n);
                    REAL tz = tzd1[k] * pz_b - tzd2[k] * pz_t;
                    sw[c] = tx + ty + tz;
                } else {
                    sw[c] = 0;
                }
            }
        }
    }
}

/*
 * Periodic lateral boundary (the halo swap a doubly periodic domain needs
 * before each evaluation of the scheme): x first, then y over the full padded
 * row, so the four corner columns take the diagonally opposite interior
 * values.  Levels k = 1..nz; the z-halo planes are left untouched.
 */
static void FN(fill_halo_periodic)(int nx, int ny, int nz, REAL *f)
{
    for (int k = 1; k <= nz; ++k) {
        for (int j = 1; j <= ny; ++j) {
            f[IDX(k, j, 0)] = f[IDX(k, j, nx)];
            f[IDX(k, j, nx + 1)] = f[IDX(k, j, 1)];
        }
        for (int i = 0; i <= nx + 1; ++i) {
            f[IDX(k, 0, i)] = f[IDX(k, ny, i)];
            f[IDX(k, ny + 1, i)] = f[IDX(k, 1, i)];
        }
    }
}
