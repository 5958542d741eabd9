/*
 * pw.h — C ABI of the GB300 library for the Piacsek-Williams (PW) advection
 * scheme (Sec. 2.2 of "Exploring the Versal AI engines for accelerating
 * stencil-based atmospheric advection simulation").
 *
 * The scheme: given the three velocity fields u, v, w on a 3D grid with one
 * halo cell, compute the advective source terms su, sv, sw; a depth-one
 * stencil over all three dimensions (Sec. 2.2), per cell and field six pair
 * sums, six products, scaled differences and a final sum (Sec. 4).  The
 * scheme's index pattern (Arakawa-C staggering, u on +x faces, v on +y
 * faces, w on the top face of each layer):
 *
 *   su = tcx [u(i-1)(u+u(i-1)) - u(i+1)(u+u(i+1))]
 *      + tcy [u(j-1)(v(j-1)+v(j-1,i+1)) - u(j+1)(v+v(i+1))]
 *      + tzc1[k] u(k-1)(w(k-1)+w(k-1,i+1)) - tzc2[k] u(k+1)(w+w(i+1))
 *   sv = tcx [v(i-1)(u(i-1)+u(j+1,i-1)) - v(i+1)(u+u(j+1))]
 *      + tcy [v(j-1)(v+v(j-1)) - v(j+1)(v+v(j+1))]
 *      + tzc1[k] v(k-1)(w(k-1)+w(k-1,j+1)) - tzc2[k] v(k+1)(w+w(j+1))
 *   sw = tcx [w(i-1)(u(i-1)+u(k+1,i-1)) - w(i+1)(u+u(k+1))]
 *      + tcy [w(j-1)(v(j-1)+v(k+1,j-1)) - w(j+1)(v+v(k+1))]
 *      + tzd1[k] w(k-1)(w+w(k-1)) - tzd2[k] w(k+1)(w+w(k+1))
 *
 * (offsets relative to (k, j, i)); su, sv at k = 2..nz with the upper vertical
 * term dropped at the lid k = nz; sw at k = 2..nz-1; su, sv at k = 1 and sw at
 * k = 1, nz are written as 0.  The halo cells of su, sv, sw are never written;
 * the z-halo planes k = 0 and nz+1 of u, v, w are never read.
 *
 * Conventions for every entry point:
 *   - Return a pw_status_t; on failure pw_last_error() (thread-local) holds a
 *     message.  Argument errors are detected on the host before any launch.
 *   - Field pointers are DEVICE pointers to caller-owned memory (for example
 *     torch tensors) of the handle's GPU, unless an entry point says HOST;
 *     each is checked on the host (once per pointer, remembered by the
 *     handle) and any other address gives PW_ERR_ARG.  The library never
 *     frees them.  Outputs must not alias inputs.
 *   - Calls are asynchronous on `stream` (a cudaStream_t cast to void*; NULL is
 *     the legacy default stream).  A kernel that gives up a bounded wait
 *     records it in the handle; pw_sync() reports it as PW_ERR_DEVICE_TIMEOUT.
 *   - A handle is bound to the device that was current at pw_create(); that
 *     device must be current for every call with the handle.
 */
#ifndef PW_H
#define PW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PW_OK = 0,
    PW_ERR_ARG = 1,             /* invalid argument (null, size, layout) */
    PW_ERR_ALIGN = 2,           /* pointer or pitch alignment not met */
    PW_ERR_CUDA = 3,            /* a CUDA runtime/driver call failed */
    PW_ERR_OOM = 4,             /* device or host allocation failed */
    PW_ERR_DEVICE_TIMEOUT = 5,  /* a kernel gave up a bounded wait */
    PW_ERR_UNSUPPORTED = 6      /* valid request this build does not implement */
} pw_status_t;

/* Storage type of the fields in device memory.  Arithmetic is always FP32. */
typedef enum { PW_F32 = 0, PW_BF16 = 1, PW_F16 = 2 } pw_dtype_t;

/*
 * Grid and field layout, shared by all six fields of a call.
 * Element (k, j, i) of a field sits at
 *     ptr[origin + k*pitch_k + j*pitch_j + i]          (element units)
 * with interior i = 1..nx, j = 1..ny, k = 1..nz, lateral halo i in
 * [1-halo, 0] and [nx+1, nx+halo] (likewise j), z halo k = 0 and nz+1.
 * Requirements: nx, ny >= 1, nz >= 3, halo >= 1, pitch_j >= nx + 2*halo,
 * pitch_k >= pitch_j*(ny + 2*halo), origin >= (halo-1)*(pitch_j + 1).
 * The scheme reads one halo cell; a deeper halo is room for the periodic
 * images that multi-step updates write.
 */
typedef struct {
    int32_t nx, ny, nz;
    int32_t halo;
    int64_t pitch_j;   /* elements between rows (j) */
    int64_t pitch_k;   /* elements between levels (k) */
    int64_t origin;    /* element offset of (k=0, j=0, i=0) from the pointer */
    pw_dtype_t dtype;
} pw_grid_t;

/* Scheme coefficients (Sec. 2.2), copied at pw_create (the caller keeps
 * ownership of its arrays): tcx, tcy scalars; tzc1, tzc2, tzd1, tzd2 HOST
 * arrays of nz+2 doubles indexed by k (k = 0..nz+1; entries the scheme does
 * not use are ignored).  Converted to FP32 for the device arithmetic. */
typedef struct {
    double tcx, tcy;
    const double *tzc1, *tzc2, *tzd1, *tzd2;
} pw_coeffs_t;

typedef struct pw_handle_s *pw_handle_t;
typedef void *pw_stream_t; /* cudaStream_t */

/*
 * Default layout for (nx, ny, nz, halo, dtype): interior rows start on a
 * 128-byte boundary, pitch_j a multiple of 128 bytes.  Writes the grid to
 * *out and the number of elements each field allocation must hold to
 * *alloc_elems (may be NULL).  This layout qualifies for the TMA k-march
 * kernel when nx is a multiple of 4.
 */
pw_status_t pw_grid_default(int32_t nx, int32_t ny, int32_t nz, int32_t halo, pw_dtype_t dtype,
                            pw_grid_t *out, int64_t *alloc_elems);

/*
 * Create a handle for one grid and coefficient set on the current device:
 * the grid of the three wind fields U, V, W and the coefficients of the PW
 * scheme's source terms (Sec. 2.2: the scheme runs every model timestep on
 * the same grid, so the handle is made once and used for every call).
 * Validates the layout, copies the coefficients (horizontal scalars tcx,
 * tcy and the per-level vertical arrays) to device memory, allocates the
 * handle's status word; the caller may free its coefficient arrays on
 * return.  Fails with PW_ERR_ARG for a bad layout or NULL argument and
 * PW_ERR_CUDA/PW_ERR_OOM for a failed device call.  *out is NULL on failure.
 */
pw_status_t pw_create(const pw_grid_t *grid, const pw_coeffs_t *coeffs, pw_handle_t *out);

/* Release the handle and everything it allocated (device memory, streams,
 * events); the caller's field buffers are not touched.  Resource handling
 * of this library: the paper has no counterpart.  Waits for nothing: work
 * still queued on the handle must be finished first (pw_sync).  NULL is
 * accepted. */
pw_status_t pw_destroy(pw_handle_t h);

/* Kernel selection for pw_tendencies, pw_step, pw_step_to and the periodic
 * pw_adjoint: 0 = automatic (TMA k-march kernel when the layout and pointers
 * qualify, else the generic kernel), 1 = generic kernel, 2 = TMA kernel
 * (pw_tendencies and the step calls return PW_ERR_UNSUPPORTED/PW_ERR_ALIGN
 * when the layout or pointers do not qualify; pw_adjoint then runs the
 * generic kernel). */
pw_status_t pw_set_kernel(pw_handle_t h, int32_t kind);

/*
 * Launch shape of the TMA k-march kernel: lanes_x = lanes per row, cells =
 * consecutive cells per thread along x (tile width lanes_x * cells columns),
 * ty = rows per CTA, stages = planes buffered per CTA, nseg = CTAs along z
 * (0 = chosen from the grid and SM count), rows_per_thread = how a thread
 * holds its cells: 1 = one row, scalar FP32 arithmetic; 2 = the same cells in
 * two rows, each cell paired with the cell one row further on in packed
 * FP32x2 arithmetic; 3 = one row, its cells packed as FP32x2 pairs along x
 * (cell q with cell q + cells/2); every form gives the same results bit for
 * bit.  A shape given here is used for every call, its zero fields at
 * (lanes_x, ty, stages, cells, rows_per_thread) = (32, 4, 4, 4, 1); all zero
 * restores the automatic choice, which depends on the call: (32, 4, 4, 4, 1)
 * for FP32; (16, 8, 4, 8, 3) for 16-bit storage (fused steps: when nx is a
 * multiple of 8, else (32, 4, 4, 4, 3)); (16, 4, 4, 4, 1) when nx <= 64; nseg
 * the count that best fills the last wave of CTAs per plane marched
 * (segments of >= 2 levels; more segments only for a >= 3 % gain).
 * Instantiated (lanes_x, ty, stages, cells, rows_per_thread): (32,4,4,4,1)
 * (32,8,3,4,1) (32,8,4,4,1) (32,8,6,4,1) (32,16,3,4,1) (16,4,4,4,1)
 * (16,8,4,4,1), and for 16-bit storage also (16,4,4,8,1) (16,8,4,8,1)
 * (32,8,4,4,2) (32,16,4,4,2) (16,8,4,4,2) (16,4,4,8,3) (16,8,4,8,3)
 * (16,16,4,8,3) (32,4,4,4,3) (32,8,4,4,3) (16,8,4,4,3) (8,8,4,8,3)
 * (8,16,4,8,3); others give
 * PW_ERR_UNSUPPORTED.  With cells = 8 the source terms accept any nx that is
 * a multiple of 4 (a row's last vector may hold 4 cells of the grid); fused
 * steps then need nx to be a multiple of 8 (else PW_ERR_UNSUPPORTED at the
 * step call).
 */
pw_status_t pw_set_tma_config(pw_handle_t h, int32_t lanes_x, int32_t cells, int32_t ty, int32_t stages,
                              int32_t nseg, int32_t rows_per_thread);

/*
 * The launch shape the TMA k-march kernel will use on this handle (the
 * automatic choice, or what pw_set_tma_config fixed) for pw_tendencies
 * (step = 0) or pw_step (step != 0): out = {lanes_x, cells, ty, stages, nseg,
 * rows_per_thread}.
 */
pw_status_t pw_get_tma_config(pw_handle_t h, int32_t step, int32_t out[6]);

/*
 * Temporal blocking of pw_step.  steps_per_pass: 1 = one step per kernel
 * pass; 2 = two steps per pass (needs the TMA path, a lateral halo >= 2 and
 * interior rows starting >= 7 elements into their padded row, else pw_step
 * returns PW_ERR_UNSUPPORTED); 0 = automatic, which is one step per pass:
 * the two-step pass halves the HBM bytes per step but recomputes the
 * intermediate state on a one-cell border of every tile and is bound by
 * instruction issue, so on GB300 it is slower per step.  Launch
 * shape of the two-step kernel (0 = automatic): ty = rows of the intermediate
 * state per CTA (ty - 2 output rows), stages = input planes in flight,
 * ctas_per_sm = the register budget (1: up to 255 registers a thread; 2: 128,
 * part of the state in local memory), nseg = CTAs along z.  Instantiated
 * (ty, stages, ctas_per_sm): (8,3,1) (8,3,2) (8,4,1) (12,3,1) (16,3,1) (16,4,1);
 * others give PW_ERR_UNSUPPORTED.  Automatic shape: (16, 3, 1).
 */
pw_status_t pw_set_step_blocking(pw_handle_t h, int32_t steps_per_pass, int32_t ty, int32_t stages,
                                 int32_t ctas_per_sm, int32_t nseg);

/*
 * Source terms su, sv, sw of the PW scheme (Sec. 2.2; arithmetic shape
 * Sec. 4) from u, v, w, all in the handle's layout and dtype, halo cells of
 * the inputs used as given (refresh them first, e.g. with
 * pw_fill_halo_periodic).  scale: NULL, or 6 floats
 * {in_u, in_v, in_w, out_su, out_sv, out_sw}: the physical value of a stored
 * input is stored*in; the stored output is physical*out (powers of two keep
 * this exact).  Interior cells of su, sv, sw are written, halos untouched.
 */
pw_status_t pw_tendencies(pw_handle_t h, const void *u, const void *v, const void *w,
                          void *su, void *sv, void *sw, const float *scale, pw_stream_t stream);

/*
 * pw_tendencies on HOST buffers (pageable or pinned) in the handle's layout:
 * copies u, v, w to device buffers the handle owns (allocated and zeroed on
 * first use), computes, copies su, sv, sw back, and returns when the results
 * are in host memory.  What travels per field: levels 1..nz of u, v, w with
 * their one-cell lateral halo (i = 0..nx+1, j = 0..ny+1: all the scheme
 * reads), and the interior of levels 1..nz of su, sv, sw; row padding and
 * cells outside those boxes do not travel, and host cells of su, sv, sw
 * outside the interior are left as they are (as pw_tendencies leaves the
 * device halos).  Levels are pipelined in chunks over copy-in, compute and
 * copy-out streams.
 */
pw_status_t pw_tendencies_host(pw_handle_t h, const void *u, const void *v, const void *w,
                               void *su, void *sv, void *sw, const float *scale, pw_stream_t stream);

/*
 * pw_tendencies_host that returns once the work is enqueued: the results are
 * in host memory once `stream` reaches the point after the call (it waits for
 * the call's last copy), for example after pw_sync(h, stream).  Until then
 * the host inputs must stay unchanged and the host outputs untouched.  Calls
 * on one handle may follow each other without waiting, on one stream or on
 * several: they share the handle's device buffers, so each call is ordered
 * after the previous one on the GPU.  On the pipelined path (the TMA layout,
 * nz >= 8) a call's inputs travel while the previous call's outputs come back
 * (with pinned host memory; with pageable memory the copies are synchronous);
 * otherwise a call starts once the previous call has finished.  Same
 * arguments and results as pw_tendencies_host.
 */
pw_status_t pw_tendencies_host_async(pw_handle_t h, const void *u, const void *v, const void *w,
                                     void *su, void *sv, void *sw, const float *scale, pw_stream_t stream);

/*
 * Advance the advection-only system nsteps forward-Euler steps,
 * q <- q + dt * s(q) for q = (u, v, w), with s the PW source terms (the scheme
 * is evaluated every model timestep, Sec. 2.2), doubly periodic lateral
 * boundaries and the rigid surface and lid (s is zero there, so those levels
 * keep their values).  On entry the interior of (u, v, w) is the state and
 * its halos are ignored; on return (u, v, w) hold the state after nsteps
 * steps with periodic halos filled.  tmp_u, tmp_v, tmp_w are caller-owned
 * scratch fields of the same layout (contents overwritten).  Each step is one
 * fused kernel pass that reads the state once and writes the next state once,
 * periodic images of the boundary cells included; the two buffer sets
 * alternate, and an odd number of passes ends with a device copy back into
 * (u, v, w).  With a lateral halo of at least 2 (and the TMA path), a pass
 * can advance two steps (temporal blocking, opt-in via pw_set_step_blocking): the
 * intermediate state stays on chip in FP32, so the bytes per step halve;
 * FP32 results are identical to single-step passes, and 16-bit storage is
 * rounded once per two steps instead of every step.
 * scale: NULL or 3 floats {s_u, s_v, s_w}: physical = stored * s (for 16-bit
 * storage; the state is rounded to the storage type after every pass).
 * All six pointers must be distinct.  nsteps = 0 only refreshes the halos.
 * pw_last_kernel reports 1 (generic), 2 (TMA, one step per pass) or 3 (TMA,
 * two steps per pass, with one single-step pass for an odd remainder).
 */
pw_status_t pw_step(pw_handle_t h, void *u, void *v, void *w, void *tmp_u, void *tmp_v, void *tmp_w,
                    float dt, int32_t nsteps, const float *scale, pw_stream_t stream);

/*
 * One forward-Euler step out of place: (nu, nv, nw) = (u, v, w) + dt *
 * s(u, v, w) on the interior levels 1..nz, plus the periodic images of the
 * result in the lateral halo (doubly periodic domain), with the kernel one
 * step of pw_step uses, so the bits equal those of pw_step(nsteps = 1).
 * The inputs are not modified and their lateral halos must already hold
 * periodic images (as pw_step, pw_step_to and pw_fill_halo_periodic leave
 * them).  scale as in pw_step.  The six pointers must be distinct.
 * pw_last_kernel reports 1 (generic) or 2 (TMA).
 */
pw_status_t pw_step_to(pw_handle_t h, const void *u, const void *v, const void *w, void *nu, void *nv, void *nw,
                       float dt, const float *scale, pw_stream_t stream);

/* Flags of pw_adjoint. */
#define PW_ADJ_ACCUMULATE 1  /* g += alpha * J^T l                        */
#define PW_ADJ_PERIODIC   2  /* doubly periodic domain (see pw_adjoint)    */
#define PW_ADJ_ADD_LAMBDA 4  /* g = l + alpha * J^T l (one reverse Euler step) */

/*
 * Adjoint of the PW scheme (Sec. 2.2) linearised about (u, v, w): given the
 * sensitivities l = (lsu, lsv, lsw) of a scalar with respect to su, sv, sw,
 * computes J(u,v,w)^T l, the sensitivities with respect to u, v, w, in gather
 * form (no atomics), and writes
 *     g = alpha * J^T l               (flags without ACCUMULATE/ADD_LAMBDA)
 *     g = g + alpha * J^T l           (PW_ADJ_ACCUMULATE)
 *     g = l + alpha * J^T l           (PW_ADJ_ADD_LAMBDA: the reverse sweep of
 *                                      one forward-Euler step q + dt*s(q) with
 *                                      alpha = dt, l = g_{n+1}, g = g_n)
 * for g = (gu, gv, gw).  Only the entries of l at the scheme's outputs count
 * (su, sv at levels 2..nz, sw at 2..nz-1, interior columns); the rest of l
 * is ignored.
 * Without PW_ADJ_PERIODIC the halo values of u, v, w are independent
 * inputs: g is written on levels 1..nz of the interior and the one-cell
 * lateral halo.  With PW_ADJ_PERIODIC the domain is doubly periodic: the
 * halos of u, v, w must hold the periodic images (pw_fill_halo_periodic),
 * output cells wrap around, and g is the sensitivity with respect to the
 * interior values (the halo contributions folded onto their images); g is
 * written on the interior only.  Cells of g not listed are not written.
 * In periodic mode, when the layout and pointers qualify for the TMA
 * kernels (and pw_set_kernel did not ask for the generic one), the TMA
 * k-march adjoint runs and the lateral halos of lsu, lsv, lsw are first
 * overwritten with their periodic images (their halo values carry no
 * meaning in this mode).  Otherwise the generic gather kernel runs; it skips
 * a term whose sensitivity is exactly 0.
 * FP32 storage only (PW_ERR_UNSUPPORTED otherwise).  g must not alias any
 * input.  pw_last_kernel reports 1 (generic) or 2 (TMA).
 */
pw_status_t pw_adjoint(pw_handle_t h, const void *u, const void *v, const void *w,
                       const void *lsu, const void *lsv, const void *lsw,
                       void *gu, void *gv, void *gw, float alpha, int32_t flags, pw_stream_t stream);

/*
 * Launch shape of the TMA adjoint on this handle (0 = automatic, field by
 * field): cells = consecutive cells a thread owns along x (a CTA covers
 * 32*cells columns), ty = rows per CTA (one warp each), stages = ring slots
 * of the six planes (levels k-1, k, k+1 resident, the rest in flight), nseg =
 * CTAs along z (1..nz; automatic: the count that best fills the last wave of
 * CTAs, segments of >= 8 levels).  Instantiated (cells, ty, stages): (4,5,4)
 * (4,4,4) (4,6,4) (2,4,4) (2,5,4) (2,6,4) (2,8,4) (2,8,3); others give
 * PW_ERR_UNSUPPORTED, a negative value or nseg > nz PW_ERR_ARG.  Each cell's
 * arithmetic is the same in every shape.  pw_get_adjoint_config: out =
 * {cells, ty, stages, nseg} that the next TMA adjoint call will use.
 */
pw_status_t pw_set_adjoint_config(pw_handle_t h, int32_t cells, int32_t ty, int32_t stages, int32_t nseg);
pw_status_t pw_get_adjoint_config(pw_handle_t h, int32_t out[4]);

/*
 * Periodic lateral boundary: copy interior values into the lateral halo of
 * f (all halo columns and rows, corners included, levels k = 1..nz), as the
 * halo swap of a doubly periodic domain before each evaluation of the scheme
 * (Sec. 2.2 describes the scheme as called every model timestep).
 */
pw_status_t pw_fill_halo_periodic(pw_handle_t h, void *f, pw_stream_t stream);

/*
 * Validation norms in FP64 over the interior cells of levels k0..k1
 * (1 <= k0 <= k1 <= nz): for a field `test` in the handle's dtype (scaled by
 * `scale`: physical = stored*scale) and a DEVICE FP64 reference `ref` in the
 * dense layout (nz+2, ny+2, nx+2) (element (k,j,i) at
 * ((k*(ny+2)+j)*(nx+2)+i)), writes out[0] = max |test - ref|,
 * out[1] = max |ref|, out[2] = sum (test - ref)^2, out[3] = sum ref^2
 * (out: HOST array of 4 doubles).  Synchronises `stream`.
 * Uses a scratch buffer the handle allocates on first use.
 */
pw_status_t pw_error_norms(pw_handle_t h, const void *test, float scale, const double *ref,
                           int32_t k0, int32_t k1, double *out, pw_stream_t stream);

/*
 * Weighted inner product in FP64 over interior cells of levels k0..k1:
 * returns in *out  sum_k wk[k] * sum_{j,i} a(k,j,i) * b(k,j,i)  for two fields
 * in the handle's layout and dtype (scales sa, sb as in pw_error_norms);
 * wk is a HOST array of nz+2 doubles (NULL = all ones).  Used for the
 * discrete energy identity of the scheme.  Synchronises `stream`.
 */
pw_status_t pw_weighted_dot(pw_handle_t h, const void *a, float sa, const void *b, float sb,
                            const double *wk, int32_t k0, int32_t k1, double *out, pw_stream_t stream);

/*
 * pw_weighted_dot without any device allocation (the paper has no
 * counterpart; this is a service for callers).  Same arguments, result and
 * synchronisation as pw_weighted_dot, but the per-block partials, the result
 * and the copied level weights live in one statically allocated device array
 * of 64.8 KB that every device loading the library holds until the process
 * exits, instead of scratch the handle allocates on first use.  For callers
 * that cannot call cudaMalloc once their run has started (a host model that
 * owns the device memory budget through its own allocator, or a time loop
 * that must not meet an allocation failure): create the handle at start-up,
 * then this call allocates nothing, neither cudaMalloc nor cudaFree nor any
 * allocating library routine.
 * Limit: nz + 2 <= 4096 levels; larger grids get PW_ERR_UNSUPPORTED (use
 * pw_weighted_dot).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) for that device; make that first call before
 * any stream capture.  All calls share the one array and it keeps the last
 * call's contents (every call overwrites what it reads, so nothing needs
 * clearing): calls that overlap on the GPU, on different streams or host
 * threads, race on it and must be serialised by the caller.
 */
pw_status_t pw_weighted_dot_noalloc(pw_handle_t h, const void *a, float sa, const void *b, float sb,
                                    const double *wk, int32_t k0, int32_t k1, double *out,
                                    pw_stream_t stream);

/*
 * Batched source terms: n independent grids, each with its own layout and
 * coefficients (one dtype for all), in one persistent launch replayed from a
 * CUDA graph.  The paper scales its design by decomposing the problem into
 * independent compute units that each own part of the grid (Sec. 5); here a
 * unit is a whole grid and every (grid, tile) pair is a work item, taken
 * from an atomic counter by one k-march CTA per SM slot: the deepest grids
 * first, each grid's tiles together in raster order.
 * Every grid's layout must qualify for the k-march kernel (pw_grid_default
 * layouts with nx a multiple of 4 do), else PW_ERR_UNSUPPORTED.
 */
typedef struct pw_batch_s *pw_batch_t;

/* Create a batch: grids[n] and coeffs[n] (HOST arrays, copied).  Allocates
 * the device tables and the work list; the tile shape starts at (lanes, 4, 4,
 * 1) for FP32 and (lanes, 8, 4, 2) for 16-bit storage, lanes = 16 when the
 * cells lie mostly in grids narrower than 256 columns, else 32. */
pw_status_t pw_batch_create(int32_t n, const pw_grid_t *grids, const pw_coeffs_t *coeffs,
                            pw_batch_t *out);

/* Tile shape of the batched kernel: lanes_x (32, 16 or 8), cells (per thread
 * along x: 4, or 8), ty, stages, rows_per_thread (1; 2: a cell and the one a
 * row further on in packed FP32x2 arithmetic; 3: one row whose cells are
 * packed as FP32x2 pairs along x; 2 and 3 for 16-bit storage only; all give
 * the same bits) from the instantiated set (lanes_x, ty, stages, cells,
 * rows_per_thread) (32,4,4,4,1) (32,8,4,4,1) (16,4,4,4,1) (16,8,4,4,1)
 * (16,16,4,4,1) (32,8,4,4,2) (16,8,4,4,2) (32,4,4,4,3) (32,8,4,4,3) (16,4,4,4,3)
 * (16,8,4,4,3) (16,4,4,8,3) (16,8,4,8,3) (8,8,4,8,3) (8,16,4,8,3)
 * (8,16,4,4,1) (32,16,4,4,1), zero fields at (32, 4, 4, 4, 1);
 * others give PW_ERR_UNSUPPORTED (cells = 8 takes grids with nx = 4 mod 8:
 * the row's last vector is computed whole and its grid cells stored).  ctas_per_sm = resident CTAs per SM of the persistent
 * launch (0 = as many as fit).  Rebuilds the work list; the next call
 * captures a new graph.  The autotuner (paper_2301_13016_gb300.autotune)
 * chooses these by measurement. */
pw_status_t pw_batch_set_config(pw_batch_t b, int32_t lanes_x, int32_t cells, int32_t ty, int32_t stages,
                                int32_t ctas_per_sm, int32_t rows_per_thread);

/* Narrow last columns (enable = 1, the default, or 0).  With the tile shapes
 * (lanes_x, ty, stages, cells, rows_per_thread) (16,16,4,4,1) (16,8,4,4,1)
 * (32,8,4,4,1) for FP32 storage and (8,16,4,8,3) (16,8,4,8,3) for 16-bit
 * storage, a grid whose last column of tiles would hold at most half a tile
 * of cells marches that column with tiles half as wide and of the same
 * thread count: (8,32,4,4,1) (8,16,4,4,1) (16,16,4,4,1), resp. (8,16,4,4,3)
 * (8,16,4,8,3).  The recipe of uneven grids (widths 32..384 in steps of 4)
 * then computes 1.10 x its cells instead of 1.17 x with 64 x 16 tiles.  The
 * results are the same bits either way (one per-cell operation sequence).
 * Other shapes ignore the setting.  Rebuilds the work list. */
pw_status_t pw_batch_set_narrow_columns(pw_batch_t b, int32_t enable);

/* The narrow shape in use (lanes_x, cells, ty; all 0 when the current shape
 * has none or narrow columns are off; any output pointer may be NULL). */
pw_status_t pw_batch_narrow_shape(pw_batch_t b, int32_t *lanes_x, int32_t *cells, int32_t *ty);

/* Work items, interior cells and persistent CTAs of the current shape (any
 * output pointer may be NULL). */
pw_status_t pw_batch_info(pw_batch_t b, int64_t *n_items, int64_t *cells, int32_t *ctas);

/*
 * Source terms of every grid of the batch (as pw_tendencies per grid):
 * u, v, w, su, sv, sw are HOST arrays of n DEVICE pointers, 16-byte aligned,
 * in each grid's layout; scale as in pw_tendencies, shared by all grids.
 * The first call, and any call whose pointers differ from the previous
 * call's, synchronises `stream` and uploads the per-grid tables; the first
 * call after pw_batch_create / pw_batch_set_config or a change of scale
 * captures the graph (counter reset + persistent kernel).  Every call then
 * launches the graph on `stream`.
 */
pw_status_t pw_batch_tendencies(pw_batch_t b, const void *const *u, const void *const *v,
                                const void *const *w, void *const *su, void *const *sv,
                                void *const *sw, const float *scale, pw_stream_t stream);

/* pw_sync for a batch: wait for `stream`, report a recorded timeout. */
pw_status_t pw_batch_sync(pw_batch_t b, pw_stream_t stream);

/* Release the batch.  NULL is accepted. */
pw_status_t pw_batch_destroy(pw_batch_t b);

/* Wait for `stream`, then report (and clear) any bounded-wait timeout a
 * kernel of this handle recorded (PW_ERR_DEVICE_TIMEOUT), and any pending
 * CUDA error (PW_ERR_CUDA).  Error reporting of this library: the paper has
 * no counterpart. */
pw_status_t pw_sync(pw_handle_t h, pw_stream_t stream);

/*
 * Self-test of failure detection (no counterpart in the paper): launches a
 * one-warp kernel that waits on a barrier phase nothing completes, gives up
 * after limit_ns nanoseconds (1e6..1e9) and records a timeout in the handle,
 * as a kernel whose copy never lands would.  The next pw_sync() returns
 * PW_ERR_DEVICE_TIMEOUT and clears it; the CUDA context stays usable.
 */
pw_status_t pw_selftest_wait_timeout(pw_handle_t h, int64_t limit_ns, pw_stream_t stream);

/*
 * Host-side failure injection for tests (no counterpart in the paper): the
 * next `count` operations of one kind that the library performs fail as the
 * CUDA call would have, before any call into CUDA:
 *   kind 0: device or pinned host allocations (cudaMalloc, cudaMallocHost)
 *           -> the entry point returns PW_ERR_OOM;
 *   kind 1: TMA descriptor encodings (cuTensorMapEncodeTiled)
 *           -> the entry point returns PW_ERR_CUDA.
 * count = 0 clears the kind.  Process-wide, thread-safe; nothing reaches
 * the GPU, so no kernel ever sees a failed allocation or descriptor.  Entry
 * points that fail this way leave their handle as it was (no partial state
 * is kept), and a later call succeeds.  PW_ERR_ARG for another kind or a
 * negative count.
 */
pw_status_t pw_inject_failures(int32_t kind, int32_t count);

/*
 * Debug bounds build (the library compiled with -DPW_DEBUG_BOUNDS=1, e.g.
 * PW_NVCC_EXTRA="-DPW_DEBUG_BOUNDS=1" python -m paper_2301_13016_gb300.build
 * --force): every global store of the k-march and two-step kernels first
 * checks its cells with the rule below; a store that fails is skipped and
 * recorded, and the next pw_sync / pw_batch_sync returns PW_ERR_CUDA.  No
 * device assert: a caught store never traps.  pw_debug_bounds_build returns
 * 1 in such a build, else 0.
 * pw_debug_layout_check applies the same rule on the host: 1 when the
 * elements offset .. offset+n-1 (offsets from a field pointer, one row) lie
 * on levels 1..nz and inside the interior (interior_only = 1) or the interior
 * and its lateral halo (0), never in row padding or beyond; 0 otherwise; -1
 * for an invalid grid or n < 1.
 */
int32_t pw_debug_bounds_build(void);
int32_t pw_debug_layout_check(const pw_grid_t *g, int64_t offset, int32_t n, int32_t interior_only);

/* Message for the last failure on this thread ("" if none). */
const char *pw_last_error(void);

/* Static name of a status code. */
const char *pw_status_string(pw_status_t s);

/* Which kernel the last pw_tendencies, pw_step or pw_adjoint call on this
 * handle launched: 1 = generic, 2 = TMA k-march, 3 = two-step TMA k-march
 * (pw_step), 0 = none yet. */
int32_t pw_last_kernel(pw_handle_t h);

#ifdef __cplusplus
}
#endif

#endif /* PW_H */
