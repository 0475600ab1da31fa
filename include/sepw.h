/*
 * sepw.h -- C ABI of the separable W-projection gridding library (libsepw.so)
 * for NVIDIA GB300 (sm_103a).
 *
 * The method (B. Merry, "Approximating W projection as a separable kernel",
 * MNRAS 2015): the W-projection gridding convolution function F_w (Sec. 2) is
 * replaced by the separable F~_w(u, v) = F1_w(u) F1_w(v) (Eq. gt, Sec. 5), so
 * that a visibility at (u_i, v_i, w_i) updates grid cell (u, v) by
 * W_i V_i F1_{w_i}(u - u_i) F1_{w_i}(v - v_i).  The 1-D kernel F1 is tabulated
 * per w-plane and per oversampled fractional offset.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Coordinates u, v, w are in wavelengths (Sec. 2), as float64 arrays of
 *    length nvis (structure of arrays).
 *  - Complex data are interleaved float32 pairs (re, im) ("complex64").
 *  - The grid is grid_size x grid_size complex64, row-major [v][u]; the cell
 *    size is du = 1/fov, and u = 0 lies at column grid_size/2.  The image
 *    has the same shape, [m][l], with l_a = (a - N/2) fov / N.
 *  - Visibility i is located at x = u*fov + N/2 (cells), rounded to the
 *    nearest 1/oversample (ties up): cell c, oversample index o.  Its
 *    footprint is the S x S block of cells c - S/2 + 1 .. c + S/2 per axis.
 *    Its w-plane is round-half-up(|w| (P-1)/w_max) and w < 0 uses the complex
 *    conjugate of the |w| kernel.  A visibility whose footprint leaves the
 *    grid, whose plane exceeds P-1, or whose coordinates are not finite is
 *    DROPPED (skipped and counted), never clamped or wrapped.  All of this is
 *    done in IEEE float64 without fused multiply-add, so cell, oversample and
 *    plane indices are reproducible bit for bit on any IEEE machine.
 *  - Every data pointer is caller-owned DEVICE memory unless stated.  The
 *    library never frees caller memory.  The context owns only its workspace
 *    (binning buffers, FFT plan, small tables).
 *  - Calls are asynchronous on `stream` (0 = legacy default stream) unless
 *    stated; errors detected on the host return before anything is enqueued.
 *  - Return value: SEPW_OK (0) or a negative SEPW_E* code.  No call throws.
 *    sepw_last_error() gives a message for the most recent failure on a ctx.
 *  - A ctx is not thread-safe: serialise calls on one ctx.  Calls on one ctx
 *    with different streams must not overlap in time (they share workspace).
 */
#ifndef SEPW_H
#define SEPW_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SEPW_API __attribute__((visibility("default")))
#else
#define SEPW_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define SEPW_VERSION 1

/* status codes */
#define SEPW_OK 0
#define SEPW_EINVAL (-1)   /* bad parameter, size, pointer or alignment */
#define SEPW_ENOMEM (-2)   /* device allocation of workspace failed */
#define SEPW_ECUDA (-3)    /* a CUDA / cuFFT call failed */
#define SEPW_ETIMEOUT (-4) /* a bounded device wait gave up */
#define SEPW_ENOTSUP (-5)  /* form not available for these parameters */
#define SEPW_ENOPLAN (-6)  /* *_planned call without a current plan */
#define SEPW_ETOOLARGE (-7) /* sepw_grid_noalloc: beyond its fixed scratch */
#define SEPW_EBOUNDS (-8)   /* bounds-checked build: a kernel found a work item,
                               plan record or index out of range and skipped it */

/* kernel forms (sepw_params.form) */
#define SEPW_FORM_PLAIN 0  /* plain FP32: one global atomic per cell update */
#define SEPW_FORM_TILED 1  /* binned tiles, register/shared accumulation, FP32 */
#define SEPW_FORM_TC_BF16 2 /* tile contraction on tensor cores (tcgen05): BF16
                               operands, FP32 accumulation; support <= 16.
                               Degridding is the contraction form too:
                               Q = conj(Av) X per window, then the
                               u-direction dot product per visibility. */
#define SEPW_FORM_TC_FP16 3 /* as SEPW_FORM_TC_BF16 with FP16 operands, scaled per
                               work item by a power of two (FP16 range).
                               Degridding errs relative to the model grid's
                               magnitude (11-bit operands), not the
                               prediction's: a grid dominated by content the
                               kernel suppresses (image edges divided by
                               c1 c1) loses accuracy accordingly. */
#define SEPW_FORM_TC_FP16X2 4 /* as SEPW_FORM_TC_FP16 with each operand split into
                                 FP16 hi + lo (all four products of the
                                 splits): FP32-class accuracy.  Degridding
                                 is the contraction form with the v-taps and
                                 the window split (three products) and FP32
                                 u-taps. */
#define SEPW_FORM_TC_BF16X2 5 /* as SEPW_FORM_TC_BF16 with each operand split into
                                 BF16 hi + lo (all four products; no scale:
                                 BF16 has the FP32 exponent range).
                                 Degridding is the contraction form with the
                                 v-taps and the window split (three
                                 products) and FP32 u-taps. */
#define SEPW_FORM_TC_TF32 6   /* as SEPW_FORM_TC_BF16 with TF32 operands (10-bit
                                 mantissa, FP32 range: no scale), rounded from
                                 the caller's FP32 taps and W V times them;
                                 FP16-class accuracy.  Degridding uses the
                                 tiled FP32 form. */

/* image directions (sepw_image) */
#define SEPW_GRID_TO_IMAGE 0
#define SEPW_IMAGE_TO_GRID 1
#define SEPW_IMAGE_TO_GRID_ADJOINT 2  /* exact adjoint of SEPW_IMAGE_TO_GRID */

typedef struct CUstream_st *sepw_stream_t; /* same type as cudaStream_t */

typedef struct sepw_params {
    int32_t grid_size;  /* N: grid and image are N x N; even, 16..65536       */
    int32_t support;    /* S: taps per axis; even, 2..32, S <= N             */
    int32_t oversample; /* OS: kernel samples per cell; 1..256               */
    int32_t n_wplanes;  /* P: planes over |w| in [0, w_max]; 1..32768        */
    double fov;         /* image extent in direction cosine, 0 < fov < 1.4;
                           du = 1/fov (Sec. 2)                                */
    double w_max;       /* |w| of the last plane, wavelengths, > 0           */
    double gamma;       /* tuning parameter of Eq. gt (5/24 minimax, 1/8
                           exact on the axes, Sec. 3)                         */
    double kb_beta;     /* Kaiser-Bessel antialiasing window parameter; the
                           taper is its transform (Sec. 2 kernel C / c)       */
    int32_t tile;       /* tiled forms: tile edge T in cells; even, 8..64,
                           T + S - 1 <= 64, and T + S - 1 <= 32 for the
                           tensor-core forms.  0 = 32 for SEPW_FORM_TILED
                           and the largest even T with T + S - 1 <= 32 for
                           the tensor-core forms (16 at S = 16)               */
    int32_t form;       /* SEPW_FORM_*                                        */
} sepw_params;

typedef struct sepw_ctx sepw_ctx;

/* Library version (SEPW_VERSION).  Host only. */
SEPW_API int sepw_version(void);

/* Message for a status code.  Host only; static storage. */
SEPW_API const char *sepw_strerror(int status);

/* Check parameters without touching the GPU.  Returns SEPW_OK or
 * SEPW_EINVAL / SEPW_ENOTSUP.  Host only. */
SEPW_API int sepw_check_params(const sepw_params *p);

/* Number of complex taps in the 1-D table: P * OS * S.  Host only; 0 if the
 * parameters are invalid. */
SEPW_API size_t sepw_taps_count(const sepw_params *p);

/* Create a context on the current CUDA device.  Allocates the context's
 * small tables (taper, twiddles) on that device; binning workspace is
 * allocated on first use and grows as needed.  *out is set to NULL on error.
 * Sec. 2 (problem statement: image size, cell size, support, oversampling,
 * number of w planes). */
SEPW_API int sepw_create(sepw_ctx **out, const sepw_params *p);

/* Free the context and everything it owns (synchronises its device).
 * NULL is ignored. */
SEPW_API void sepw_destroy(sepw_ctx *ctx);

/* Message for the most recent failure on ctx (host memory owned by ctx). */
SEPW_API const char *sepw_last_error(const sepw_ctx *ctx);

/* 1-D GCF tables, Eq. gt and Sec. 2 (the GCF is the transform of the taper
 * times the screen):
 *   taps[p][o][j] = F1_{w_p}(d),  d = j - S/2 + 1 - o/OS,  w_p = p w_max/(P-1),
 *   F1_w(d) = (1/N) sum_{a=0}^{N-1} c1(nu_a) g1_w(l_a) exp(-2 pi i d nu_a),
 *   g1_w(l) = exp(2 pi i w (-l^2/2 - gamma l^4)),  nu_a = (a - N/2)/N,
 *   l_a = nu_a fov, c1 = Kaiser-Bessel transform normalised to c1(0) = 1.
 * Computed in float64 on the GPU.  sepw_make_taps writes complex64
 * (P*OS*S*2 floats, layout [p][o][j][re,im]); sepw_make_taps_f64 writes the
 * float64 values (P*OS*S*2 doubles).  Off the hot path. */
SEPW_API int sepw_make_taps(sepw_ctx *ctx, float *taps, sepw_stream_t stream);
SEPW_API int sepw_make_taps_f64(sepw_ctx *ctx, double *taps, sepw_stream_t stream);

/* Locate each visibility (the convention above): writes cell indices cu, cv
 * (int32), oversample indices ou, ov (int32), plane (int32), conj and keep
 * flags (uint8, 1 = true) for i < nvis.  Dropped visibilities have keep = 0
 * and zeros elsewhere.  Any output pointer may be NULL.  Sec. 2 (coordinates)
 * and the oversampled kernel lookup of Sec. 2. */
SEPW_API int sepw_locate(sepw_ctx *ctx, int64_t nvis, const double *u, const double *v,
                const double *w, int32_t *cu, int32_t *cv, int32_t *ou,
                int32_t *ov, int32_t *plane, uint8_t *conj, uint8_t *keep,
                sepw_stream_t stream);

/* Locate and bin nvis visibilities into the context's plan (tiled forms:
 * counting sort by tile and by 4 x 4 sub-block of the footprint origin
 * inside the tile, cut into work items, each sorted by origin).  The
 * plan is reused by sepw_grid_planned / sepw_degrid_planned until the next
 * sepw_plan; u, v, w need not stay alive.  Binning is amortisable over the
 * gridding/degridding calls of a major cycle (Sec. 6).  For the plain form
 * the plan only records the coordinates' pointers, which must then stay
 * valid and unchanged until the next sepw_plan.  The plan allocates or grows
 * the context's workspace (bins, work items, and for the tensor-core forms
 * the gridder's per-call tap tables); sepw_grid_planned and
 * sepw_degrid_planned then allocate nothing, so those calls can be captured
 * in a CUDA graph. */
SEPW_API int sepw_plan(sepw_ctx *ctx, int64_t nvis, const double *u, const double *v,
              const double *w, sepw_stream_t stream);

/* Batched plan (W-stacking layers, frequency channels, Sec. 4.3): ngrids
 * separate N x N grids, visibilities of grid g at indices
 * vis_offsets[g] .. vis_offsets[g+1]-1 of u, v, w (and vis, weight in the
 * gridding calls).  vis_offsets is a HOST array of ngrids + 1 non-decreasing
 * values starting at 0; it is copied during the call (so the call itself
 * cannot be captured in a CUDA graph; capture the *_planned calls instead).
 * The tiled and tensor-core forms grid the whole batch in ONE persistent
 * launch of sepw_grid_planned / sepw_degrid_planned, whose grid argument is
 * then ngrids * N * N complex64 (grid g at offset g * N * N); the plain form
 * issues one launch per grid.  Tiles of all grids share the work list. */
SEPW_API int sepw_plan_batched(sepw_ctx *ctx, int32_t ngrids, const int64_t *vis_offsets,
                               const double *u, const double *v, const double *w,
                               sepw_stream_t stream);

/* sepw_plan_batched + sepw_grid_planned: grids (ngrids * N * N complex64)
 * are accumulated into (+=). */
SEPW_API int sepw_grid_batched(sepw_ctx *ctx, const float *taps, int32_t ngrids,
                               const int64_t *vis_offsets, const double *u,
                               const double *v, const double *w, const float *vis,
                               const float *weight, float *grids, int64_t *n_dropped,
                               sepw_stream_t stream);

/* Number of visibilities dropped by the current plan.  Host pointer;
 * synchronises `stream`. */
SEPW_API int sepw_plan_dropped(sepw_ctx *ctx, int64_t *n_dropped_host,
                      sepw_stream_t stream);

/* Gridding, Sec. 5:  grid[c_v - S/2 + 1 + k][c_u - S/2 + 1 + j] +=
 *   (W_i V_i taps[p][o_u][j]) * taps[p][o_v][k]   (conjugated taps if w_i < 0)
 * for every kept visibility i.  `grid` is ACCUMULATED into (+=).  vis:
 * complex64 [nvis]; weight: float32 [nvis] or NULL (= 1); taps: the table of
 * sepw_make_taps.  FP32 arithmetic.  The planned variant uses the plan's
 * visibilities (vis and weight indexed as in the call to sepw_plan).
 * n_dropped (device int64, may be NULL) receives the number dropped. */
SEPW_API int sepw_grid(sepw_ctx *ctx, const float *taps, int64_t nvis, const double *u,
              const double *v, const double *w, const float *vis,
              const float *weight, float *grid, int64_t *n_dropped,
              sepw_stream_t stream);
SEPW_API int sepw_grid_planned(sepw_ctx *ctx, const float *taps, const float *vis,
                      const float *weight, float *grid, sepw_stream_t stream);

/* Degridding (prediction, Sec. 2; used for prediction in Cotton-Schwab major
 * cycles, Sec. 6), the exact adjoint of sepw_grid:
 *   vis_out[i] = W_i sum_k conj(tv[k]) sum_j conj(tu[j]) grid[y_k][x_j]
 * with tu, tv the (conjugated if w_i < 0) taps used by sepw_grid.  vis_out
 * (complex64 [nvis]) is OVERWRITTEN; dropped visibilities get 0. */
SEPW_API int sepw_degrid(sepw_ctx *ctx, const float *taps, int64_t nvis, const double *u,
                const double *v, const double *w, const float *grid,
                const float *weight, float *vis_out, int64_t *n_dropped,
                sepw_stream_t stream);
SEPW_API int sepw_degrid_planned(sepw_ctx *ctx, const float *taps, const float *grid,
                        const float *weight, float *vis_out,
                        sepw_stream_t stream);

/* Device status of the context's kernels: a kernel that gives up a bounded
 * wait records SEPW_ETIMEOUT in a device word.  Synchronises `stream`, copies
 * the word to *status (SEPW_OK if nothing was recorded) and resets it. */
SEPW_API int sepw_device_status(sepw_ctx *ctx, int *status, sepw_stream_t stream);

/* Limit of every bounded wait inside the tensor-core kernels of this context
 * (nanoseconds of the GPU's global timer; default 2 s; 1 us .. 60 s, else
 * SEPW_EINVAL).  A kernel whose wait runs out records SEPW_ETIMEOUT (see
 * sepw_device_status), stops issuing work, waits for its own tensor-core
 * operations (bounded by the same limit), releases its tensor memory and
 * returns; its output is then incomplete.  Host only; applies to later calls. */
SEPW_API int sepw_set_wait_limit(sepw_ctx *ctx, uint64_t limit_ns);

/* Schedule of the tiled and tensor-core plans (the visibility-per-tile
 * schedule of a batch of W-stacking layers or channels with uneven counts,
 * Sec. 4.3): `chunk` visibilities per work item (64 .. 2048, a multiple of
 * 32; 0 = 2048, the default) and the number of parts a warp of the FP32
 * block gridder (S = 8, 16) takes of an item at a time (1 .. 16; 0 = 8 on
 * plans of at least 256 visibilities per tile, else 1, the default).  Takes
 * effect at the next sepw_plan (the current plan is invalidated); results
 * do not depend on it beyond FP32 rounding order.  Host only. */
SEPW_API int sepw_set_schedule(sepw_ctx *ctx, int32_t chunk, int32_t grid_parts);

/* FP32 FMA rate probe (no counterpart in the paper): the scatter-form
 * kernels are bound by FP32 fused multiply-adds, and their roofline is stated
 * against the FMA peak derived from unit counts and the clock.  This launches,
 * on `stream`, one kernel that does only FMAs: 4 CTAs of 256 threads per SM,
 * each thread running 8 independent chains of `iters` (1 .. 2^30) FMAs,
 * scalar FFMA (paired = 0) or paired FFMA2 on float2 operands (paired != 0).
 * `out` is a device buffer of at least out_len >= SMs x 1024 floats that
 * receives one per-thread sum (it keeps the chains live); *flops (host)
 * receives the flop count of the launch (2 per FMA).  The caller times the
 * launch with CUDA events on the stream.  Returns SEPW_EINVAL for bad
 * arguments or a short buffer, SEPW_ECUDA if the launch fails. */
SEPW_API int sepw_fma_probe(int paired, int64_t iters, float *out, int64_t out_len,
                            int64_t *flops, sepw_stream_t stream);

/* Bounds-checked build (no counterpart in the paper).  libsepw_checked.so is
 * the same library compiled with SEPW_CHECKED=1: the tiled (scatter-form)
 * gridder and degridder check every work item (tile, visibility range) and
 * every plan record (visibility index, plane, oversample indices, footprint
 * inside the tile and the grid) before use; a failed check records
 * SEPW_EBOUNDS in the context's device status word (sepw_device_status) and
 * the kernel skips that item or visibility instead of accessing out of
 * range.  sepw_checked_build returns 1 in that build, 0 in the default one,
 * which compiles the checks away. */
SEPW_API int sepw_checked_build(void);

/* Test hook of the checked build (no counterpart in the paper): overwrites,
 * in the current plan of ctx, the slot -> visibility index of `slot`
 * (which = 0) or the plane field of the slot's record (which = 1) with
 * `value`, so that a test can see the checks catch it.  Synchronous.  Returns
 * SEPW_ENOTSUP in the default build (nothing there guards such a value),
 * SEPW_ENOPLAN without a tiled plan, SEPW_EINVAL for a slot outside the plan
 * or another `which`. */
SEPW_API int sepw_test_corrupt_plan(sepw_ctx *ctx, int which, int64_t slot, int32_t value);

/* Test hook for the timeout path (no counterpart in the paper): with enable
 * != 0 the tensor-core kernels of this context issue no matrix operations and
 * signal none, so their other roles' bounded waits run out and the call ends
 * with SEPW_ETIMEOUT recorded and the grid or predictions incomplete.  Nothing
 * is left waiting: every wait is bounded (sepw_set_wait_limit).  enable = 0
 * restores normal operation.  Host only. */
SEPW_API int sepw_test_stall_mma(sepw_ctx *ctx, int enable);

/* Image step with grid correction, Sec. 2 (I_D / n = F^-1[grid] / c), in
 * place on an N x N complex64 buffer:
 *   SEPW_GRID_TO_IMAGE:  I[b][a] = n_ab / (c1(nu_a) c1(nu_b)) *
 *       sum_{cu,cv} grid[cv][cu] exp(2 pi i ((cu-N/2) nu_a + (cv-N/2) nu_b))
 *   SEPW_IMAGE_TO_GRID (prediction direction):  grid[cv][cu] =
 *       sum_{a,b} exp(-2 pi i ((cu-N/2) nu_a + (cv-N/2) nu_b)) I[b][a] /
 *       (n_ab c1(nu_a) c1(nu_b))
 * with n_ab = sqrt(1 - l_a^2 - m_b^2).
 *   SEPW_IMAGE_TO_GRID_ADJOINT (the backward pass of prediction):
 *       I[b][a] = 1 / (n_ab c1(nu_a) c1(nu_b)) *
 *       sum_{cu,cv} grid[cv][cu] exp(2 pi i ((cu-N/2) nu_a + (cv-N/2) nu_b))
 *       = GRID_TO_IMAGE / n_ab^2.
 * Uses cuFFT (FP32 C2C); the plan is created on first use. */
SEPW_API int sepw_image(sepw_ctx *ctx, int direction, float *buf, sepw_stream_t stream);

/* Taper of the grid correction: taper[a] = c1(nu_a), nu_a = (a - N/2)/N, the
 * transform of the antialiasing window normalised to c1(0) = 1 (Sec. 2), as
 * used by sepw_image (FP32, device, N floats, overwritten). */
SEPW_API int sepw_taper(sepw_ctx *ctx, float *taper, sepw_stream_t stream);

/* Stored correction of the separable kernel, Sec. 7 (store and apply
 * F_w - F~_w in a small full-dimension table).  The table holds
 *   res[p][ovr][our][k][j] = F_w(d_u, d_v) - F1_w(d_u) F1_w(d_v)
 * (F_w the exact 2-D W-projection kernel, the transform of
 * c1 c1 exp(2 pi i w (n - 1)) over the N x N pixels; F1 the taps of
 * sepw_make_taps) for the support_r x support_r central cells of the S x S
 * footprint (first at (S - support_r)/2) and oversample_r offsets per axis
 * (entry c stands for the fine offset c * OS / oversample_r; a visibility at
 * fine offset o uses entry floor(o / (OS / oversample_r))).  Constraints:
 * 1 <= support_r <= S, S - support_r even, oversample_r divides OS.
 * sepw_residual_count: number of complex entries,
 *   P * oversample_r^2 * support_r^2 (0 for invalid sizes).
 * sepw_make_residual / _f64: build it in float64 on the GPU (complex64 /
 * complex128 output, device).  Not in facet mode (SEPW_ENOTSUP).  Allocates
 * and frees a temporary of P * oversample_r * support_r * N complex128 and
 * synchronises `stream`: a set-up step, not for the hot loop.
 * sepw_grid_residual_planned: the correction pass, ADDS to grid the
 * W_i V_i res (conj(res) for w_i < 0) of every planned visibility; after
 * sepw_grid_planned with the full table (support_r = S, oversample_r = OS)
 * the grid is that of exact 2-D W projection.
 * sepw_degrid_residual_planned: its adjoint, ADDS to vis_out (after
 * sepw_degrid_planned).  Both need a tiled or tensor-core plan (SEPW_ENOTSUP
 * for SEPW_FORM_PLAIN), including batched and W-stacking plans. */
SEPW_API size_t sepw_residual_count(const sepw_params *p, int32_t support_r,
                                    int32_t oversample_r);
SEPW_API int sepw_make_residual(sepw_ctx *ctx, int32_t support_r, int32_t oversample_r,
                                float *table, sepw_stream_t stream);
SEPW_API int sepw_make_residual_f64(sepw_ctx *ctx, int32_t support_r, int32_t oversample_r,
                                    double *table, sepw_stream_t stream);
SEPW_API int sepw_grid_residual_planned(sepw_ctx *ctx, int32_t support_r, int32_t oversample_r,
                                        const float *table, const float *vis,
                                        const float *weight, float *grid, sepw_stream_t stream);
SEPW_API int sepw_degrid_residual_planned(sepw_ctx *ctx, int32_t support_r,
                                          int32_t oversample_r, const float *table,
                                          const float *grid, const float *weight,
                                          float *vis_out, sepw_stream_t stream);

/* Image-plane faceting, Sec. 4.1 (Eq. gt-facet).  sepw_set_facet puts the
 * context in facet mode for the facet centred at (l0, m0) (direction cosines
 * of the original image plane, l0^2 + m0^2 < 1; the context's grid_size and
 * fov are the facet's).  In facet mode:
 *   - sepw_make_taps / _f64 write TWO tables, [2][P][OS][S]: the u-direction
 *     table of the screen g^l_w(l) = exp(2 pi i w a_l l^2) and then the
 *     v-direction table of g^m_w(m) = exp(2 pi i w a_m m^2), with
 *     a_l = -(1/n0 + l0^2/n0^3)/2, a_m = -(1/n0 + m0^2/n0^3)/2, n0 = h(l0, m0),
 *     l, m relative to the facet centre (no quartic term);
 *   - gridding and degridding take the v-direction taps from the second table;
 *   - the image steps (sepw_image, W stacking) take n at l0 + l, m0 + m.
 * sepw_set_facet(ctx, 0, 0, 0) (enable = 0) returns to the one-table screen of
 * Eq. gt.  The plan is unaffected; regenerate the taps after a change. */
SEPW_API int sepw_set_facet(sepw_ctx *ctx, int enable, double l0, double m0);

/* Visibilities of the context's facet (Sec. 4.1).  SEPW_FACET_IN:
 *   u_out = u - w l0 / n0,  v_out = v - w m0 / n0   (IEEE double, this order)
 *   vis_out = vis exp(2 pi i (u l0 + v m0 + w (n0 - 1)))
 * (plan and grid with u_out, v_out, w and vis_out).  SEPW_FACET_OUT:
 *   vis_out = vis exp(-2 pi i (u l0 + v m0 + w (n0 - 1)))
 * (predictions of the facet back to the original phase centre).  u_out,
 * v_out (device doubles) may be NULL to skip the shift, vis / vis_out
 * (device complex64) may be NULL to skip the rotation; vis_out may equal vis.
 * Requires facet mode (SEPW_ENOTSUP otherwise). */
#define SEPW_FACET_IN 0
#define SEPW_FACET_OUT 1
SEPW_API int sepw_facet_shift(sepw_ctx *ctx, int direction, int64_t nvis, const double *u,
                              const double *v, const double *w, const float *vis,
                              double *u_out, double *v_out, float *vis_out,
                              sepw_stream_t stream);

/* Hybrid W stacking, Sec. 4.3: visibilities are partitioned by w into
 * slices; the mean w term of a slice is corrected in image space by the
 * phase of its centre and the residual w by the separable W-projection kernel
 * (whose planes span |w - w_c| <= w_max of the context).
 *
 * sepw_wstack_plan: w_centres (HOST, nslices doubles, finite, strictly
 * increasing) are the slice centres.  Visibility i goes to the slice with the
 * nearest centre (|w_i - w_c| in IEEE double, ties to the lower centre;
 * non-finite w to slice 0) and its residual is w_i - w_c (IEEE double).  A
 * batched plan of nslices grids is then built on (u, v, w - w_c) and becomes
 * the context's plan: sepw_grid_planned / sepw_degrid_planned then take
 * vis, weight and vis_out in the CALLER'S order and nslices x N x N
 * complex64 grids [slice][v][u].  Visibilities whose residual falls beyond
 * w_max or whose footprint leaves the grid are dropped (sepw_plan_dropped).
 * slice_out (device int32 [nvis]) receives each visibility's slice, or NULL.
 * Requires a tiled or tensor-core form (SEPW_ENOTSUP for SEPW_FORM_PLAIN);
 * synchronises `stream` once (slice counts).  The centres are kept for
 * sepw_wstack_image / sepw_wstack_model_grids until the next call. */
SEPW_API int sepw_wstack_plan(sepw_ctx *ctx, int32_t nslices, const double *w_centres,
                              int64_t nvis, const double *u, const double *v, const double *w,
                              int32_t *slice_out, sepw_stream_t stream);

/* Dirty image of hybrid W stacking from the slice grids (nslices x N x N
 * complex64, device; transformed IN PLACE, their contents are destroyed):
 *   image[b][a] = sum_c exp(2 pi i w_c (n_ab - 1)) GRID_TO_IMAGE(grid_c)[b][a]
 * (GRID_TO_IMAGE as in sepw_image).  image (N x N complex64) is overwritten.
 * One batched cuFFT over the slices; FP32. */
SEPW_API int sepw_wstack_image(sepw_ctx *ctx, float *slice_grids, float *image,
                               sepw_stream_t stream);

/* Prediction direction: slice_grids[c] (overwritten) =
 *   IMAGE_TO_GRID(image * exp(-2 pi i w_c (n - 1)))   (IMAGE_TO_GRID as in
 * sepw_image); degridding them with the W-stacking plan predicts the
 * visibilities of the model image (N x N complex64, device, not modified). */
SEPW_API int sepw_wstack_model_grids(sepw_ctx *ctx, const float *image, float *slice_grids,
                                     sepw_stream_t stream);

/* Limits of sepw_grid_noalloc's fixed scratch array. */
#define SEPW_NOALLOC_MAX_VIS 524288    /* visibilities per call            */
#define SEPW_NOALLOC_MAX_TILES 65536   /* ((N - S)/T + 1)^2 tiles per grid */

/* Gridding that allocates no device memory.  The paper has no counterpart:
 * this is a service for callers that cannot let a library allocate, such as
 * a real-time pipeline that reserves all of its device memory at start-up and
 * must not block on cudaMalloc (which may synchronise the device) while it
 * observes, or a plugin inside a framework that owns the device memory pool.
 *
 * Same result as sepw_grid with the tiled FP32 form (p->form is ignored: the
 * parameters are checked as for SEPW_FORM_TILED, tile 0 meaning 32), but no
 * context is needed and nothing is allocated: the binning workspace is one
 * file-scope device array of about 26 MB compiled into the library, which
 * every GPU that loads the library keeps until the process exits.  The call
 * makes no cudaMalloc / cudaFree and no allocating library call.
 *   - p, taps, u, v, w, vis, weight (NULL = 1), grid (accumulated, +=):
 *     as for sepw_grid; taps must be 16-byte aligned (SEPW_EINVAL
 *     otherwise); n_dropped: device int64 or NULL.
 *   - nvis > SEPW_NOALLOC_MAX_VIS, or a grid/tile combination with more than
 *     SEPW_NOALLOC_MAX_TILES tiles, returns SEPW_ETOOLARGE before anything is
 *     enqueued; split the visibilities into several calls instead (gridding
 *     accumulates).
 *   - Start-up: the array's device memory is reserved by the CUDA driver when
 *     it loads the library's device code on a device.  Under CUDA's lazy
 *     module loading (the default) that happens at the first call on that
 *     device (or at the first launch of any other libsepw entry point there).
 *     The first call also looks up the array's device address, with that
 *     device current, and caches it.  A caller that may not allocate later
 *     should therefore make one call at start-up (nvis = 0 is enough), and
 *     before any stream capture on the device.
 *   - Every call reuses the same array.  Two calls whose GPU work can overlap
 *     in time race on it and give wrong results, whether they come from two
 *     streams, two host threads or a captured graph replayed beside a direct
 *     call: order them on one stream or with events.  Calls on different
 *     devices do not share an array. */
SEPW_API int sepw_grid_noalloc(const sepw_params *p, const float *taps, int64_t nvis,
                               const double *u, const double *v, const double *w,
                               const float *vis, const float *weight, float *grid,
                               int64_t *n_dropped, sepw_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SEPW_H */
