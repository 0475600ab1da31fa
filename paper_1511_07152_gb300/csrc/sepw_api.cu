// C ABI of libsepw: parameter checks, context and workspace management, and
// the launch sequence of each entry point.  See include/sepw.h for the
// contract of every function.
#include <cufft.h>
#include <math.h>
#include <new>
#include <vector>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include "sepw_internal.cuh"
#include "sepw_tc_ptx.cuh"

using namespace sepw;

namespace {
// NVTX range over one entry point (host side: it brackets the launches the
// call enqueues).  The header-only NVTX library does nothing unless a
// profiler is attached.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};
}  // namespace

struct sepw_ctx {
    sepw_params p;
    DevParams dp;
    int device = 0;
    int num_sms = 0;
    double *d_taper64 = nullptr;
    float *d_taper32 = nullptr;
    double2 *d_tw = nullptr;
    int32_t *d_status = nullptr;  // SEPW_ETIMEOUT recorded by a kernel
    TcControl tc_ctl{tcx::kDefaultWaitNs, 0};
    // workspace of the contraction gridder's pre-shifted tap tables
    unsigned char *d_tc2 = nullptr;
    size_t tc2_cap = 0;
    // workspace of the tiled gridder's planar copy of the caller's tap
    // table(s) (two tables: facet mode)
    float *d_planar = nullptr;
    Plan plan;
    cufftHandle fft = 0;
    bool fft_ready = false;
    // hybrid W stacking: slice centres of the last sepw_wstack_plan and the
    // workspace of the slice sort
    std::vector<double> ws_centres;
    double *d_ws_c64 = nullptr;
    float *d_ws_c32 = nullptr;
    int32_t ws_centres_cap = 0;
    int32_t *d_ws_count = nullptr;  // per slice: counts, then cursors
    int32_t *d_ws_slice = nullptr;
    int32_t *d_ws_part = nullptr;
    double *d_ws_u = nullptr, *d_ws_v = nullptr, *d_ws_w = nullptr;
    int64_t ws_cap = 0;
    cufftHandle fft_batch = 0;
    int fft_batch_n = 0;  // slices of fft_batch, 0 = none
    char err[512] = {0};
};

namespace {

int fail(sepw_ctx *ctx, int code, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(sepw_ctx *ctx, cudaError_t e, const char *where)
{
    return fail(ctx, SEPW_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define SEPW_CUDA(ctx, call)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess)                                \
            return cuda_fail((ctx), e_, #call);               \
    } while (0)

bool is_tc_form(int form)
{
    return form == SEPW_FORM_TC_BF16 || form == SEPW_FORM_TC_FP16 ||
           form == SEPW_FORM_TC_FP16X2 || form == SEPW_FORM_TC_BF16X2 ||
           form == SEPW_FORM_TC_TF32;
}

int tc_prec(int form)
{
    return form == SEPW_FORM_TC_BF16 ? 0 : form == SEPW_FORM_TC_FP16 ? 1
         : form == SEPW_FORM_TC_FP16X2 ? 2 : form == SEPW_FORM_TC_BF16X2 ? 3 : 4;
}

// tensor-core workspace: the gridder's tables, then (256-byte aligned) the
// degridder's
size_t tc_grid_part_bytes(const DevParams &dp, int64_t items_capacity)
{
    return (tc2_tables_bytes(dp, items_capacity) + 255) & ~(size_t)255;
}

size_t tc_workspace_bytes(const DevParams &dp, int64_t items_capacity)
{
    return tc_grid_part_bytes(dp, items_capacity) + tc_degrid_tables_bytes(dp, items_capacity);
}

int effective_tile(const sepw_params *p)
{
    if (p->tile != 0)
        return p->tile;
    return is_tc_form(p->form) ? tc2_tile_for_support(p->support) : 32;
}

}  // namespace

// Device-side parameters of p (tile resolved by its form); shared with the
// allocation-free entry point.
DevParams sepw::make_dev_params(const sepw_params *p)
{
    DevParams d;
    d.N = p->grid_size;
    d.S = p->support;
    d.OS = p->oversample;
    d.P = p->n_wplanes;
    d.T = effective_tile(p);
    d.ntx = (d.N - d.S) / d.T + 1;
    d.t_inv = tile_reciprocal(d.T);
    d.fov = p->fov;
    d.half = (double)(d.N / 2);
    d.os_d = (double)d.OS;
    d.os_log2 = -1;
    for (int k = 0; k < 31; ++k)
        if ((1 << k) == d.OS)
            d.os_log2 = k;
    locate_fast_bounds(d.N, d.os_log2, d.fast_elim, d.fast_near);
    d.plane_r = d.P > 1 ? (double)(d.P - 1) / p->w_max : 0.0;
    d.w_max = p->w_max;
    d.gamma = p->gamma;
    d.beta = p->kb_beta;
    return d;
}

namespace {

DevParams make_dev(const sepw_params *p) { return sepw::make_dev_params(p); }

template <typename T>
int grow(sepw_ctx *ctx, T **ptr, size_t count)
{
    if (*ptr)
        cudaFree(*ptr);
    *ptr = nullptr;
    if (count == 0)
        count = 1;
    cudaError_t e = cudaMalloc((void **)ptr, count * sizeof(T));
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(ctx, SEPW_ENOMEM, "cudaMalloc of %zu bytes: %s", count * sizeof(T),
                    cudaGetErrorString(e));
    }
    return SEPW_OK;
}

void free_plan(Plan &pl)
{
    cudaFree(pl.d_tile);
    cudaFree(pl.d_rank);
    cudaFree(pl.d_rec0);
    cudaFree(pl.d_rec);
    cudaFree(pl.d_perm);
    cudaFree(pl.d_drop_list);
    cudaFree(pl.d_bin);
    cudaFree(pl.d_tile_count);
    cudaFree(pl.d_tile_cursor);
    cudaFree(pl.d_items);
    cudaFree(pl.d_nitems);
    cudaFree(pl.d_item_counter);
    cudaFree(pl.d_dropped);
    cudaFree(pl.d_offsets);
    pl = Plan();
}

bool is_device_ptr(const void *ptr)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int check_dev(sepw_ctx *ctx, const void *ptr, const char *name, bool allow_null)
{
    if (!ptr)
        return allow_null ? SEPW_OK : fail(ctx, SEPW_EINVAL, "%s is NULL", name);
    if (!is_device_ptr(ptr))
        return fail(ctx, SEPW_EINVAL, "%s is not device memory", name);
    if (((uintptr_t)ptr) & 7)
        return fail(ctx, SEPW_EINVAL, "%s is not 8-byte aligned", name);
    return SEPW_OK;
}

int ensure_plan_capacity(sepw_ctx *ctx, int64_t nvis, int ngrids)
{
    Plan &pl = ctx->plan;
    int rc;
    const int64_t ntiles64 = (int64_t)ctx->dp.ntx * ctx->dp.ntx * ngrids;
    if (ntiles64 > (1ll << 26))  // bin ids (tile * kSubBins + sub) stay in int32
        return fail(ctx, SEPW_EINVAL, "too many tiles (%lld)", (long long)ntiles64);
    const int ntiles = (int)ntiles64;
    if (!pl.d_nitems) {
        if ((rc = grow(ctx, &pl.d_nitems, 1)) || (rc = grow(ctx, &pl.d_item_counter, 2)) ||
            (rc = grow(ctx, &pl.d_dropped, 1)))
            return rc;
    }
    if (pl.tiles_capacity < ntiles) {
        if ((rc = grow(ctx, &pl.d_tile_count, ntiles)) ||
            (rc = grow(ctx, &pl.d_tile_cursor, ntiles)) ||
            (rc = grow(ctx, &pl.d_bin, (size_t)ntiles * kSubBins)))
            return rc;
        pl.tiles_capacity = ntiles;
    }
    pl.ntiles = ntiles;
    if (ctx->p.form == SEPW_FORM_PLAIN)
        return SEPW_OK;  // the plain form keeps no per-visibility state
    if (pl.capacity < nvis) {
        int64_t cap = nvis;
        if ((rc = grow(ctx, &pl.d_tile, cap)) || (rc = grow(ctx, &pl.d_rank, cap)) ||
            (rc = grow(ctx, &pl.d_rec0, cap)) ||
            (rc = grow(ctx, &pl.d_rec, cap)) || (rc = grow(ctx, &pl.d_perm, cap)) ||
            (rc = grow(ctx, &pl.d_drop_list, cap)))
            return rc;
        pl.capacity = cap;
    }
    int64_t items = (int64_t)ntiles + nvis / ctx->dp.chunk + 1;
    if (items > INT32_MAX)
        return fail(ctx, SEPW_EINVAL, "too many work items");
    if (pl.items_capacity < items) {
        if ((rc = grow(ctx, &pl.d_items, (size_t)items)))
            return rc;
        pl.items_capacity = (int32_t)items;
    }
    return SEPW_OK;
}

}  // namespace

extern "C" {

int sepw_version(void) { return SEPW_VERSION; }

const char *sepw_strerror(int status)
{
    switch (status) {
    case SEPW_OK: return "ok";
    case SEPW_EINVAL: return "invalid argument";
    case SEPW_ENOMEM: return "out of device memory";
    case SEPW_ECUDA: return "CUDA error";
    case SEPW_ETIMEOUT: return "device wait timed out";
    case SEPW_ENOTSUP: return "not supported for these parameters";
    case SEPW_ENOPLAN: return "no current plan";
    case SEPW_ETOOLARGE: return "size exceeds the fixed scratch of sepw_grid_noalloc";
    case SEPW_EBOUNDS: return "a bounds check of the checked build failed";
    default: return "unknown status";
    }
}

int sepw_check_params(const sepw_params *p)
{
    if (!p)
        return SEPW_EINVAL;
    const int N = p->grid_size, S = p->support, OS = p->oversample, P = p->n_wplanes;
    if (N < 16 || N > 65536 || (N & 1))
        return SEPW_EINVAL;
    if (S < 2 || S > 32 || (S & 1) || S > N)
        return SEPW_EINVAL;
    if (OS < 1 || OS > 256)
        return SEPW_EINVAL;
    if (P < 1 || P > 32768)
        return SEPW_EINVAL;
    if (!(p->fov > 0.0) || !(p->fov < 1.4) || !isfinite(p->fov))
        return SEPW_EINVAL;
    if (!(p->w_max > 0.0) || !isfinite(p->w_max))
        return SEPW_EINVAL;
    if (!isfinite(p->gamma))
        return SEPW_EINVAL;
    if (!(p->kb_beta > 0.0) || !(p->kb_beta < 1e4))
        return SEPW_EINVAL;
    const int T = effective_tile(p);
    if (T < 8 || T > 64 || (T & 1) || T + S - 1 > kMaxWindow)
        return SEPW_EINVAL;
    if (p->form != SEPW_FORM_PLAIN && p->form != SEPW_FORM_TILED && !is_tc_form(p->form))
        return SEPW_ENOTSUP;
    if (is_tc_form(p->form) && S > 16)
        return SEPW_ENOTSUP;
    if (is_tc_form(p->form) && T + S - 1 > 32)  // the contraction gridder's window
        return SEPW_EINVAL;
    return SEPW_OK;
}

size_t sepw_taps_count(const sepw_params *p)
{
    if (sepw_check_params(p) != SEPW_OK)
        return 0;
    return (size_t)p->n_wplanes * p->oversample * p->support;
}

int sepw_create(sepw_ctx **out, const sepw_params *p)
{
    if (!out)
        return SEPW_EINVAL;
    *out = nullptr;
    int rc = sepw_check_params(p);
    if (rc != SEPW_OK)
        return rc;
    sepw_ctx *ctx = new (std::nothrow) sepw_ctx();
    if (!ctx)
        return SEPW_ENOMEM;
    ctx->p = *p;
    ctx->dp = make_dev(p);
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount,
                                   ctx->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return SEPW_ECUDA;
    }
    const int N = p->grid_size;
    if ((rc = grow(ctx, &ctx->d_taper64, N)) || (rc = grow(ctx, &ctx->d_taper32, N)) ||
        (rc = grow(ctx, &ctx->d_tw, (size_t)N * p->oversample)) ||
        (rc = grow(ctx, &ctx->d_status, 1)) ||
        (rc = grow(ctx, &ctx->d_planar, 2 * 2 * sepw_taps_count(p)))) {
        sepw_destroy(ctx);
        return rc;
    }
    e = cudaMemset(ctx->d_status, 0, sizeof(int32_t));
    if (e == cudaSuccess)
        e = launch_taper(ctx->dp, ctx->d_taper64, ctx->d_taper32, 0);
    if (e == cudaSuccess)
        e = launch_twiddles(ctx->dp, ctx->d_tw, 0);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sepw_destroy(ctx);
        return SEPW_ECUDA;
    }
    *out = ctx;
    return SEPW_OK;
}

void sepw_destroy(sepw_ctx *ctx)
{
    if (!ctx)
        return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->fft_ready)
        cufftDestroy(ctx->fft);
    if (ctx->fft_batch_n)
        cufftDestroy(ctx->fft_batch);
    cudaFree(ctx->d_ws_c64);
    cudaFree(ctx->d_ws_c32);
    cudaFree(ctx->d_ws_count);
    cudaFree(ctx->d_ws_slice);
    cudaFree(ctx->d_ws_part);
    cudaFree(ctx->d_ws_u);
    cudaFree(ctx->d_ws_v);
    cudaFree(ctx->d_ws_w);
    cudaFree(ctx->d_taper64);
    cudaFree(ctx->d_taper32);
    cudaFree(ctx->d_tw);
    cudaFree(ctx->d_status);
    cudaFree(ctx->d_planar);
    cudaFree(ctx->d_tc2);
    free_plan(ctx->plan);
    cudaSetDevice(cur);
    delete ctx;
}

const char *sepw_last_error(const sepw_ctx *ctx) { return ctx ? ctx->err : "no context"; }

int sepw_make_taps(sepw_ctx *ctx, float *taps, sepw_stream_t stream)
{
    Range range_("sepw_make_taps");
    if (!ctx)
        return SEPW_EINVAL;
    int rc = check_dev(ctx, taps, "taps", false);
    if (rc)
        return rc;
    SEPW_CUDA(ctx, launch_taps(ctx->dp, ctx->d_taper64, ctx->d_tw, nullptr,
                               (float2 *)taps, (cudaStream_t)stream));
    return SEPW_OK;
}

int sepw_make_taps_f64(sepw_ctx *ctx, double *taps, sepw_stream_t stream)
{
    if (!ctx)
        return SEPW_EINVAL;
    int rc = check_dev(ctx, taps, "taps", false);
    if (rc)
        return rc;
    SEPW_CUDA(ctx, launch_taps(ctx->dp, ctx->d_taper64, ctx->d_tw, (double2 *)taps,
                               nullptr, (cudaStream_t)stream));
    return SEPW_OK;
}

int sepw_locate(sepw_ctx *ctx, int64_t nvis, const double *u, const double *v,
                const double *w, int32_t *cu, int32_t *cv, int32_t *ou, int32_t *ov,
                int32_t *plane, uint8_t *conj, uint8_t *keep, sepw_stream_t stream)
{
    Range range_("sepw_locate");
    if (!ctx)
        return SEPW_EINVAL;
    if (nvis < 0)
        return fail(ctx, SEPW_EINVAL, "nvis < 0");
    if (nvis == 0)
        return SEPW_OK;
    int rc;
    if ((rc = check_dev(ctx, u, "u", false)) || (rc = check_dev(ctx, v, "v", false)) ||
        (rc = check_dev(ctx, w, "w", false)))
        return rc;
    SEPW_CUDA(ctx, launch_locate(ctx->dp, nvis, u, v, w, cu, cv, ou, ov, plane, conj,
                                 keep, (cudaStream_t)stream));
    return SEPW_OK;
}

static int plan_impl(sepw_ctx *ctx, int32_t ngrids, const int64_t *offsets_host, int64_t nvis,
                     const double *u, const double *v, const double *w, cudaStream_t s)
{
    Range range_("sepw_plan");
    ctx->plan.valid = false;
    if (nvis < 0 || nvis > (int64_t)INT32_MAX - 1)
        return fail(ctx, SEPW_EINVAL, "nvis out of range [0, 2^31 - 2]");
    if (ngrids < 1)
        return fail(ctx, SEPW_EINVAL, "ngrids < 1");
    int rc;
    if (nvis > 0 && ((rc = check_dev(ctx, u, "u", false)) ||
                     (rc = check_dev(ctx, v, "v", false)) ||
                     (rc = check_dev(ctx, w, "w", false))))
        return rc;
    if ((rc = ensure_plan_capacity(ctx, nvis, ngrids)))
        return rc;
    Plan &pl = ctx->plan;
    pl.form = ctx->p.form;
    pl.nvis = nvis;
    pl.ngrids = ngrids;
    pl.h_offsets.assign(offsets_host, offsets_host + ngrids + 1);
    if (ngrids > 1) {
        if (pl.offsets_capacity < ngrids + 1) {
            if ((rc = grow(ctx, &pl.d_offsets, (size_t)ngrids + 1)))
                return rc;
            pl.offsets_capacity = ngrids + 1;
        }
        SEPW_CUDA(ctx, cudaMemcpyAsync(pl.d_offsets, pl.h_offsets.data(),
                                       sizeof(int64_t) * (ngrids + 1), cudaMemcpyHostToDevice,
                                       s));
    }
    if (ctx->p.form == SEPW_FORM_PLAIN) {
        pl.u = u;
        pl.v = v;
        pl.w = w;
        SEPW_CUDA(ctx, cudaMemsetAsync(pl.d_dropped, 0, sizeof(unsigned long long), s));
        SEPW_CUDA(ctx, launch_count_dropped(ctx->dp, nvis, u, v, w, pl.d_dropped, s));
    } else {
        pl.u = pl.v = pl.w = nullptr;
        if (is_tc_form(ctx->p.form)) {
            // the contraction gridder's per-call tables and per-item scales:
            // allocated here, so that the *_planned calls allocate nothing and
            // can be captured in a CUDA graph
            const size_t need = tc_workspace_bytes(ctx->dp, pl.items_capacity);
            if (ctx->tc2_cap < need) {
                ctx->tc2_cap = 0;
                if ((rc = grow(ctx, &ctx->d_tc2, need)))
                    return rc;
                ctx->tc2_cap = need;
            }
        }
        SEPW_CUDA(ctx, launch_plan(ctx->dp, nvis, u, v, w, pl, s));
    }
    pl.valid = true;
    return SEPW_OK;
}

int sepw_plan(sepw_ctx *ctx, int64_t nvis, const double *u, const double *v,
              const double *w, sepw_stream_t stream)
{
    if (!ctx)
        return SEPW_EINVAL;
    const int64_t offsets[2] = {0, nvis};
    return plan_impl(ctx, 1, offsets, nvis, u, v, w, (cudaStream_t)stream);
}

int sepw_plan_batched(sepw_ctx *ctx, int32_t ngrids, const int64_t *vis_offsets,
                      const double *u, const double *v, const double *w,
                      sepw_stream_t stream)
{
    if (!ctx)
        return SEPW_EINVAL;
    if (ngrids < 1 || !vis_offsets)
        return fail(ctx, SEPW_EINVAL, "ngrids < 1 or vis_offsets NULL");
    if (vis_offsets[0] != 0)
        return fail(ctx, SEPW_EINVAL, "vis_offsets[0] != 0");
    for (int g = 0; g < ngrids; ++g)
        if (vis_offsets[g + 1] < vis_offsets[g])
            return fail(ctx, SEPW_EINVAL, "vis_offsets decrease at grid %d", g);
    return plan_impl(ctx, ngrids, vis_offsets, vis_offsets[ngrids], u, v, w,
                     (cudaStream_t)stream);
}

int sepw_plan_dropped(sepw_ctx *ctx, int64_t *n_dropped_host, sepw_stream_t stream)
{
    if (!ctx || !n_dropped_host)
        return SEPW_EINVAL;
    if (!ctx->plan.valid)
        return fail(ctx, SEPW_ENOPLAN, "no plan");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long n = 0;
    SEPW_CUDA(ctx, cudaMemcpyAsync(&n, ctx->plan.d_dropped, sizeof(n),
                                   cudaMemcpyDeviceToHost, s));
    SEPW_CUDA(ctx, cudaStreamSynchronize(s));
    *n_dropped_host = (int64_t)n;
    return SEPW_OK;
}

int sepw_grid_planned(sepw_ctx *ctx, const float *taps, const float *vis,
                      const float *weight, float *grid, sepw_stream_t stream)
{
    Range range_("sepw_grid");
    if (!ctx)
        return SEPW_EINVAL;
    if (!ctx->plan.valid)
        return fail(ctx, SEPW_ENOPLAN, "no plan");
    int rc;
    if ((rc = check_dev(ctx, taps, "taps", false)) || (rc = check_dev(ctx, grid, "grid", false)))
        return rc;
    const Plan &pl = ctx->plan;
    if (pl.nvis == 0)
        return SEPW_OK;
    if ((rc = check_dev(ctx, vis, "vis", false)) ||
        (rc = check_dev(ctx, weight, "weight", true)))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (pl.form == SEPW_FORM_PLAIN) {
        // one plain launch per grid of the batch
        const int64_t n2 = (int64_t)ctx->p.grid_size * ctx->p.grid_size;
        for (int g = 0; g < pl.ngrids; ++g) {
            const int64_t a0 = pl.h_offsets[g], n = pl.h_offsets[g + 1] - a0;
            SEPW_CUDA(ctx, launch_grid_plain(ctx->dp, n, pl.u + a0, pl.v + a0, pl.w + a0,
                                             (const float2 *)vis + a0,
                                             weight ? weight + a0 : nullptr,
                                             (const float2 *)taps, (float2 *)grid + g * n2,
                                             nullptr, s));
        }
    } else if (is_tc_form(pl.form)) {
        if (ctx->tc2_cap < tc_workspace_bytes(ctx->dp, pl.items_capacity))
            return fail(ctx, SEPW_ENOPLAN, "tensor-core workspace missing (plan first)");
        SEPW_CUDA(ctx, launch_grid_tc2(ctx->dp, pl, (const float2 *)vis, weight,
                                       (const float2 *)taps, ctx->d_tc2, (float2 *)grid,
                                       ctx->num_sms, tc_prec(pl.form), ctx->d_status,
                                       ctx->tc_ctl, s));
    } else {
        if (((uintptr_t)taps) & 15)
            return fail(ctx, SEPW_EINVAL, "taps must be 16-byte aligned");
        DevParams dp = ctx->dp;
        dp.chk_status = ctx->d_status;  // the checked build's bounds failures
        SEPW_CUDA(ctx, launch_grid_tiled(dp, pl, (const float2 *)vis, weight,
                                         (const float2 *)taps, ctx->d_planar, (float2 *)grid,
                                         ctx->num_sms, s));
    }
    return SEPW_OK;
}

int sepw_degrid_planned(sepw_ctx *ctx, const float *taps, const float *grid,
                        const float *weight, float *vis_out, sepw_stream_t stream)
{
    Range range_("sepw_degrid");
    if (!ctx)
        return SEPW_EINVAL;
    if (!ctx->plan.valid)
        return fail(ctx, SEPW_ENOPLAN, "no plan");
    int rc;
    if ((rc = check_dev(ctx, taps, "taps", false)) || (rc = check_dev(ctx, grid, "grid", false)))
        return rc;
    const Plan &pl = ctx->plan;
    if (pl.nvis == 0)
        return SEPW_OK;
    if ((rc = check_dev(ctx, vis_out, "vis_out", false)) ||
        (rc = check_dev(ctx, weight, "weight", true)))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (pl.form == SEPW_FORM_PLAIN) {
        const int64_t n2 = (int64_t)ctx->p.grid_size * ctx->p.grid_size;
        for (int g = 0; g < pl.ngrids; ++g) {
            const int64_t a0 = pl.h_offsets[g], n = pl.h_offsets[g + 1] - a0;
            SEPW_CUDA(ctx, launch_degrid_plain(ctx->dp, n, pl.u + a0, pl.v + a0, pl.w + a0,
                                               (const float2 *)grid + g * n2,
                                               weight ? weight + a0 : nullptr,
                                               (const float2 *)taps,
                                               (float2 *)vis_out + a0, nullptr, s));
        }
    } else {
        if (((uintptr_t)taps) & 15)
            return fail(ctx, SEPW_EINVAL, "taps must be 16-byte aligned");
        SEPW_CUDA(ctx, launch_zero_dropped(pl, (float2 *)vis_out, s));
        if (pl.form == SEPW_FORM_TC_BF16 || pl.form == SEPW_FORM_TC_FP16 ||
            pl.form == SEPW_FORM_TC_FP16X2 || pl.form == SEPW_FORM_TC_BF16X2) {
            if (ctx->tc2_cap < tc_workspace_bytes(ctx->dp, pl.items_capacity))
                return fail(ctx, SEPW_ENOPLAN, "tensor-core workspace missing (plan first)");
            SEPW_CUDA(ctx, launch_degrid_tc(ctx->dp, pl, (const float2 *)grid, weight,
                                            (const float2 *)taps,
                                            ctx->d_tc2 + tc_grid_part_bytes(ctx->dp,
                                                                            pl.items_capacity),
                                            (float2 *)vis_out, ctx->num_sms, tc_prec(pl.form),
                                            ctx->d_status, ctx->tc_ctl, s));
        } else {
            DevParams dp = ctx->dp;
            dp.chk_status = ctx->d_status;  // the checked build's bounds failures
            SEPW_CUDA(ctx, launch_degrid_tiled(dp, pl, (const float2 *)grid, weight,
                                               (const float2 *)taps, (float2 *)vis_out,
                                               ctx->num_sms, s));
        }
    }
    return SEPW_OK;
}

static int copy_dropped(sepw_ctx *ctx, int64_t *n_dropped, cudaStream_t s)
{
    if (!n_dropped)
        return SEPW_OK;
    int rc = check_dev(ctx, n_dropped, "n_dropped", false);
    if (rc)
        return rc;
    SEPW_CUDA(ctx, cudaMemcpyAsync(n_dropped, ctx->plan.d_dropped, sizeof(int64_t),
                                   cudaMemcpyDeviceToDevice, s));
    return SEPW_OK;
}

int sepw_grid(sepw_ctx *ctx, const float *taps, int64_t nvis, const double *u,
              const double *v, const double *w, const float *vis, const float *weight,
              float *grid, int64_t *n_dropped, sepw_stream_t stream)
{
    if (!ctx)
        return SEPW_EINVAL;
    int rc = sepw_plan(ctx, nvis, u, v, w, stream);
    if (rc)
        return rc;
    if ((rc = sepw_grid_planned(ctx, taps, vis, weight, grid, stream)))
        return rc;
    return copy_dropped(ctx, n_dropped, (cudaStream_t)stream);
}

int sepw_grid_batched(sepw_ctx *ctx, const float *taps, int32_t ngrids,
                      const int64_t *vis_offsets, const double *u, const double *v,
                      const double *w, const float *vis, const float *weight, float *grids,
                      int64_t *n_dropped, sepw_stream_t stream)
{
    if (!ctx)
        return SEPW_EINVAL;
    int rc = sepw_plan_batched(ctx, ngrids, vis_offsets, u, v, w, stream);
    if (rc)
        return rc;
    if ((rc = sepw_grid_planned(ctx, taps, vis, weight, grids, stream)))
        return rc;
    return copy_dropped(ctx, n_dropped, (cudaStream_t)stream);
}

int sepw_degrid(sepw_ctx *ctx, const float *taps, int64_t nvis, const double *u,
                const double *v, const double *w, const float *grid, const float *weight,
                float *vis_out, int64_t *n_dropped, sepw_stream_t stream)
{
    if (!ctx)
        return SEPW_EINVAL;
    int rc = sepw_plan(ctx, nvis, u, v, w, stream);
    if (rc)
        return rc;
    if ((rc = sepw_degrid_planned(ctx, taps, grid, weight, vis_out, stream)))
        return rc;
    return copy_dropped(ctx, n_dropped, (cudaStream_t)stream);
}

int sepw_device_status(sepw_ctx *ctx, int *status, sepw_stream_t stream)
{
    if (!ctx || !status)
        return SEPW_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t v = 0;
    SEPW_CUDA(ctx, cudaMemcpyAsync(&v, ctx->d_status, sizeof(v), cudaMemcpyDeviceToHost, s));
    SEPW_CUDA(ctx, cudaStreamSynchronize(s));
    SEPW_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int32_t), s));
    *status = v;
    return SEPW_OK;
}

int sepw_set_wait_limit(sepw_ctx *ctx, uint64_t limit_ns)
{
    if (!ctx)
        return SEPW_EINVAL;
    if (limit_ns < 1000 || limit_ns > 60000000000ull)
        return fail(ctx, SEPW_EINVAL, "wait limit %llu ns outside [1 us, 60 s]",
                    (unsigned long long)limit_ns);
    ctx->tc_ctl.wait_ns = limit_ns;
    return SEPW_OK;
}

int sepw_set_schedule(sepw_ctx *ctx, int32_t chunk, int32_t grid_parts)
{
    if (!ctx)
        return SEPW_EINVAL;
    if (chunk == 0)
        chunk = kChunk;
    if (chunk < 64 || chunk > kChunk || chunk % 32)
        return fail(ctx, SEPW_EINVAL, "chunk %d outside 64..%d or not a multiple of 32", chunk,
                    kChunk);
    if (grid_parts < 0 || grid_parts > 16)
        return fail(ctx, SEPW_EINVAL, "grid_parts %d outside 0..16", grid_parts);
    ctx->dp.chunk = chunk;
    ctx->dp.grid_parts = grid_parts;
    ctx->plan.valid = false;  // the next sepw_plan cuts items of the new size
    return SEPW_OK;
}

int sepw_checked_build(void) { return SEPW_CHECKED ? 1 : 0; }

int sepw_test_corrupt_plan(sepw_ctx *ctx, int which, int64_t slot, int32_t value)
{
    if (!SEPW_CHECKED)
        return SEPW_ENOTSUP;  // nothing in the default build guards such a value
    if (!ctx)
        return SEPW_EINVAL;
    const Plan &pl = ctx->plan;
    if (!pl.valid || pl.form == SEPW_FORM_PLAIN || is_tc_form(pl.form))
        return fail(ctx, SEPW_ENOPLAN, "no tiled plan");
    if (slot < 0 || slot >= pl.nvis || (which != 0 && which != 1))
        return fail(ctx, SEPW_EINVAL, "slot %lld or which %d out of range", (long long)slot,
                    which);
    cudaError_t e;
    if (which == 0) {
        e = cudaMemcpy(pl.d_perm + slot, &value, sizeof(int32_t), cudaMemcpyHostToDevice);
    } else {
        uint64_t r = 0;
        e = cudaMemcpy(&r, pl.d_rec + slot, sizeof(r), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) {
            r = (r & ~((uint64_t)32767 << 28)) | ((uint64_t)(value & 32767) << 28);
            e = cudaMemcpy(pl.d_rec + slot, &r, sizeof(r), cudaMemcpyHostToDevice);
        }
    }
    return e == cudaSuccess ? SEPW_OK : cuda_fail(ctx, e, "sepw_test_corrupt_plan");
}

int sepw_test_stall_mma(sepw_ctx *ctx, int enable)
{
    if (!ctx)
        return SEPW_EINVAL;
    ctx->tc_ctl.stall = enable ? 1 : 0;
    return SEPW_OK;
}

int sepw_image(sepw_ctx *ctx, int direction, float *buf, sepw_stream_t stream)
{
    Range range_("sepw_image");
    if (!ctx)
        return SEPW_EINVAL;
    if (direction != SEPW_GRID_TO_IMAGE && direction != SEPW_IMAGE_TO_GRID &&
        direction != SEPW_IMAGE_TO_GRID_ADJOINT)
        return fail(ctx, SEPW_EINVAL, "bad direction %d", direction);
    int rc = check_dev(ctx, buf, "buf", false);
    if (rc)
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (!ctx->fft_ready) {
        cufftResult r = cufftPlan2d(&ctx->fft, ctx->p.grid_size, ctx->p.grid_size, CUFFT_C2C);
        if (r != CUFFT_SUCCESS)
            return fail(ctx, SEPW_ECUDA, "cufftPlan2d failed (%d)", (int)r);
        ctx->fft_ready = true;
    }
    if (cufftSetStream(ctx->fft, s) != CUFFT_SUCCESS)
        return fail(ctx, SEPW_ECUDA, "cufftSetStream failed");
    SEPW_CUDA(ctx, launch_image_pre(ctx->dp, direction, ctx->d_taper32, (float2 *)buf, s));
    cufftResult r = cufftExecC2C(ctx->fft, (cufftComplex *)buf, (cufftComplex *)buf,
                                 direction == SEPW_IMAGE_TO_GRID ? CUFFT_FORWARD
                                                                 : CUFFT_INVERSE);
    if (r != CUFFT_SUCCESS)
        return fail(ctx, SEPW_ECUDA, "cufftExecC2C failed (%d)", (int)r);
    SEPW_CUDA(ctx, launch_image_post(ctx->dp, direction, ctx->d_taper32, (float2 *)buf, s));
    return SEPW_OK;
}

int sepw_taper(sepw_ctx *ctx, float *taper, sepw_stream_t stream)
{
    if (!ctx)
        return SEPW_EINVAL;
    int rc = check_dev(ctx, taper, "taper", false);
    if (rc)
        return rc;
    SEPW_CUDA(ctx, cudaMemcpyAsync(taper, ctx->d_taper32, sizeof(float) * ctx->p.grid_size,
                                   cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return SEPW_OK;
}

static bool residual_sizes_ok(const sepw_params *p, int32_t Sr, int32_t OSr)
{
    return Sr >= 1 && Sr <= p->support && (p->support - Sr) % 2 == 0 && OSr >= 1 &&
           p->oversample % OSr == 0;
}

size_t sepw_residual_count(const sepw_params *p, int32_t support_r, int32_t oversample_r)
{
    if (!p || sepw_check_params(p) != SEPW_OK || !residual_sizes_ok(p, support_r, oversample_r))
        return 0;
    return (size_t)p->n_wplanes * oversample_r * oversample_r * support_r * support_r;
}

static int make_residual(sepw_ctx *ctx, int32_t Sr, int32_t OSr, double2 *out64,
                         float2 *out32, cudaStream_t s)
{
    if (!residual_sizes_ok(&ctx->p, Sr, OSr))
        return fail(ctx, SEPW_EINVAL, "need 1 <= support_r <= S, S - support_r even, "
                                      "oversample_r dividing OS");
    if (ctx->dp.facet)
        return fail(ctx, SEPW_ENOTSUP, "correction table not available in facet mode");
    const DevParams &p = ctx->dp;
    double2 *X = nullptr, *t64 = nullptr;
    const size_t nx = (size_t)p.P * OSr * Sr * p.N, nt = (size_t)p.P * p.OS * p.S;
    int rc;
    if ((rc = grow(ctx, &X, nx)) || (rc = grow(ctx, &t64, nt))) {
        cudaFree(X);
        cudaFree(t64);
        return rc;
    }
    cudaError_t e = launch_taps(p, ctx->d_taper64, ctx->d_tw, t64, nullptr, s);
    if (e == cudaSuccess)
        e = launch_residual_table(p, Sr, OSr, ctx->d_taper64, ctx->d_tw, t64, X, out64, out32,
                                  s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    cudaFree(X);
    cudaFree(t64);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "correction table");
    return SEPW_OK;
}

int sepw_make_residual(sepw_ctx *ctx, int32_t support_r, int32_t oversample_r, float *table,
                       sepw_stream_t stream)
{
    if (!ctx)
        return SEPW_EINVAL;
    int rc = check_dev(ctx, table, "table", false);
    if (rc)
        return rc;
    return make_residual(ctx, support_r, oversample_r, nullptr, (float2 *)table,
                         (cudaStream_t)stream);
}

int sepw_make_residual_f64(sepw_ctx *ctx, int32_t support_r, int32_t oversample_r,
                           double *table, sepw_stream_t stream)
{
    if (!ctx)
        return SEPW_EINVAL;
    int rc = check_dev(ctx, table, "table", false);
    if (rc)
        return rc;
    return make_residual(ctx, support_r, oversample_r, (double2 *)table, nullptr,
                         (cudaStream_t)stream);
}

static int residual_pass_check(sepw_ctx *ctx, int32_t Sr, int32_t OSr, const float *table)
{
    if (!ctx->plan.valid)
        return fail(ctx, SEPW_ENOPLAN, "no plan");
    if (ctx->plan.form == SEPW_FORM_PLAIN)
        return fail(ctx, SEPW_ENOTSUP, "the correction pass needs a tiled or tensor-core plan");
    if (!residual_sizes_ok(&ctx->p, Sr, OSr))
        return fail(ctx, SEPW_EINVAL, "need 1 <= support_r <= S, S - support_r even, "
                                      "oversample_r dividing OS");
    return check_dev(ctx, table, "table", false);
}

int sepw_grid_residual_planned(sepw_ctx *ctx, int32_t support_r, int32_t oversample_r,
                               const float *table, const float *vis, const float *weight,
                               float *grid, sepw_stream_t stream)
{
    Range range_("sepw_grid_residual");
    if (!ctx)
        return SEPW_EINVAL;
    int rc;
    if ((rc = residual_pass_check(ctx, support_r, oversample_r, table)) ||
        (rc = check_dev(ctx, grid, "grid", false)))
        return rc;
    if (ctx->plan.nvis == 0)
        return SEPW_OK;
    if ((rc = check_dev(ctx, vis, "vis", false)) || (rc = check_dev(ctx, weight, "weight", true)))
        return rc;
    SEPW_CUDA(ctx, launch_grid_residual(ctx->dp, support_r, oversample_r, ctx->plan,
                                        (const float2 *)vis, weight, (const float2 *)table,
                                        (float2 *)grid, ctx->num_sms, (cudaStream_t)stream));
    return SEPW_OK;
}

int sepw_degrid_residual_planned(sepw_ctx *ctx, int32_t support_r, int32_t oversample_r,
                                 const float *table, const float *grid, const float *weight,
                                 float *vis_out, sepw_stream_t stream)
{
    Range range_("sepw_degrid_residual");
    if (!ctx)
        return SEPW_EINVAL;
    int rc;
    if ((rc = residual_pass_check(ctx, support_r, oversample_r, table)) ||
        (rc = check_dev(ctx, grid, "grid", false)))
        return rc;
    if (ctx->plan.nvis == 0)
        return SEPW_OK;
    if ((rc = check_dev(ctx, vis_out, "vis_out", false)) ||
        (rc = check_dev(ctx, weight, "weight", true)))
        return rc;
    SEPW_CUDA(ctx, launch_degrid_residual(ctx->dp, support_r, oversample_r, ctx->plan,
                                          (const float2 *)grid, weight, (const float2 *)table,
                                          (float2 *)vis_out, ctx->num_sms,
                                          (cudaStream_t)stream));
    return SEPW_OK;
}

int sepw_set_facet(sepw_ctx *ctx, int enable, double l0, double m0)
{
    if (!ctx)
        return SEPW_EINVAL;
    if (!enable) {
        ctx->dp.facet = 0;
        ctx->dp.voff = 0;
        ctx->dp.l0 = ctx->dp.m0 = 0.0;
        ctx->dp.a2u = ctx->dp.a2v = -0.5;
        return SEPW_OK;
    }
    if (!isfinite(l0) || !isfinite(m0) || !(l0 * l0 + m0 * m0 < 1.0))
        return fail(ctx, SEPW_EINVAL, "facet centre (%g, %g) not inside the unit circle", l0,
                    m0);
    const double n0 = sqrt(1.0 - l0 * l0 - m0 * m0);
    ctx->dp.facet = 1;
    ctx->dp.voff = (int64_t)ctx->p.n_wplanes * ctx->p.oversample * ctx->p.support;
    ctx->dp.l0 = l0;
    ctx->dp.m0 = m0;
    ctx->dp.a2u = -0.5 * (1.0 / n0 + l0 * l0 / (n0 * n0 * n0));
    ctx->dp.a2v = -0.5 * (1.0 / n0 + m0 * m0 / (n0 * n0 * n0));
    return SEPW_OK;
}

int sepw_facet_shift(sepw_ctx *ctx, int direction, int64_t nvis, const double *u,
                     const double *v, const double *w, const float *vis, double *u_out,
                     double *v_out, float *vis_out, sepw_stream_t stream)
{
    if (!ctx)
        return SEPW_EINVAL;
    if (!ctx->dp.facet)
        return fail(ctx, SEPW_ENOTSUP, "context not in facet mode");
    if (direction != SEPW_FACET_IN && direction != SEPW_FACET_OUT)
        return fail(ctx, SEPW_EINVAL, "bad facet direction %d", direction);
    if (nvis < 0)
        return fail(ctx, SEPW_EINVAL, "nvis < 0");
    if (nvis == 0)
        return SEPW_OK;
    if ((u_out == nullptr) != (v_out == nullptr))
        return fail(ctx, SEPW_EINVAL, "u_out and v_out must both be given or both NULL");
    if ((vis == nullptr) != (vis_out == nullptr))
        return fail(ctx, SEPW_EINVAL, "vis and vis_out must both be given or both NULL");
    int rc;
    if ((rc = check_dev(ctx, u, "u", false)) || (rc = check_dev(ctx, v, "v", false)) ||
        (rc = check_dev(ctx, w, "w", false)) || (rc = check_dev(ctx, vis, "vis", true)) ||
        (rc = check_dev(ctx, vis_out, "vis_out", true)) ||
        (rc = check_dev(ctx, u_out, "u_out", true)) ||
        (rc = check_dev(ctx, v_out, "v_out", true)))
        return rc;
    SEPW_CUDA(ctx, launch_facet_shift(nvis, ctx->dp.l0, ctx->dp.m0, direction, u, v, w,
                                      (const float2 *)vis, u_out, v_out, (float2 *)vis_out,
                                      (cudaStream_t)stream));
    return SEPW_OK;
}

int sepw_wstack_plan(sepw_ctx *ctx, int32_t nslices, const double *w_centres, int64_t nvis,
                     const double *u, const double *v, const double *w, int32_t *slice_out,
                     sepw_stream_t stream)
{
    Range range_("sepw_wstack_plan");
    if (!ctx)
        return SEPW_EINVAL;
    ctx->ws_centres.clear();
    ctx->plan.valid = false;
    if (ctx->p.form == SEPW_FORM_PLAIN)
        return fail(ctx, SEPW_ENOTSUP, "W stacking needs a tiled or tensor-core form");
    if (nslices < 1 || !w_centres)
        return fail(ctx, SEPW_EINVAL, "nslices < 1 or w_centres NULL");
    for (int c = 0; c < nslices; ++c) {
        if (!isfinite(w_centres[c]))
            return fail(ctx, SEPW_EINVAL, "w_centres[%d] not finite", c);
        if (c > 0 && !(w_centres[c] > w_centres[c - 1]))
            return fail(ctx, SEPW_EINVAL, "w_centres not strictly increasing at %d", c);
    }
    if (nvis < 0 || nvis > (int64_t)INT32_MAX - 1)
        return fail(ctx, SEPW_EINVAL, "nvis out of range [0, 2^31 - 2]");
    int rc;
    if (nvis > 0 && ((rc = check_dev(ctx, u, "u", false)) || (rc = check_dev(ctx, v, "v", false)) ||
                     (rc = check_dev(ctx, w, "w", false)) ||
                     (slice_out && (rc = check_dev(ctx, slice_out, "slice_out", false)))))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (nslices > ctx->ws_centres_cap) {
        if ((rc = grow(ctx, &ctx->d_ws_c64, (size_t)nslices)) ||
            (rc = grow(ctx, &ctx->d_ws_c32, (size_t)nslices)) ||
            (rc = grow(ctx, &ctx->d_ws_count, (size_t)nslices)))
            return rc;
        ctx->ws_centres_cap = nslices;
    }
    if (nvis > ctx->ws_cap) {
        const size_t cap = (size_t)nvis + nvis / 8;
        if ((rc = grow(ctx, &ctx->d_ws_slice, cap)) || (rc = grow(ctx, &ctx->d_ws_part, cap)) ||
            (rc = grow(ctx, &ctx->d_ws_u, cap)) || (rc = grow(ctx, &ctx->d_ws_v, cap)) ||
            (rc = grow(ctx, &ctx->d_ws_w, cap)))
            return rc;
        ctx->ws_cap = (int64_t)cap;
    }
    std::vector<float> c32(w_centres, w_centres + nslices);
    SEPW_CUDA(ctx, cudaMemcpyAsync(ctx->d_ws_c64, w_centres, sizeof(double) * nslices,
                                   cudaMemcpyHostToDevice, s));
    SEPW_CUDA(ctx, cudaMemcpyAsync(ctx->d_ws_c32, c32.data(), sizeof(float) * nslices,
                                   cudaMemcpyHostToDevice, s));
    SEPW_CUDA(ctx, cudaMemsetAsync(ctx->d_ws_count, 0, sizeof(int32_t) * nslices, s));
    int32_t *slice = slice_out ? slice_out : ctx->d_ws_slice;
    SEPW_CUDA(ctx, launch_wstack_assign(nvis, w, ctx->d_ws_c64, nslices, slice, ctx->d_ws_count, s));
    std::vector<int32_t> cnt(nslices);
    SEPW_CUDA(ctx, cudaMemcpyAsync(cnt.data(), ctx->d_ws_count, sizeof(int32_t) * nslices,
                                   cudaMemcpyDeviceToHost, s));
    SEPW_CUDA(ctx, cudaStreamSynchronize(s));
    std::vector<int64_t> off(nslices + 1, 0);
    std::vector<int32_t> cur(nslices);
    for (int c = 0; c < nslices; ++c) {
        cur[c] = (int32_t)off[c];
        off[c + 1] = off[c] + cnt[c];
    }
    SEPW_CUDA(ctx, cudaMemcpyAsync(ctx->d_ws_count, cur.data(), sizeof(int32_t) * nslices,
                                   cudaMemcpyHostToDevice, s));
    SEPW_CUDA(ctx, launch_wstack_scatter(nvis, u, v, w, ctx->d_ws_c64, nslices, slice,
                                         ctx->d_ws_count,
                                         ctx->d_ws_part, ctx->d_ws_u, ctx->d_ws_v, ctx->d_ws_w,
                                         s));
    if ((rc = plan_impl(ctx, nslices, off.data(), nvis, ctx->d_ws_u, ctx->d_ws_v, ctx->d_ws_w,
                        s)))
        return rc;
    SEPW_CUDA(ctx, launch_wstack_compose(nvis, ctx->plan, ctx->d_ws_part, s));
    // the host copies above must outlive the asynchronous transfers
    SEPW_CUDA(ctx, cudaStreamSynchronize(s));
    ctx->ws_centres.assign(w_centres, w_centres + nslices);
    return SEPW_OK;
}

static int ensure_fft_batch(sepw_ctx *ctx, int L)
{
    if (ctx->fft_batch_n == L)
        return SEPW_OK;
    if (ctx->fft_batch_n)
        cufftDestroy(ctx->fft_batch);
    ctx->fft_batch_n = 0;
    int n[2] = {ctx->p.grid_size, ctx->p.grid_size};
    const int dist = ctx->p.grid_size * ctx->p.grid_size;
    cufftResult r = cufftPlanMany(&ctx->fft_batch, 2, n, nullptr, 1, dist, nullptr, 1, dist,
                                  CUFFT_C2C, L);
    if (r != CUFFT_SUCCESS)
        return fail(ctx, SEPW_ECUDA, "cufftPlanMany (%d slices) failed (%d)", L, (int)r);
    ctx->fft_batch_n = L;
    return SEPW_OK;
}

int sepw_wstack_image(sepw_ctx *ctx, float *slice_grids, float *image, sepw_stream_t stream)
{
    Range range_("sepw_wstack_image");
    if (!ctx)
        return SEPW_EINVAL;
    if (ctx->ws_centres.empty())
        return fail(ctx, SEPW_ENOPLAN, "no W-stacking plan");
    int rc;
    if ((rc = check_dev(ctx, slice_grids, "slice_grids", false)) ||
        (rc = check_dev(ctx, image, "image", false)))
        return rc;
    const int L = (int)ctx->ws_centres.size();
    if ((rc = ensure_fft_batch(ctx, L)))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (cufftSetStream(ctx->fft_batch, s) != CUFFT_SUCCESS)
        return fail(ctx, SEPW_ECUDA, "cufftSetStream failed");
    SEPW_CUDA(ctx, launch_wstack_sign(ctx->dp, L, (float2 *)slice_grids, s));
    cufftResult r = cufftExecC2C(ctx->fft_batch, (cufftComplex *)slice_grids,
                                 (cufftComplex *)slice_grids, CUFFT_INVERSE);
    if (r != CUFFT_SUCCESS)
        return fail(ctx, SEPW_ECUDA, "cufftExecC2C failed (%d)", (int)r);
    SEPW_CUDA(ctx, launch_wstack_combine(ctx->dp, L, ctx->d_taper32, ctx->d_ws_c32,
                                         (const float2 *)slice_grids, (float2 *)image, s));
    return SEPW_OK;
}

int sepw_wstack_model_grids(sepw_ctx *ctx, const float *image, float *slice_grids,
                            sepw_stream_t stream)
{
    Range range_("sepw_wstack_model_grids");
    if (!ctx)
        return SEPW_EINVAL;
    if (ctx->ws_centres.empty())
        return fail(ctx, SEPW_ENOPLAN, "no W-stacking plan");
    int rc;
    if ((rc = check_dev(ctx, slice_grids, "slice_grids", false)) ||
        (rc = check_dev(ctx, image, "image", false)))
        return rc;
    const int L = (int)ctx->ws_centres.size();
    if ((rc = ensure_fft_batch(ctx, L)))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (cufftSetStream(ctx->fft_batch, s) != CUFFT_SUCCESS)
        return fail(ctx, SEPW_ECUDA, "cufftSetStream failed");
    SEPW_CUDA(ctx, launch_wstack_split(ctx->dp, L, ctx->d_taper32, ctx->d_ws_c32,
                                       (const float2 *)image, (float2 *)slice_grids, s));
    cufftResult r = cufftExecC2C(ctx->fft_batch, (cufftComplex *)slice_grids,
                                 (cufftComplex *)slice_grids, CUFFT_FORWARD);
    if (r != CUFFT_SUCCESS)
        return fail(ctx, SEPW_ECUDA, "cufftExecC2C failed (%d)", (int)r);
    SEPW_CUDA(ctx, launch_wstack_sign(ctx->dp, L, (float2 *)slice_grids, s));
    return SEPW_OK;
}

}  // extern "C"
