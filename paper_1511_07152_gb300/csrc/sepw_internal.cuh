// Internal declarations shared by the CUDA translation units of libsepw.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/sepw.h"

namespace sepw {

// Device-side copy of the parameters plus derived constants.  Passed by
// value to every kernel.
struct DevParams {
    int32_t N, S, OS, P, T;
    int32_t ntx;      // tiles per axis for the tiled forms
    uint32_t t_inv;   // ceil(2^32 / T), see div_tile
    double fov;       // inverse cell size: x = u * fov + N/2
    double half;      // N/2 as a double
    double os_d;      // OS as a double
    int32_t os_log2;  // log2(OS) if OS is a power of two, else -1
    int32_t fast_elim;  // locate_axis: exponent bound of its integer path (-1: off)
    int32_t fast_near;  // locate_axis: its fall-back margin, in units of 2^-40
    double plane_r;   // (P-1)/w_max (0 if P == 1)
    double w_max;
    double gamma;
    double beta;
    // image-plane faceting (Sec. 4.1): the v-direction taps sit voff elements
    // after the u-direction ones (0: one table for both); the image step takes
    // n at the facet's pixels (l0 + l, m0 + m); the facet tables use the
    // screens exp(2 pi i w a2 l^2) with a2 = a2u (u table), a2v (v table)
    int64_t voff = 0;
    int32_t facet = 0;
    // schedule of the tiled and tensor-core plans (sepw_set_schedule):
    // visibilities per work item (<= kChunk) and the parts a block-gridder
    // warp unit takes of an item (0: by the plan's density)
    int32_t chunk = 2048;
    int32_t grid_parts = 0;
    double l0 = 0.0, m0 = 0.0;
    double a2u = -0.5, a2v = -0.5;
    // bounds of the current plan, read only by the checked build's checks
    // (work_item_ok, record_ok): the status word they report into, the
    // plan's visibility slots and its tile count over all grids
    int32_t *chk_status = nullptr;
    int64_t chk_nvis = 0;
    int64_t chk_tiles = 0;
};

// Result of locating one visibility.
struct Loc {
    int32_t cu, cv, ou, ov, plane;
    bool conj;
    bool keep;
};

// floor(fl(x + 0.5)), the IEEE sum rounded to nearest then floored, computed
// exactly from the bits of x without an FP64 add.  For |x| < 2^52 the sum
// x + 0.5 either is representable or rounds only within [2^k, 2^k + 1) for an
// integer power of two 2^k, which leaves its floor unchanged; the one
// exception is x = 0.5 - 2^-54, whose sum 1 - 2^-54 is a tie that rounds to
// 1.0.  So the result is floor(x + 1/2) of the exact real sum, except there.
// Returns false for NaN, +-inf and |x| >= 2^52 (outside the accepted range).
__device__ __forceinline__ bool floor_add_half_bits(double x, long long &out)
{
    const long long b = __double_as_longlong(x);
    const int eb = (int)((b >> 52) & 0x7FF);
    if (eb >= 1023 + 52)
        return false;
    if (eb < 1022) {  // |x| < 1/2: the sum lies in (0, 1)
        out = (b == 0x3FDFFFFFFFFFFFFFll) ? 1 : 0;
        return true;
    }
    const int shift = 52 - (eb - 1023);  // 1..53
    const long long mant = (b & 0x000FFFFFFFFFFFFFll) | 0x0010000000000000ll;
    const long long num = (b < 0 ? -mant : mant) + (1ll << (shift - 1));
    out = num >> shift;  // arithmetic shift: floor division by 2^shift
    return true;
}

// x * 2^k, exact: exponent add when x is normal and stays normal, IEEE
// multiply otherwise (zero, subnormal, overflow; all rounded identically).
__device__ __forceinline__ double scale_pow2(double x, int k, double os_d)
{
    const long long b = __double_as_longlong(x);
    const int eb = (int)((b >> 52) & 0x7FF);
    if (eb >= 1 && eb + k <= 2046)
        return __longlong_as_double(b + ((long long)k << 52));
    return __dmul_rn(x, os_d);
}

// Locate one axis: x = coord*fov + N/2, t = floor(x*OS + 0.5) in IEEE double
// with every operation rounded separately (no FMA contraction), then
// c = floor(t/OS), o = t - c*OS; the footprint c - S/2 + 1 .. c + S/2 must lie
// inside [0, N).  Returns false (drop) otherwise or for non-finite input.
// Only u*fov uses the FP64 pipe on the common path (+ N/2 only within the
// fall-back margin below); the power-of-two scaling, the rounded + 0.5 with
// its floor, and the range checks are exact integer operations on the bits.
//
// Integer path (OS a power of two): with y = fl(coord*fov) the IEEE product,
// t = floor(fl(y + N/2) OS + 1/2).  The exact value floor((y + N/2) OS + 1/2)
// = (N/2) OS + floor(y OS + 1/2) follows from the bits of y (y OS is exact),
// and differs from t only if fl(y + N/2) moves (y + N/2) OS + 1/2 across an
// integer: fl rounds by at most half an ulp of a sum below N, so that needs
// y OS + 1/2 within N OS 2^-53 of an integer.  Those cases (and |y OS| at or
// beyond 2^fast_elim, which bounds the sum and the fixed-point range) take
// the FP64 path below.
__device__ __forceinline__ bool locate_axis_int(double y, const DevParams &p, long long &ti,
                                                bool &done)
{
    done = false;
    const long long b = __double_as_longlong(y);
    const int eb = (int)((b >> 52) & 0x7FF);
    if (eb == 0x7FF)
        return false;  // non-finite
    long long z;       // floor((y OS + 1/2) 2^40), then split
    if (eb == 0) {
        z = (b < 0 ? -1ll : 0ll) + (1ll << 39);  // zero or subnormal: |y OS| < 2^-40
    } else {
        const int ey = eb - 1023 + p.os_log2;  // exponent of y OS
        if (ey >= p.fast_elim)
            return true;  // FP64 path
        const long long m = (b & 0x000FFFFFFFFFFFFFll) | 0x0010000000000000ll;
        const int sh = ey - 12;  // y OS 2^40 = m 2^(ey - 12)
        long long a;
        if (sh >= 0) {
            a = m << sh;  // ey < fast_elim <= 21: below 2^62
            a = b < 0 ? -a : a;
        } else if (sh > -53) {
            const long long q = m >> (-sh);
            const bool rem = (m & ((1ll << (-sh)) - 1)) != 0;
            a = b < 0 ? -q - (rem ? 1 : 0) : q;  // floor
        } else {
            a = b < 0 ? -1 : 0;
        }
        z = a + (1ll << 39);
    }
    const long long fr = z & ((1ll << 40) - 1);
    if (fr <= p.fast_near || fr >= (1ll << 40) - p.fast_near)
        return true;  // within the rounding margin of an integer: FP64 path
    ti = ((long long)(p.N / 2) << p.os_log2) + (z >> 40);
    done = true;
    return true;
}

__device__ __forceinline__ bool locate_axis(double coord, const DevParams &p,
                                            int32_t &c, int32_t &o)
{
    const double y = __dmul_rn(coord, p.fov);
    long long ti, cc, oo;
    bool done = false;
    if (p.fast_elim >= 0 && !locate_axis_int(y, p, ti, done))
        return false;
    if (done) {
        cc = ti >> p.os_log2;
        oo = ti - (cc << p.os_log2);
        const long long f = cc - p.S / 2 + 1;
        if (f < 0 || f + p.S - 1 > p.N - 1)
            return false;
        c = (int32_t)cc;
        o = (int32_t)oo;
        return true;
    }
    const double x = __dadd_rn(y, p.half);
    if (p.os_log2 >= 0) {
        if (!floor_add_half_bits(scale_pow2(x, p.os_log2, p.os_d), ti))
            return false;
        if (ti >= 1099511627776ll || ti <= -1099511627776ll)  // |t| < 2^40
            return false;
        cc = ti >> p.os_log2;  // floor division by OS = 2^k
        oo = ti - (cc << p.os_log2);
    } else {
        if (!floor_add_half_bits(__dmul_rn(x, p.os_d), ti))
            return false;
        if (ti >= 1099511627776ll || ti <= -1099511627776ll)
            return false;
        const long long OS = p.OS;
        cc = ti >= 0 ? ti / OS : -((-ti + OS - 1) / OS);
        oo = ti - cc * OS;
    }
    const long long f = cc - p.S / 2 + 1;
    if (f < 0 || f + p.S - 1 > p.N - 1)
        return false;
    c = (int32_t)cc;
    o = (int32_t)oo;
    return true;
}

// Plane: floor(|w| * r + 0.5) with r = (P-1)/w_max, dropped beyond P-1 or if
// not finite; conj = (w < 0).
__device__ __forceinline__ Loc locate(double u, double v, double w, const DevParams &p)
{
    Loc L;
    L.cu = L.cv = L.ou = L.ov = L.plane = 0;
    L.conj = false;
    int32_t cu, cv, ou, ov;
    bool ok = locate_axis(u, p, cu, ou);
    ok = locate_axis(v, p, cv, ov) && ok;
    const long long wb = __double_as_longlong(w);
    const double aw = __longlong_as_double(wb & 0x7FFFFFFFFFFFFFFFll);
    long long q;
    const bool wfin = ((wb >> 52) & 0x7FF) != 0x7FF;
    ok = ok && wfin && floor_add_half_bits(__dmul_rn(aw, p.plane_r), q) &&
         q <= (long long)(p.P - 1);
    L.keep = ok;
    if (ok) {
        L.cu = cu;
        L.cv = cv;
        L.ou = ou;
        L.ov = ov;
        L.plane = (int32_t)q;
        L.conj = wb < 0 && (wb & 0x7FFFFFFFFFFFFFFFll) != 0;
    }
    return L;
}

// Tile id -> origin of the tile in its grid.  A batched plan numbers the
// tiles of grid g after those of grids 0 .. g-1 (ntx^2 tiles per grid), so the
// grid's base offset follows from the tile id as well.
struct TileOrigin {
    int64_t base;  // element offset of the tile's grid
    int64_t gy0;   // first row of the tile
    int64_t gx0;   // first column of the tile
};
__device__ __forceinline__ TileOrigin tile_origin(const DevParams &p, int tile)
{
    const int per = p.ntx * p.ntx;
    const int g = tile / per;
    const int tl = tile - g * per;
    const int ty = tl / p.ntx, tx = tl - ty * p.ntx;
    TileOrigin o;
    o.base = (int64_t)g * p.N * p.N;
    o.gy0 = (int64_t)ty * p.T;
    o.gx0 = (int64_t)tx * p.T;
    return o;
}

// Packed per-visibility record of a plan (tiled forms), in slot order:
//   bits  0..5   lx  footprint origin column inside the tile (0..T-1)
//   bits  6..11  ly  footprint origin row inside the tile
//   bits 12..19  ou
//   bits 20..27  ov
//   bits 28..42  plane
//   bit  43      conj
__host__ __device__ __forceinline__ uint64_t pack_rec(int lx, int ly, int ou, int ov,
                                                      int plane, bool conj)
{
    return (uint64_t)lx | ((uint64_t)ly << 6) | ((uint64_t)ou << 12) |
           ((uint64_t)ov << 20) | ((uint64_t)plane << 28) | ((uint64_t)conj << 43);
}
__host__ __device__ __forceinline__ int rec_lx(uint64_t r) { return (int)(r & 63); }
__host__ __device__ __forceinline__ int rec_ly(uint64_t r) { return (int)((r >> 6) & 63); }
__host__ __device__ __forceinline__ int rec_ou(uint64_t r) { return (int)((r >> 12) & 255); }
__host__ __device__ __forceinline__ int rec_ov(uint64_t r) { return (int)((r >> 20) & 255); }
__host__ __device__ __forceinline__ int rec_plane(uint64_t r) { return (int)((r >> 28) & 32767); }
__host__ __device__ __forceinline__ bool rec_conj(uint64_t r) { return (r >> 43) & 1; }

// One work item of the tiled kernels: a chunk of at most kChunk visibilities
// of one tile, stored contiguously in slot order.
struct WorkItem {
    int32_t tile;
    int32_t start;  // first slot
    int32_t count;  // number of slots
    int32_t pad;
};

// Checked build (nvcc -DSEPW_CHECKED=1, libsepw_checked.so): the scatter-
// form kernels check each work item and each plan record against the plan's
// bounds before use; a failed check records SEPW_EBOUNDS in the context's
// status word and the kernel skips the item or visibility.  The default build
// compiles every check to `true`.
#ifndef SEPW_CHECKED
#define SEPW_CHECKED 0
#endif

__device__ __forceinline__ bool check_ok(const DevParams &p, bool ok)
{
#if SEPW_CHECKED
    if (!ok && p.chk_status)
        atomicExch(p.chk_status, SEPW_EBOUNDS);
    return ok;
#else
    (void)p;
    (void)ok;
    return true;
#endif
}

// the item's tile and slot range lie inside the plan
__device__ __forceinline__ bool work_item_ok(const DevParams &p, const WorkItem &it)
{
    return check_ok(p, it.tile >= 0 && it.tile < p.chk_tiles && it.start >= 0 &&
                           it.count >= 0 && (int64_t)it.start + it.count <= p.chk_nvis);
}

// the slot's visibility index, table rows and footprint (inside the tile's
// window and the grid, the tile at grid origin (gy0, gx0)) are in range
__device__ __forceinline__ bool record_ok(const DevParams &p, uint64_t r, int i, int64_t gy0,
                                          int64_t gx0)
{
    return check_ok(p, i >= 0 && i < p.chk_nvis && rec_plane(r) < p.P && rec_ou(r) < p.OS &&
                           rec_ov(r) < p.OS && rec_lx(r) < p.T && rec_ly(r) < p.T &&
                           gx0 + rec_lx(r) + p.S <= p.N && gy0 + rec_ly(r) + p.S <= p.N);
}

constexpr int kChunk = 2048;      // largest work item (visibilities), the default
constexpr int kMaxWindow = 64;    // T + S - 1 <= kMaxWindow

// Plan workspace (owned by the context).
// Binning below the tile: each tile's visibilities are grouped by the 4 x 4
// sub-block of the tile that holds their footprint origin and by conj, 32
// bins per tile, before the tile is cut into work items.  An item then spans
// few sub-blocks, so after the per-item sort its runs of one origin are long
// (one register block accumulates a whole run).
constexpr int kSubBins = 32;

// ceil(2^32 / T) for the tile edge T (8 <= T <= 64)
// Bounds of locate_axis's integer path for grid size N and OS = 2^os_log2
// (os_log2 < 0: path off): |y OS| < 2^elim with 2^elim <= N OS / 2 and
// elim <= 21; margin (N OS) 2^-53 in units of 2^-40, rounded up, plus 2.
inline void locate_fast_bounds(int N, int os_log2, int32_t &elim, int32_t &near)
{
    elim = -1;
    near = 0;
    if (os_log2 < 0)
        return;
    const long long half_span = ((long long)N << os_log2) / 2;  // N OS / 2
    int e = 0;
    while (e < 21 && (1ll << (e + 1)) <= half_span)
        ++e;
    elim = (1ll << e) <= half_span ? e : -1;
    near = (int32_t)((((long long)N << os_log2) >> 13) + 2);
}

inline uint32_t tile_reciprocal(int T)
{
    return (uint32_t)((0x100000000ull + (uint64_t)T - 1) / (uint64_t)T);
}

// floor(n / T) for 0 <= n < 2^26 as one multiply-high.  With
// M = ceil(2^32 / T) = (2^32 + e) / T, 0 <= e < T, and n = q T + r
// (0 <= r <= T - 1): n M / 2^32 = q + (r + n e / 2^32) / T, whose fraction
// stays below 1 while n e < 2^32, true for n < 2^26 and T <= 64.
__device__ __forceinline__ int div_tile(int n, const DevParams &p)
{
    return (int)__umulhi((unsigned)n, p.t_inv);
}

// column-major: the eight bins of one column of sub-blocks are consecutive
__device__ __forceinline__ int sub_bin(int lx, int ly, bool conj, const DevParams &p)
{
    return ((div_tile(lx * 4, p) * 4 + div_tile(ly * 4, p)) << 1) | (conj ? 1 : 0);
}

struct Plan {
    int64_t nvis = 0;
    int64_t capacity = 0;       // allocated visibility slots
    int32_t ntiles = 0;
    int32_t tiles_capacity = 0;
    int32_t items_capacity = 0;
    bool valid = false;
    int form = 0;
    // tiled forms
    int32_t *d_tile = nullptr;      // [nvis] bin id per visibility (-1 dropped)
    int32_t *d_rank = nullptr;      // [nvis] rank of the visibility inside its bin
    int32_t *d_bin = nullptr;       // [ntiles * kSubBins] bin counts, then cursors
    uint64_t *d_rec0 = nullptr;     // [nvis] record, input order
    uint64_t *d_rec = nullptr;      // [nvis] record, slot order
    int32_t *d_perm = nullptr;      // [nvis] slot -> visibility index
    int32_t *d_tile_count = nullptr;   // [ntiles]
    int32_t *d_tile_cursor = nullptr;  // [ntiles]
    WorkItem *d_items = nullptr;       // [items_capacity]
    int32_t *d_nitems = nullptr;       // [1]
    int32_t *d_item_counter = nullptr; // [2] persistent-kernel work counters
    unsigned long long *d_dropped = nullptr;  // [1]
    int32_t *d_drop_list = nullptr;           // [nvis] indices of dropped visibilities
    int32_t ngrids = 1;                // batched plans: grids in the batch
    int64_t *d_offsets = nullptr;      // [ngrids + 1] visibility offsets per grid
    int32_t offsets_capacity = 0;
    std::vector<int64_t> h_offsets;    // plain form: per-grid ranges
    // plain form: the coordinates are read directly
    const double *u = nullptr, *v = nullptr, *w = nullptr;
};

// Device-side parameters of a checked sepw_params (sepw_api.cu): derived
// constants, and the tile edge resolved for the form when p->tile is 0.
DevParams make_dev_params(const sepw_params *p);

// ---- launchers (each .cu file implements its own) -------------------------

// sepw_taps.cu
cudaError_t launch_taper(const DevParams &p, double *taper64, float *taper32,
                         cudaStream_t s);
cudaError_t launch_twiddles(const DevParams &p, double2 *tw, cudaStream_t s);
cudaError_t launch_taps(const DevParams &p, const double *taper64, const double2 *tw,
                        double2 *out64, float2 *out32, cudaStream_t s);

// sepw_plain.cu
cudaError_t launch_count_dropped(const DevParams &p, int64_t nvis, const double *u,
                                 const double *v, const double *w,
                                 unsigned long long *dropped, cudaStream_t s);
cudaError_t launch_locate(const DevParams &p, int64_t nvis, const double *u,
                          const double *v, const double *w, int32_t *cu, int32_t *cv,
                          int32_t *ou, int32_t *ov, int32_t *plane, uint8_t *conj,
                          uint8_t *keep, cudaStream_t s);
cudaError_t launch_grid_plain(const DevParams &p, int64_t nvis, const double *u,
                              const double *v, const double *w, const float2 *vis,
                              const float *weight, const float2 *taps, float2 *grid,
                              unsigned long long *dropped, cudaStream_t s);
cudaError_t launch_degrid_plain(const DevParams &p, int64_t nvis, const double *u,
                                const double *v, const double *w, const float2 *grid,
                                const float *weight, const float2 *taps, float2 *vis,
                                unsigned long long *dropped, cudaStream_t s);

// sepw_bin.cu
cudaError_t launch_plan(const DevParams &p, int64_t nvis, const double *u,
                        const double *v, const double *w, Plan &plan, cudaStream_t s);
// batched: plan.ngrids > 1 and plan.d_offsets hold the per-grid ranges
cudaError_t launch_zero_dropped(const Plan &plan, float2 *vis, cudaStream_t s);

// sepw_tiled.cu
// planar: workspace of 2 x (taps of both tables) floats for the lane-ordered
// planar copy of the tap table that the block gridder (S = 8, 16) builds and
// reads its v-taps from; null: the interleaved table is read directly
cudaError_t launch_grid_tiled(const DevParams &p, const Plan &plan, const float2 *vis,
                              const float *weight, const float2 *taps, float *planar,
                              float2 *grid, int num_sms, cudaStream_t s);
cudaError_t launch_degrid_tiled(const DevParams &p, const Plan &plan,
                                const float2 *grid, const float *weight,
                                const float2 *taps, float2 *vis, int num_sms,
                                cudaStream_t s);

// Control of the tensor-core kernels: the limit of every bounded mbarrier
// wait, and a test hook (stall != 0: the MMA thread issues and commits
// nothing, so the other roles' waits run out and the kernel reports
// SEPW_ETIMEOUT).
struct TcControl {
    unsigned long long wait_ns;
    int32_t stall;
};

// sepw_tc.cu: contraction-form degridder, prec 0 = BF16, 1 = FP16 (scaled
// per item), 2 = FP16 hi + lo (scaled), 3 = BF16 hi + lo; T + S - 1 <= 32,
// S <= 16.  tables: tc_degrid_tables_bytes(p,
// plan.items_capacity) bytes of device workspace for the per-call tap tables
// (the FP16 forms' per-item window scale is found in the kernel; the item
// count does not enter the size).
size_t tc_degrid_tables_bytes(const DevParams &p, int64_t items_capacity);
cudaError_t launch_degrid_tc(const DevParams &p, const Plan &plan, const float2 *grid,
                             const float *weight, const float2 *taps, void *tables, float2 *vis,
                             int num_sms, int prec, int32_t *status, TcControl ctl,
                             cudaStream_t s);

// sepw_tc_grid.cu: contraction-form gridder, T + S - 1 <= 32, S <= 16.
// prec: 0 = BF16, 1 = FP16 (scaled per item), 2 = FP16 hi + lo (scaled),
// 3 = BF16 hi + lo.  tables: tc2_tables_bytes(p, plan.items_capacity) bytes of
// device workspace for the per-call pre-shifted tap tables and the per-item
// scale exponents.
int tc2_tile_for_support(int S);
size_t tc2_tables_bytes(const DevParams &p, int64_t items_capacity);
cudaError_t launch_grid_tc2(const DevParams &p, const Plan &plan, const float2 *vis,
                            const float *weight, const float2 *taps, void *tables, float2 *grid,
                            int num_sms, int prec, int32_t *status, TcControl ctl,
                            cudaStream_t s);

// sepw_wstack.cu
cudaError_t launch_wstack_assign(int64_t nvis, const double *w, const double *c, int L,
                                 int32_t *slice, int32_t *count, cudaStream_t s);
cudaError_t launch_wstack_scatter(int64_t nvis, const double *u, const double *v,
                                  const double *w, const double *c, int L, const int32_t *slice,
                                  int32_t *cursor, int32_t *part, double *up, double *vp,
                                  double *wp, cudaStream_t s);
cudaError_t launch_wstack_compose(int64_t nvis, const Plan &plan, const int32_t *part,
                                  cudaStream_t s);
cudaError_t launch_wstack_sign(const DevParams &p, int L, float2 *g, cudaStream_t s);
cudaError_t launch_wstack_combine(const DevParams &p, int L, const float *taper,
                                  const float *wc, const float2 *g, float2 *image,
                                  cudaStream_t s);
cudaError_t launch_wstack_split(const DevParams &p, int L, const float *taper, const float *wc,
                                const float2 *image, float2 *g, cudaStream_t s);

// sepw_facet.cu (direction 0: into the facet, 1: back out)
cudaError_t launch_facet_shift(int64_t nvis, double l0, double m0, int direction,
                               const double *u, const double *v, const double *w,
                               const float2 *vin, double *uo, double *vo, float2 *vout,
                               cudaStream_t s);

// sepw_residual.cu (stored correction F_w - F~_w)
cudaError_t launch_residual_table(const DevParams &p, int Sr, int OSr, const double *taper64,
                                  const double2 *tw, const double2 *taps64, double2 *X,
                                  double2 *out64, float2 *out32, cudaStream_t s);
cudaError_t launch_grid_residual(const DevParams &p, int Sr, int OSr, const Plan &plan,
                                 const float2 *vis, const float *weight, const float2 *res,
                                 float2 *grid, int num_sms, cudaStream_t s);
cudaError_t launch_degrid_residual(const DevParams &p, int Sr, int OSr, const Plan &plan,
                                   const float2 *grid, const float *weight, const float2 *res,
                                   float2 *vis_out, int num_sms, cudaStream_t s);

// sepw_image.cu
cudaError_t launch_image_pre(const DevParams &p, int direction, const float *taper,
                             float2 *buf, cudaStream_t s);
cudaError_t launch_image_post(const DevParams &p, int direction, const float *taper,
                              float2 *buf, cudaStream_t s);

}  // namespace sepw
