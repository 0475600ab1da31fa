// Internal declarations shared by the CUDA translation units of libsepw.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sepw.h"

namespace sepw {

// Device-side copy of the parameters plus derived constants.  Passed by
// value to every kernel.
struct DevParams {
    int32_t N, S, OS, P, T;
    int32_t ntx;      // tiles per axis for the tiled forms
    double fov;       // inverse cell size: x = u * fov + N/2
    double half;      // N/2 as a double
    double os_d;      // OS as a double
    double plane_r;   // (P-1)/w_max (0 if P == 1)
    double w_max;
    double gamma;
    double beta;
};

// Result of locating one visibility.
struct Loc {
    int32_t cu, cv, ou, ov, plane;
    bool conj;
    bool keep;
};

// Locate one axis: x = coord*fov + N/2, t = floor(x*OS + 0.5) in IEEE double
// with every operation rounded separately (no FMA contraction), then
// c = floor(t/OS), o = t - c*OS; the footprint c - S/2 + 1 .. c + S/2 must lie
// inside [0, N).  Returns false (drop) otherwise or for non-finite input.
__device__ __forceinline__ bool locate_axis(double coord, const DevParams &p,
                                            int32_t &c, int32_t &o)
{
    double x = __dadd_rn(__dmul_rn(coord, p.fov), p.half);
    double t = floor(__dadd_rn(__dmul_rn(x, p.os_d), 0.5));
    if (!(fabs(t) < 1099511627776.0))  // 2^40; false for NaN
        return false;
    long long ti = (long long)t;
    long long OS = p.OS;
    long long cc = ti >= 0 ? ti / OS : -((-ti + OS - 1) / OS);
    long long oo = ti - cc * OS;
    long long f = cc - p.S / 2 + 1;
    if (f < 0 || f + p.S - 1 > p.N - 1)
        return false;
    c = (int32_t)cc;
    o = (int32_t)oo;
    return true;
}

// Plane: floor(|w| * r + 0.5) with r = (P-1)/w_max, dropped beyond P-1;
// conj = (w < 0).
__device__ __forceinline__ Loc locate(double u, double v, double w, const DevParams &p)
{
    Loc L;
    L.cu = L.cv = L.ou = L.ov = L.plane = 0;
    L.conj = false;
    int32_t cu, cv, ou, ov;
    bool ok = locate_axis(u, p, cu, ou);
    ok = locate_axis(v, p, cv, ov) && ok;
    double q = floor(__dadd_rn(__dmul_rn(fabs(w), p.plane_r), 0.5));
    ok = ok && isfinite(w) && (q <= (double)(p.P - 1));
    L.keep = ok;
    if (ok) {
        L.cu = cu;
        L.cv = cv;
        L.ou = ou;
        L.ov = ov;
        L.plane = (int32_t)q;
        L.conj = w < 0.0;
    }
    return L;
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

constexpr int kChunk = 2048;      // visibilities per work item (tiled forms)
constexpr int kMaxWindow = 64;    // T + S - 1 <= kMaxWindow

// Plan workspace (owned by the context).
struct Plan {
    int64_t nvis = 0;
    int64_t capacity = 0;       // allocated visibility slots
    int32_t ntiles = 0;
    int32_t tiles_capacity = 0;
    int32_t items_capacity = 0;
    bool valid = false;
    int form = 0;
    // tiled forms
    int32_t *d_tile = nullptr;      // [nvis] tile id per visibility (-1 dropped)
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
    int32_t nkept_host_bound = 0;
    // plain form: the coordinates are read directly
    const double *u = nullptr, *v = nullptr, *w = nullptr;
};

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
cudaError_t launch_zero_dropped(const Plan &plan, float2 *vis, cudaStream_t s);

// sepw_tiled.cu
cudaError_t launch_grid_tiled(const DevParams &p, const Plan &plan, const float2 *vis,
                              const float *weight, const float2 *taps, float2 *grid,
                              int num_sms, cudaStream_t s);
cudaError_t launch_degrid_tiled(const DevParams &p, const Plan &plan,
                                const float2 *grid, const float *weight,
                                const float2 *taps, float2 *vis, int num_sms,
                                cudaStream_t s);

// sepw_tc.cu
int tc_tile_for_support(int S);
cudaError_t launch_grid_tc(const DevParams &p, const Plan &plan, const float2 *vis,
                           const float *weight, const float2 *taps, float2 *grid,
                           int num_sms, bool fp16, int32_t *status, cudaStream_t s);

// sepw_image.cu
cudaError_t launch_image_pre(const DevParams &p, int direction, const float *taper,
                             float2 *buf, cudaStream_t s);
cudaError_t launch_image_post(const DevParams &p, int direction, const float *taper,
                              float2 *buf, cudaStream_t s);

}  // namespace sepw
