// sepw_grid_noalloc: tiled FP32 gridding that performs no device allocation.
//
// Some callers cannot let a library allocate device memory.  Examples: a
// real-time imaging pipeline that reserves all of its memory at start-up and
// must not block on cudaMalloc (which can synchronise the device) while it is
// observing, or a host framework that owns the device memory pool and forbids
// raw allocations from plugins.  This entry point serves them: instead of a
// context's workspace it uses one fixed scratch array compiled into the
// library as a file-scope __device__ variable, so every GPU that loads the
// library holds that array (kNoallocBytes, about 26 MB) until the process
// exits.
//
// The scratch holds the same plan as the context path (bin ids and ranks,
// packed records, slot permutation, dropped-index list, per-tile counts and
// cursors, per-bin counts, work items and counters), and the existing plan
// and tiled-gridder launchers run on it unchanged.  Every call reuses the
// array: the plan launcher clears the bin counts and the dropped counter at
// the start of each call, the gridder clears its work counter, and
// everything else is overwritten before it is read.  Calls whose work
// overlaps on the GPU (other streams, other host threads) race on the array.
#include <mutex>

#include "sepw_internal.cuh"

namespace sepw {
namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int64_t kMaxVis = SEPW_NOALLOC_MAX_VIS;
constexpr int64_t kMaxTiles = SEPW_NOALLOC_MAX_TILES;
constexpr int64_t kMaxItems = kMaxTiles + kMaxVis / kChunk + 1;

// byte offsets of the plan arrays inside the scratch
constexpr size_t kOffTile = 0;
constexpr size_t kOffRank = align256(kOffTile + sizeof(int32_t) * kMaxVis);
constexpr size_t kOffRec0 = align256(kOffRank + sizeof(int32_t) * kMaxVis);
constexpr size_t kOffRec = align256(kOffRec0 + sizeof(uint64_t) * kMaxVis);
constexpr size_t kOffPerm = align256(kOffRec + sizeof(uint64_t) * kMaxVis);
constexpr size_t kOffDrop = align256(kOffPerm + sizeof(int32_t) * kMaxVis);
constexpr size_t kOffCount = align256(kOffDrop + sizeof(int32_t) * kMaxVis);
constexpr size_t kOffCursor = align256(kOffCount + sizeof(int32_t) * kMaxTiles);
constexpr size_t kOffBin = align256(kOffCursor + sizeof(int32_t) * kMaxTiles);
constexpr size_t kOffItems = align256(kOffBin + sizeof(int32_t) * kSubBins * kMaxTiles);
constexpr size_t kOffNitems = align256(kOffItems + sizeof(WorkItem) * kMaxItems);
constexpr size_t kOffCounter = align256(kOffNitems + sizeof(int32_t));
constexpr size_t kOffDropped = align256(kOffCounter + 2 * sizeof(int32_t));
constexpr size_t kNoallocBytes = align256(kOffDropped + sizeof(unsigned long long));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch per device.  In host code the name
// g_noalloc_scratch is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SEPW_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices)
        return SEPW_ENOTSUP;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return SEPW_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SEPW_OK;
}

bool device_ptr_ok(const void *ptr, bool allow_null)
{
    if (!ptr)
        return allow_null;
    if (((uintptr_t)ptr) & 7)
        return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace sepw

using namespace sepw;

extern "C" int sepw_grid_noalloc(const sepw_params *prm, const float *taps, int64_t nvis,
                                 const double *u, const double *v, const double *w,
                                 const float *vis, const float *weight, float *grid,
                                 int64_t *n_dropped, sepw_stream_t stream)
{
    if (!prm)
        return SEPW_EINVAL;
    // the tiled FP32 form runs whatever form the caller names: check (and
    // resolve the default tile of) that form, not the caller's
    sepw_params tp = *prm;
    tp.form = SEPW_FORM_TILED;
    int rc = sepw_check_params(&tp);
    if (rc != SEPW_OK)
        return rc;
    if (nvis < 0)
        return SEPW_EINVAL;
    if (nvis > kMaxVis)
        return SEPW_ETOOLARGE;

    const DevParams dp = make_dev_params(&tp);
    const int64_t ntiles = (int64_t)dp.ntx * dp.ntx;
    if (ntiles > kMaxTiles)
        return SEPW_ETOOLARGE;

    if (!device_ptr_ok(taps, false) || !device_ptr_ok(grid, false) ||
        !device_ptr_ok(n_dropped, true))
        return SEPW_EINVAL;
    // the tiled gridder reads rows of taps as 16-byte vectors
    if (((uintptr_t)taps) & 15)
        return SEPW_EINVAL;
    if (nvis > 0 && (!device_ptr_ok(u, false) || !device_ptr_ok(v, false) ||
                     !device_ptr_ok(w, false) || !device_ptr_ok(vis, false) ||
                     !device_ptr_ok(weight, true)))
        return SEPW_EINVAL;

    void *base = nullptr;
    if ((rc = scratch_address(&base)) != SEPW_OK)
        return rc;
    int dev = 0, num_sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return SEPW_ECUDA;
    }

    unsigned char *b = (unsigned char *)base;
    Plan pl;
    pl.nvis = nvis;
    pl.capacity = kMaxVis;
    pl.ntiles = (int32_t)ntiles;
    pl.tiles_capacity = (int32_t)kMaxTiles;
    pl.items_capacity = (int32_t)(ntiles + nvis / kChunk + 1);
    pl.valid = true;
    pl.form = SEPW_FORM_TILED;
    pl.d_tile = (int32_t *)(b + kOffTile);
    pl.d_rank = (int32_t *)(b + kOffRank);
    pl.d_rec0 = (uint64_t *)(b + kOffRec0);
    pl.d_rec = (uint64_t *)(b + kOffRec);
    pl.d_perm = (int32_t *)(b + kOffPerm);
    pl.d_drop_list = (int32_t *)(b + kOffDrop);
    pl.d_tile_count = (int32_t *)(b + kOffCount);
    pl.d_tile_cursor = (int32_t *)(b + kOffCursor);
    pl.d_bin = (int32_t *)(b + kOffBin);
    pl.d_items = (WorkItem *)(b + kOffItems);
    pl.d_nitems = (int32_t *)(b + kOffNitems);
    pl.d_item_counter = (int32_t *)(b + kOffCounter);
    pl.d_dropped = (unsigned long long *)(b + kOffDropped);

    cudaStream_t s = (cudaStream_t)stream;
    if (launch_plan(dp, nvis, u, v, w, pl, s) != cudaSuccess) {
        cudaGetLastError();
        return SEPW_ECUDA;
    }
    if (nvis > 0 && launch_grid_tiled(dp, pl, (const float2 *)vis, weight,
                                      (const float2 *)taps, nullptr, (float2 *)grid, num_sms,
                                      s) != cudaSuccess) {
        cudaGetLastError();
        return SEPW_ECUDA;
    }
    if (n_dropped && cudaMemcpyAsync(n_dropped, pl.d_dropped, sizeof(int64_t),
                                     cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return SEPW_ECUDA;
    }
    return SEPW_OK;
}
