// Plan construction for the tiled forms: locate every visibility, bin it by
// the T x T tile that holds its footprint origin and, inside the tile, by the
// 4 x 4 sub-block of the origin and conj (counting sort with warp-aggregated
// atomics), cut each tile into work items of at most kChunk visibilities, and
// sort each item by (footprint origin, conj) so that consecutive visibilities
// with the same origin and kernel conjugation can be accumulated in one
// register block.
//
// The update structure this serves is Sec. 5: every visibility adds a
// separable S x S block at its own offset; visibilities that share a tile
// share one shared-memory window, and visibilities that share an origin share
// one register block.
#include "sepw_internal.cuh"

namespace sepw {

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Pass 1: locate, record, bin histogram with each visibility's rank inside
// its bin (the order of arrival at the bin's counter), dropped count.
__global__ void __launch_bounds__(256) locate_bin_kernel(
    DevParams p, int64_t nvis, const double *__restrict__ u, const double *__restrict__ v,
    const double *__restrict__ w, int32_t *__restrict__ bin_of,
    int32_t *__restrict__ rank_of, uint64_t *__restrict__ rec0, int32_t *bin_count,
    unsigned long long *dropped, int32_t *__restrict__ drop_list, int ngrids,
    const int64_t *__restrict__ offsets)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool active = i < nvis;
    int bin = -1;
    if (active) {
        Loc L = locate(u[i], v[i], w[i], p);
        if (L.keep) {
            int fx = L.cu - p.S / 2 + 1, fy = L.cv - p.S / 2 + 1;
            const int tx = div_tile(fx, p), ty = div_tile(fy, p);
            int g = 0;
            if (ngrids > 1) {  // grid of visibility i: offsets[g] <= i < offsets[g+1]
                int lo = 0, hi = ngrids - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (offsets[mid] <= i)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                g = lo;
            }
            const int lx = fx - tx * p.T, ly = fy - ty * p.T;
            bin = ((g * p.ntx + ty) * p.ntx + tx) * kSubBins + sub_bin(lx, ly, L.conj, p);
            rec0[i] = pack_rec(lx, ly, L.ou, L.ov, L.plane, L.conj);
        }
        bin_of[i] = bin;
    }
    unsigned act = __ballot_sync(0xffffffffu, active && bin >= 0);
    unsigned drop = __ballot_sync(0xffffffffu, active && bin < 0);
    int lane = threadIdx.x & 31;
    if (drop) {
        // append the dropped indices (degridding writes 0 there)
        int leader = __ffs(drop) - 1;
        unsigned long long base = 0;
        if (lane == leader)
            base = atomicAdd(dropped, (unsigned long long)__popc(drop));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (active && bin < 0)
            drop_list[base + __popc(drop & lanemask_lt())] = (int32_t)i;
    }
    if (active && bin >= 0) {
        const unsigned peers = __match_any_sync(act, bin);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader)
            base = atomicAdd(bin_count + bin, __popc(peers));
        base = __shfl_sync(act, base, leader);
        rank_of[i] = base + __popc(peers & lanemask_lt());
    }
}

// Pass 1b (one warp per tile): the tile's visibility count, and each bin's
// count replaced by its offset inside the tile (exclusive scan of the 32).
__global__ void __launch_bounds__(256) bin_scan_kernel(int32_t ntiles,
                                                       int32_t *__restrict__ bin,
                                                       int32_t *__restrict__ tile_count)
{
    static_assert(kSubBins == 32, "one lane per bin");
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= ntiles)
        return;
    const int c = bin[t * kSubBins + lane];
    int incl = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off)
            incl += y;
    }
    bin[t * kSubBins + lane] = incl - c;
    if (lane == 31)
        tile_count[t] = incl;
}

// Pass 2 (one block of 1024 threads): exclusive scans of the tile counts
// (-> slot cursors) and of the per-tile chunk counts (-> work items).  Full
// chunks (`chunk` visibilities) are listed before the partial ones, so that
// dynamically scheduled workers take the heavy items first; within each list
// the items are in tile order.  Warp w owns the tiles [w R, (w + 1) R) and
// walks them 32 at a time, one tile per lane, so that its loads and its
// cursor and item stores are coalesced: a first walk sums the range, a block
// scan gives every warp its bases, and a second walk writes the cursors and
// items from warp-shuffle scans of each group of 32 tiles.
constexpr int kScanThreads = 1024;
constexpr int kScanWarps = kScanThreads / 32;

__device__ __forceinline__ void warp_scan3(int64_t &a, int32_t &b, int32_t &c, int lane)
{
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t x = __shfl_up_sync(0xffffffffu, a, off);
        const int32_t y = __shfl_up_sync(0xffffffffu, b, off);
        const int32_t z = __shfl_up_sync(0xffffffffu, c, off);
        if (lane >= off) {
            a += x;
            b += y;
            c += z;
        }
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_kernel(
    int32_t ntiles, int32_t chunk, const int32_t *__restrict__ tile_count,
    int32_t *__restrict__ cursor, WorkItem *__restrict__ items, int32_t *nitems)
{
    __shared__ int64_t s_cnt[kScanWarps];
    __shared__ int32_t s_full[kScanWarps], s_part[kScanWarps];
    __shared__ int32_t s_tot_full, s_tot_part;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int R = (((ntiles + kScanWarps - 1) / kScanWarps) + 31) & ~31;  // tiles per warp
    const int lo = min(ntiles, warp * R), hi = min(ntiles, lo + R);
    // walk 1: the range's totals (visibilities, full chunks, partial chunks)
    int64_t c = 0;
    int32_t nf = 0, np = 0;
    for (int i0 = lo; i0 < hi; i0 += 32 * 4) {
        int n[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + 32 * k + lane;
            n[k] = i < hi ? tile_count[i] : 0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            c += n[k];
            nf += n[k] / chunk;
            np += (n[k] % chunk) != 0;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, off);
        nf += __shfl_xor_sync(0xffffffffu, nf, off);
        np += __shfl_xor_sync(0xffffffffu, np, off);
    }
    if (lane == 0) {
        s_cnt[warp] = c;
        s_full[warp] = nf;
        s_part[warp] = np;
    }
    __syncthreads();
    if (warp == 0) {
        int64_t wc = s_cnt[lane];
        int32_t wf = s_full[lane], wp = s_part[lane];
        const int64_t c0 = wc;
        const int32_t f0 = wf, p0 = wp;
        warp_scan3(wc, wf, wp, lane);
        s_cnt[lane] = wc - c0;  // exclusive warp bases
        s_full[lane] = wf - f0;
        s_part[lane] = wp - p0;
        if (lane == 31) {
            s_tot_full = wf;
            s_tot_part = wp;
        }
    }
    __syncthreads();
    const int32_t total_full = s_tot_full;
    int64_t base_c = s_cnt[warp];
    int32_t base_f = s_full[warp], base_p = total_full + s_part[warp];
    // walk 2: cursors and items, 32 tiles at a time
    for (int i0 = lo; i0 < hi; i0 += 32) {
        const int i = i0 + lane;
        const int n = i < hi ? tile_count[i] : 0;
        const int nk = n / chunk, part = (n % chunk) != 0;
        int64_t ic = n;
        int32_t ik = nk, ipt = part;
        warp_scan3(ic, ik, ipt, lane);
        const int64_t off_c = base_c + ic - n;  // exclusive
        const int32_t off_f = base_f + ik - nk, off_p = base_p + ipt - part;
        if (i < hi) {
            cursor[i] = (int32_t)off_c;
            for (int q = 0; q < nk; ++q) {
                WorkItem it;
                it.tile = i;
                it.start = (int32_t)(off_c + (int64_t)q * chunk);
                it.count = chunk;
                it.pad = 0;
                items[off_f + q] = it;
            }
            if (part) {
                WorkItem it;
                it.tile = i;
                it.start = (int32_t)(off_c + (int64_t)nk * chunk);
                it.count = n % chunk;
                it.pad = 0;
                items[off_p] = it;
            }
        }
        base_c += __shfl_sync(0xffffffffu, ic, 31);
        base_f += __shfl_sync(0xffffffffu, ik, 31);
        base_p += __shfl_sync(0xffffffffu, ipt, 31);
    }
    if (t == 0)
        *nitems = total_full + s_tot_part;
}

// Pass 3: scatter visibility ids and records to their slots: tile start +
// offset of the bin inside the tile + rank inside the bin.
__global__ void __launch_bounds__(256) scatter_kernel(
    int64_t nvis, const int32_t *__restrict__ bin_of, const int32_t *__restrict__ rank_of,
    const uint64_t *__restrict__ rec0, const int32_t *__restrict__ tile_start,
    const int32_t *__restrict__ bin_off, int32_t *__restrict__ perm,
    uint64_t *__restrict__ rec)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvis)
        return;
    const int b = bin_of[i];
    if (b < 0)
        return;
    const int slot = __ldg(tile_start + b / kSubBins) + __ldg(bin_off + b) + rank_of[i];
    perm[slot] = (int32_t)i;
    rec[slot] = rec0[i];
}

// Pass 4: inside each work item, counting sort by (footprint origin, conj),
// sub-block major: the key orders by the 4 x 4 sub-block of the origin and
// conj (the bin of pass 1), then by the origin's row and column inside the
// sub-block (edge at most E = ceil(T / 4)), 32 E^2 <= 8192 keys.
// Visibilities that share a key share one register block in the tiled
// kernels, and the block never mixes conjugated and plain kernels; the
// sub-blocks stay contiguous inside an item, so a run of slots that starts
// and ends in one sub-block lies inside it.  One block per item; the item's
// slots are rewritten in place.  The order among equal keys is arbitrary.
constexpr int kSortThreads = 512;
constexpr int kMaxSortBins = 2 * 64 * 64;
constexpr int kMaxBinsPerThread = kMaxSortBins / kSortThreads;

__device__ __forceinline__ int sort_key(uint64_t r, const DevParams &p, int E)
{
    const int lx = rec_lx(r), ly = rec_ly(r);
    const int sx = div_tile(lx * 4, p), sy = div_tile(ly * 4, p);
    const int x0 = (sx * p.T + 3) >> 2, y0 = (sy * p.T + 3) >> 2;  // first cell
    const int sub = ((sx * 4 + sy) << 1) | (rec_conj(r) ? 1 : 0);  // as sub_bin
    return (sub * E + (ly - y0)) * E + (lx - x0);
}

__global__ void __launch_bounds__(kSortThreads) item_sort_kernel(
    DevParams p, const WorkItem *__restrict__ items, const int32_t *__restrict__ nitems,
    int32_t *__restrict__ perm, uint64_t *__restrict__ rec)
{
    extern __shared__ int32_t hist[];  // per * kSortThreads bins
    __shared__ uint64_t s_rec[kChunk];
    __shared__ int32_t s_perm[kChunk];
    __shared__ int32_t s_wsum[32];
    // blocks stride over the plan's items (sparse plans have far fewer items
    // than their capacity, so the grid is sized by the SM count, not by it)
    const int n_items = *nitems;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const WorkItem it = items[item];
    const int n = it.count;
    const int E = (p.T + 3) / 4;
    const int nb = 32 * E * E;
    const int per = (nb + kSortThreads - 1) / kSortThreads;
    for (int b = threadIdx.x; b < per * kSortThreads; b += kSortThreads)
        hist[b] = 0;
    __syncthreads();
    // a warp's lanes hold consecutive slots, where runs of one key are
    // common: one shared-memory atomic per distinct key per warp
    const int lane_id = threadIdx.x & 31;
    for (int q0 = 0; q0 < n; q0 += kSortThreads) {
        const int q = q0 + (int)threadIdx.x;
        const bool act = q < n;
        int key = -1;
        if (act) {
            const uint64_t r = rec[it.start + q];
            s_rec[q] = r;
            s_perm[q] = perm[it.start + q];
            key = sort_key(r, p, E);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (act && lane_id == __ffs(peers) - 1)
            atomicAdd(hist + key, __popc(peers));
    }
    __syncthreads();
    // exclusive scan: thread t owns bins [t*per, t*per + per)
    const int t = threadIdx.x;
    int local[kMaxBinsPerThread];
    int sum = 0;
#pragma unroll
    for (int q = 0; q < kMaxBinsPerThread; ++q) {
        local[q] = q < per ? hist[t * per + q] : 0;
        sum += local[q];
    }
    const int lane = t & 31, warp = t >> 5;
    int incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off)
            incl += y;
    }
    if (lane == 31)
        s_wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = kSortThreads / 32;
        const int x = lane < nw ? s_wsum[lane] : 0;
        int y = x;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int z = __shfl_up_sync(0xffffffffu, y, off);
            if (lane >= off)
                y += z;
        }
        if (lane < nw)
            s_wsum[lane] = y - x;  // exclusive warp offsets
    }
    __syncthreads();
    int run = s_wsum[warp] + incl - sum;
#pragma unroll
    for (int q = 0; q < kMaxBinsPerThread; ++q) {
        if (q < per)
            hist[t * per + q] = run;
        run += local[q];
    }
    __syncthreads();
    for (int q0 = 0; q0 < n; q0 += kSortThreads) {
        const int q = q0 + (int)threadIdx.x;
        const bool act = q < n;
        uint64_t r = 0;
        int key = -1;
        if (act) {
            r = s_rec[q];
            key = sort_key(r, p, E);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (act && lane_id == leader)
            base = atomicAdd(hist + key, __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (act) {
            const int dst = base + __popc(peers & lanemask_lt());
            rec[it.start + dst] = r;
            perm[it.start + dst] = s_perm[q];
        }
    }
    __syncthreads();  // shared memory is reused by the next item
    }
}

// Degridding writes 0 for every dropped visibility of the plan.
__global__ void zero_dropped_kernel(const int32_t *__restrict__ drop_list,
                                    const unsigned long long *__restrict__ ndrop,
                                    float2 *__restrict__ vis)
{
    const unsigned long long n = *ndrop;
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         k < n; k += (unsigned long long)gridDim.x * blockDim.x)
        vis[drop_list[k]] = make_float2(0.f, 0.f);
}

cudaError_t launch_zero_dropped(const Plan &plan, float2 *vis, cudaStream_t s)
{
    zero_dropped_kernel<<<64, 256, 0, s>>>(plan.d_drop_list, plan.d_dropped, vis);
    return cudaGetLastError();
}

cudaError_t launch_plan(const DevParams &p, int64_t nvis, const double *u,
                        const double *v, const double *w, Plan &plan, cudaStream_t s)
{
    cudaError_t e;
    e = cudaMemsetAsync(plan.d_bin, 0, sizeof(int32_t) * kSubBins * (size_t)plan.ntiles, s);
    if (e != cudaSuccess)
        return e;
    e = cudaMemsetAsync(plan.d_dropped, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess)
        return e;
    if (nvis > 0) {
        locate_bin_kernel<<<(unsigned)((nvis + 255) / 256), 256, 0, s>>>(
            p, nvis, u, v, w, plan.d_tile, plan.d_rank, plan.d_rec0, plan.d_bin,
            plan.d_dropped, plan.d_drop_list, plan.ngrids, plan.d_offsets);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
    }
    bin_scan_kernel<<<(unsigned)(((int64_t)plan.ntiles * 32 + 255) / 256), 256, 0, s>>>(
        plan.ntiles, plan.d_bin, plan.d_tile_count);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    scan_kernel<<<1, kScanThreads, 0, s>>>(plan.ntiles, p.chunk, plan.d_tile_count,
                                           plan.d_tile_cursor, plan.d_items, plan.d_nitems);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    if (nvis > 0) {
        scatter_kernel<<<(unsigned)((nvis + 255) / 256), 256, 0, s>>>(
            nvis, plan.d_tile, plan.d_rank, plan.d_rec0, plan.d_tile_cursor, plan.d_bin,
            plan.d_perm, plan.d_rec);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        // the per-item sort by (sub-block, conj, origin) serves the kernels
        // that walk runs of one origin (the tiled FP32 gridder and
        // degridder); the 16-bit tensor-core forms (one-part and hi + lo)
        // grid and degrid in any order within an item and skip it
        if (plan.form == SEPW_FORM_TC_BF16 || plan.form == SEPW_FORM_TC_FP16 ||
            plan.form == SEPW_FORM_TC_FP16X2 || plan.form == SEPW_FORM_TC_BF16X2)
            return cudaSuccess;
        const int E = (p.T + 3) / 4;
        const int nb = 32 * E * E;
        const size_t shm =
            sizeof(int32_t) * kSortThreads * ((nb + kSortThreads - 1) / kSortThreads);
        e = cudaFuncSetAttribute(item_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)shm);
        if (e != cudaSuccess)
            return e;
        int dev = 0, sms = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        const int nblk = std::max(1, std::min(plan.items_capacity, 16 * sms));
        item_sort_kernel<<<nblk, kSortThreads, shm, s>>>(p, plan.d_items, plan.d_nitems,
                                                         plan.d_perm, plan.d_rec);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace sepw
