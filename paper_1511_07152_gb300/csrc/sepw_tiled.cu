// Tiled FP32 gridder and degridder (the separable update of Sec. 5, binned).
//
// Work items are <= kChunk visibilities of one T x T tile, sorted by
// (footprint origin, conj) ("key"), taken from an atomic counter: by a whole
// warp in the gridder, by a whole CTA in the degridder, which keeps the
// tile's window of (T + S - 1)^2 cells in shared memory.  Per batch of
// visibilities a warp first decodes the records once (one per lane: tap-row
// offsets, W V or the output index and weight, key) into shared memory; the
// inner loop reads them as broadcasts.
//
// What limits these kernels is the load data returned to the registers, the
// latency of those loads (gridder) and the instruction issue (degridder),
// not the FMA pipe: every lane loads the taps of the cells it owns for every
// visibility.  Larger per-lane register blocks load fewer taps per cell, so
// the forms below use, by support:
//   * gridding, S = 8, 16: lane (rg, cg) = (lane >> 3, lane & 7) owns
//     rows rg + 4 r and columns cg + 8 c (S / 4 + S / 8 taps per lane per
//     visibility);
//   * degridding, S = 4 .. 16, S % 4 = 0: two virtual warps of 16 lanes take
//     two visibilities per step; lane (rg, cg) = (t >> 2, t & 3) owns rows
//     rg + 4 r and columns cg + 4 c (2 S / 4 taps per lane per visibility);
//   * other supports: lane (rg, j) owns footprint column j and S / RG rows.
// The interleaved cell assignment makes the lanes of one atomic or window
// read cover a compact patch (few sectors per atomic, no bank conflicts).
//
// Gridding: per visibility the lane forms the partial product W V F1(u - u_i)
// for its columns once (Sec. 5: reused down every row) and accumulates its
// cells' products with the v-taps into a register block, as paired FP32 FMAs
// over its row pairs (v-taps from a lane-ordered planar copy of the table,
// rebuilt per call).  Visibilities with
// one key share the register block; conj visibilities accumulate
// conj(W V) F1 F1 and the block is conjugated when it is flushed, so the
// inner loop needs no sign handling.  The block is added to the HBM grid with
// float2 atomics (native L2 reductions) when the key changes.  (A
// shared-memory window in between was slower: float adds to shared memory
// run as compare-and-swap loops, several instructions per add.)
//
// Degridding (the adjoint): the lane keeps its window cells (conjugated for
// plain-kernel groups) in registers while the key is unchanged, forms
// sum_r F1_v(r) X(r, c) per column and then the sum over its columns with
// F1_u(c); the partial sums of several visibilities are reduced over the
// lanes together (reduce-scatter), conjugated back as needed and scaled by W.
#include <type_traits>

#include "sepw_internal.cuh"

namespace sepw {

template <int S>
struct Layout {
    static constexpr int RG = (32 / S) > 0 ? (32 / S) : 1;  // row groups per warp
    static constexpr int RPL = (S + RG - 1) / RG;            // rows per lane
    static constexpr bool VEC = (RPL % 2) == 0;              // 16-byte tap loads
    static constexpr bool FULL_ROWS = RG * RPL == S;         // no row beyond S
    static constexpr bool ALL_LANES = RG * S == 32;          // every lane works
};

// Per-visibility metadata staged in shared memory, one 16-byte record:
//   x = row offset of the u-taps in the table, (plane * OS + ou) * S
//   y = key | (v-tap row - u-tap row) << 13, key = (ly * 64 + lx) << 1 | conj
//   z, w = gridding: W V (conjugated for conj visibilities) as float bits;
//          degridding: visibility index, weight as float bits
__device__ __forceinline__ int meta_key(int y) { return y & 0x1fff; }
__device__ __forceinline__ int meta_dv(int y) { return y >> 13; }

constexpr int kTiledThreads = 256;
constexpr int kTiledWarps = kTiledThreads / 32;
constexpr int kTiledBlocksPerSM = 4;
// block gridder on dense plans: work units per item (see its work loop)
constexpr int kGridParts = 8;
constexpr int kGridPartsMinDensity = 256;  // visibilities per tile

__device__ __forceinline__ int key_ly(int key) { return (key >> 1) >> 6; }
__device__ __forceinline__ int key_lx(int key) { return (key >> 1) & 63; }

// Loads the RPL v-taps of this lane's rows (rows >= S give zero).
template <int S>
__device__ __forceinline__ void load_vtaps(const float2 *__restrict__ row, int rg,
                                           float (&tr)[Layout<S>::RPL],
                                           float (&ti)[Layout<S>::RPL])
{
    constexpr int RPL = Layout<S>::RPL;
    const int k0 = rg * RPL;
    if constexpr (Layout<S>::VEC) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row + k0);
#pragma unroll
        for (int q = 0; q < RPL / 2; ++q) {
            float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
            if (Layout<S>::FULL_ROWS || k0 + 2 * q < S)
                t = __ldg(r4 + q);
            tr[2 * q] = t.x;
            ti[2 * q] = t.y;
            tr[2 * q + 1] = t.z;
            ti[2 * q + 1] = t.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            float2 t = make_float2(0.f, 0.f);
            if (Layout<S>::FULL_ROWS || k0 + q < S)
                t = __ldg(row + k0 + q);
            tr[q] = t.x;
            ti[q] = t.y;
        }
    }
}

template <int S>
__global__ void __launch_bounds__(kTiledThreads, kTiledBlocksPerSM) grid_tiled_kernel(
    DevParams p, const WorkItem *__restrict__ items, const int32_t *__restrict__ nitems,
    int32_t *counter, const uint64_t *__restrict__ rec, const int32_t *__restrict__ perm,
    const float2 *__restrict__ vis, const float *__restrict__ weight,
    const float2 *__restrict__ taps, float2 *grid)
{
    constexpr int RG = Layout<S>::RG, RPL = Layout<S>::RPL;
    __shared__ int4 s_meta[kTiledWarps * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int4 *meta = s_meta + warp * 32;
    const int rg = lane / S, j = lane % S;
    const bool lane_ok = Layout<S>::ALL_LANES || rg < RG;
    const int n_items = *nitems;

    // every warp takes whole work items on its own: no block-wide barrier
    for (;;) {
        int item = 0;
        if (lane == 0)
            item = atomicAdd(counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items)
            break;
        const WorkItem it = items[item];
        const TileOrigin o = tile_origin(p, it.tile);
        float2 *const tgrid = grid + o.base + o.gy0 * p.N + o.gx0;
        const int b0 = it.start, b1 = it.start + it.count;

        float ar[RPL], ai[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            ar[q] = ai[q] = 0.f;
        int cur = -1;

        // adds the register block of key `cur` to the grid (float2 atomics,
        // native L2 reductions) and clears it
        auto flush = [&]() {
            if (cur >= 0 && lane_ok) {
                const float sg = (cur & 1) ? -1.f : 1.f;
                float2 *g = tgrid + (int64_t)(key_ly(cur) + rg * RPL) * p.N + key_lx(cur) + j;
#pragma unroll
                for (int q = 0; q < RPL; ++q)
                    if (Layout<S>::FULL_ROWS || rg * RPL + q < S)
                        atomicAdd(g + (int64_t)q * p.N, make_float2(ar[q], sg * ai[q]));
            }
#pragma unroll
            for (int q = 0; q < RPL; ++q)
                ar[q] = ai[q] = 0.f;
        };

        for (int base = b0; base < b1; base += 32) {
            const int s = base + lane;
            if (s < b1) {
                const uint64_t r = rec[s];
                const int i = perm[s];
                const float wt = weight ? __ldg(weight + i) : 1.0f;
                const float2 x = __ldg(vis + i);
                const bool cj = rec_conj(r);
                const int row = rec_plane(r) * p.OS;
                const int key = ((rec_ly(r) * 64 + rec_lx(r)) << 1) | (cj ? 1 : 0);
                meta[lane] = make_int4((row + rec_ou(r)) * S,
                                       key | ((rec_ov(r) - rec_ou(r)) * S) * 8192,
                                       __float_as_int(wt * x.x),
                                       __float_as_int(cj ? -wt * x.y : wt * x.y));
            }
            __syncwarp();
            const int n = min(32, b1 - base);
            for (int q = 0; q < n; ++q) {
                const int4 m = meta[q];
                const int key = meta_key(m.y);
                if (key != cur) {
                    flush();
                    cur = key;
                }
                if (lane_ok) {
                    const float wx = __int_as_float(m.z), wy = __int_as_float(m.w);
                    const float2 *tu = taps + m.x;
                    const float2 a = __ldg(tu + j);
                    const float pr = wx * a.x - wy * a.y;
                    const float pi = wx * a.y + wy * a.x;
                    float tr[RPL], ti[RPL];
                    load_vtaps<S>(tu + p.voff + meta_dv(m.y), rg, tr, ti);
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        ar[k] = fmaf(pr, tr[k], ar[k]);
                        ar[k] = fmaf(-pi, ti[k], ar[k]);
                        ai[k] = fmaf(pr, ti[k], ai[k]);
                        ai[k] = fmaf(pi, tr[k], ai[k]);
                    }
                }
            }
            __syncwarp();
        }
        flush();
    }
}

// Sum of v[e] over the 32 lanes for e = 0..7; on return v[0] holds the sum
// for e = (lane >> 2) & 7.
__device__ __forceinline__ void reduce8(float (&v)[8], int lane)
{
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = b4 ? v[i] : v[i + 4];
        const float keep = b4 ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b3 ? v[i] : v[i + 2];
        const float keep = b3 ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    {
        const float send = b2 ? v[0] : v[1];
        const float keep = b2 ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <int S>
__global__ void __launch_bounds__(kTiledThreads, kTiledBlocksPerSM) degrid_tiled_kernel(
    DevParams p, int WP, const WorkItem *__restrict__ items,
    const int32_t *__restrict__ nitems, int32_t *counter, const uint64_t *__restrict__ rec,
    const int32_t *__restrict__ perm, const float2 *__restrict__ grid,
    const float *__restrict__ weight, const float2 *__restrict__ taps,
    float2 *__restrict__ vis_out)
{
    constexpr int RG = Layout<S>::RG, RPL = Layout<S>::RPL;
    extern __shared__ float4 smem4[];
    __shared__ int s_item;
    const int W = p.T + S - 1;
    float *wre = reinterpret_cast<float *>(smem4);
    float *wim = wre + W * WP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int4 *meta = reinterpret_cast<int4 *>(smem4 + ((2 * W * WP + 3) / 4)) + warp * 32;
    const int rg = lane / S, j = lane % S;
    const bool lane_ok = Layout<S>::ALL_LANES || rg < RG;
    const int n_items = *nitems;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0)
            s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items)
            break;
        const WorkItem it = items[item];
        const TileOrigin o = tile_origin(p, it.tile);
        for (int rr = warp; rr < W; rr += kTiledWarps) {
            const int64_t gy = o.gy0 + rr;
            const float2 *grow = grid + o.base + gy * p.N + o.gx0;
            for (int cc = lane; cc < W; cc += 32) {
                float2 g = make_float2(0.f, 0.f);
                if (gy < p.N && o.gx0 + cc < p.N)
                    g = __ldg(grow + cc);
                wre[rr * WP + cc] = g.x;
                wim[rr * WP + cc] = g.y;
            }
        }
        __syncthreads();
        const int per = (it.count + kTiledWarps - 1) / kTiledWarps;
        const int b0 = it.start + min(it.count, warp * per);
        const int b1 = it.start + min(it.count, (warp + 1) * per);

        float xr[RPL], xi[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            xr[q] = xi[q] = 0.f;
        int cur = -1;

        for (int base = b0; base < b1; base += 32) {
            const int s = base + lane;
            if (s < b1) {
                const uint64_t r = rec[s];
                const int i = perm[s];
                const int row = rec_plane(r) * p.OS;
                const int key = ((rec_ly(r) * 64 + rec_lx(r)) << 1) | (rec_conj(r) ? 1 : 0);
                meta[lane] = make_int4((row + rec_ou(r)) * S,
                                       key | ((rec_ov(r) - rec_ou(r)) * S) * 8192, i,
                                       __float_as_int(weight ? __ldg(weight + i) : 1.0f));
            }
            __syncwarp();
            const int n = min(32, b1 - base);
            for (int qb = 0; qb < n; qb += 8) {
                float vr[8], vi[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    vr[e] = vi[e] = 0.f;
                    if (qb + e < n) {
                        const int4 m = meta[qb + e];
                        const int key = meta_key(m.y);
                        if (key != cur) {
                            cur = key;
                            if (lane_ok) {
                                const int ly = key_ly(cur), lx = key_lx(cur);
                                // plain-kernel groups work on conj(X)
                                const float sg = (cur & 1) ? 1.f : -1.f;
#pragma unroll
                                for (int q = 0; q < RPL; ++q) {
                                    const int k = rg * RPL + q;
                                    if (k < S) {
                                        const int a = (ly + k) * WP + lx + j;
                                        xr[q] = wre[a];
                                        xi[q] = sg * wim[a];
                                    }
                                }
                            }
                        }
                        if (lane_ok) {
                            const float2 *tu = taps + m.x;
                            float tr[RPL], ti[RPL];
                            load_vtaps<S>(tu + p.voff + meta_dv(m.y), rg, tr, ti);
                            float sr = 0.f, si = 0.f;
#pragma unroll
                            for (int k = 0; k < RPL; ++k) {
                                sr = fmaf(tr[k], xr[k], sr);
                                sr = fmaf(-ti[k], xi[k], sr);
                                si = fmaf(tr[k], xi[k], si);
                                si = fmaf(ti[k], xr[k], si);
                            }
                            const float2 a = __ldg(tu + j);
                            vr[e] = sr * a.x - si * a.y;
                            vi[e] = sr * a.y + si * a.x;
                        }
                    }
                }
                reduce8(vr, lane);
                reduce8(vi, lane);
                const int e = lane >> 2;
                if ((lane & 3) == 0 && qb + e < n) {
                    const int4 m = meta[qb + e];
                    const float wt = __int_as_float(m.w);
                    // plain-kernel groups computed conj(V / W)
                    const float im = (m.y & 1) ? vi[0] : -vi[0];
                    vis_out[m.z] = make_float2(wt * vr[0], wt * im);
                }
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// Degridding with 4 x 4 lane grids of B x B register blocks (S = 4 B).
//
// A warp is two virtual warps of 16 lanes, each with its own contiguous
// slice of the item, so two visibilities are updated per warp step.  Lane
// (rg, cg) = (t >> 2, t & 3) of a virtual warp owns the cells at footprint
// rows rg + 4 r and columns cg + 4 c (r, c < B): per visibility B u-taps and
// B v-taps.  Its 16 lanes read a 4 x 4 patch of the window at a time, which
// with a row stride of 4 (mod 8) float2 hits every bank once.  Batches in
// which both virtual warps hold K visibilities (all but a slice's last) run
// a copy of the loop without per-slot bounds tests (7% faster).
// ---------------------------------------------------------------------------
template <int S>
struct Blk {
    static constexpr bool OK = S % 4 == 0 && S >= 4 && S <= 16;
    static constexpr int B = S / 4;  // cells per lane along each axis
    static constexpr int K = 16;     // visibilities staged per virtual warp
    static constexpr int MS = K + 1; // staging stride (virtual warps on other banks)
    static constexpr int BPS = S == 16 ? 3 : 4;  // resident CTAs per SM (registers)
};

// Loads the B taps k0, k0 + 4, ... of one table row.
template <int B>
__device__ __forceinline__ void load_taps4(const float2 *__restrict__ row, int k0,
                                           float (&re)[B], float (&im)[B])
{
#pragma unroll
    for (int c = 0; c < B; ++c) {
        const float2 t = __ldg(row + k0 + 4 * c);
        re[c] = t.x;
        im[c] = t.y;
    }
}


// Sum of v[e] over the 16 lanes of a virtual warp for e = 0..7 (re of four
// visibilities, then im); on return v[0] holds the sum for component
// (t >> 3) of visibility (t >> 1) & 3, identical on lanes t and t ^ 1.
__device__ __forceinline__ void reduce16x8(float (&v)[8], int t)
{
    const bool b3 = t & 8, b2 = t & 4, b1 = t & 2;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = b3 ? v[i] : v[i + 4];
        const float keep = b3 ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b2 ? v[i] : v[i + 2];
        const float keep = b2 ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const float send = b1 ? v[0] : v[1];
        const float keep = b1 ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <int S>
__global__ void __launch_bounds__(kTiledThreads, Blk<S>::BPS) degrid_tiled_block_kernel(
    DevParams p, int WP, const WorkItem *__restrict__ items,
    const int32_t *__restrict__ nitems, int32_t *counter, const uint64_t *__restrict__ rec,
    const int32_t *__restrict__ perm, const float2 *__restrict__ grid,
    const float *__restrict__ weight, const float2 *__restrict__ taps,
    float2 *__restrict__ vis_out)
{
    constexpr int B = Blk<S>::B, K = Blk<S>::K, MS = Blk<S>::MS;
    extern __shared__ float4 smem4[];
    __shared__ int s_item;
    const int W = p.T + S - 1;
    float2 *const win = reinterpret_cast<float2 *>(smem4);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int vw = lane >> 4, t = lane & 15, rg = t >> 2, cg = t & 3;
    int4 *const meta = reinterpret_cast<int4 *>(smem4 + ((W * WP + 1) / 2)) + (warp * 2 + vw) * MS;
    int *const keys = reinterpret_cast<int *>(meta - (warp * 2 + vw) * MS + kTiledWarps * 2 * MS) +
                      (warp * 2 + vw) * MS;
    // tap offsets (table elements) of this lane's first u- and v-tap: the
    // loads add unsigned 32-bit offsets to the table base (1% faster than
    // per-lane pointers plus signed offsets)
    const unsigned ocol = (unsigned)cg;
    const unsigned orow = (unsigned)(p.voff + rg);
    const int n_items = *nitems;
    // this lane's first window cell relative to the footprint origin
    const float2 *const lwin = win + rg * WP + cg;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0)
            s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items)
            break;
        const WorkItem it = items[item];
        if (!work_item_ok(p, it))
            continue;  // checked build only (uniform over the CTA)
        const TileOrigin o = tile_origin(p, it.tile);
        for (int rr = warp; rr < W; rr += kTiledWarps) {
            const int64_t gy = o.gy0 + rr;
            const float2 *grow = grid + o.base + gy * p.N + o.gx0;
            for (int cc = lane; cc < W; cc += 32) {
                float2 g = make_float2(0.f, 0.f);
                if (gy < p.N && o.gx0 + cc < p.N)
                    g = __ldg(grow + cc);
                win[rr * WP + cc] = g;
            }
        }
        __syncthreads();
        // 16 workers (two per warp) take contiguous slices of the item
        const int per = (it.count + 2 * kTiledWarps - 1) / (2 * kTiledWarps);
        const int wk = warp * 2 + vw;
        const int v0 = it.start + min(it.count, wk * per);
        const int v1 = it.start + min(it.count, (wk + 1) * per);

        float xr[B][B], xi[B][B];
        int cur = -1;
        // both virtual warps run the same number of steps (warp shuffles)
        for (int base = 0; base < per; base += K) {
            const int s = v0 + base + t;
            if (s < v1) {
                const uint64_t r = rec[s];
                const int i = perm[s];
                if (record_ok(p, r, i, o.gy0, o.gx0)) {
                    const int row = rec_plane(r) * p.OS;
                    meta[t] = make_int4((row + rec_ou(r)) * S, (row + rec_ov(r)) * S, i,
                                        __float_as_int(weight ? __ldg(weight + i) : 1.0f));
                    keys[t] = ((rec_ly(r) * 64 + rec_lx(r)) << 1) | (rec_conj(r) ? 1 : 0);
                } else {
                    // checked build: taps of row 0 at window origin 0, no output
                    meta[t] = make_int4(0, 0, -1, 0);
                    keys[t] = 0;
                }
            }
            __syncwarp();
            const int n = min(K, v1 - (v0 + base));  // may be <= 0
            const int nw = max(n, __shfl_xor_sync(0xffffffffu, n, 16));
            // one group of four visibilities per virtual warp; CHK = false
            // when both halves hold a full batch (no per-slot bounds test)
            auto groups = [&](auto chk) {
                constexpr bool CHK = decltype(chk)::value;
                for (int qb = 0; qb < nw; qb += 4) {
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        v[e] = v[e + 4] = 0.f;
                        if (!CHK || qb + e < n) {
                            const int key = keys[qb + e];
                            if (key != cur) {
                                cur = key;
                                // plain-kernel groups work on conj(X)
                                const float sg = (cur & 1) ? 1.f : -1.f;
                                const float2 *wl = lwin + key_ly(cur) * WP + key_lx(cur);
#pragma unroll
                                for (int r = 0; r < B; ++r)
#pragma unroll
                                    for (int c = 0; c < B; ++c) {
                                        const float2 x = wl[4 * r * WP + 4 * c];
                                        xr[r][c] = x.x;
                                        xi[r][c] = sg * x.y;
                                    }
                            }
                            const int4 m = meta[qb + e];
                            float ur[B], ui[B], vr[B], vi[B];
                            load_taps4<B>(taps + (ocol + (unsigned)m.x), 0, ur, ui);
                            load_taps4<B>(taps + (orow + (unsigned)m.y), 0, vr, vi);
                            float sr = 0.f, si = 0.f;
#pragma unroll
                            for (int c = 0; c < B; ++c) {
                                float tr = 0.f, ti = 0.f;  // sum_r F1_v(r) X(r, c)
#pragma unroll
                                for (int r = 0; r < B; ++r) {
                                    tr = fmaf(vr[r], xr[r][c], tr);
                                    tr = fmaf(-vi[r], xi[r][c], tr);
                                    ti = fmaf(vr[r], xi[r][c], ti);
                                    ti = fmaf(vi[r], xr[r][c], ti);
                                }
                                sr = fmaf(tr, ur[c], sr);
                                sr = fmaf(-ti, ui[c], sr);
                                si = fmaf(tr, ui[c], si);
                                si = fmaf(ti, ur[c], si);
                            }
                            v[e] = sr;
                            v[e + 4] = si;
                        }
                    }
                    reduce16x8(v, t);
                    // lanes t < 8 with even t hold re of visibility (t >> 1);
                    // lane t + 8 holds its im
                    const float im = __shfl_down_sync(0xffffffffu, v[0], 8);
                    const int e = t >> 1;
                    if (t < 8 && (t & 1) == 0 && (!CHK || qb + e < n)) {
                        const int4 m = meta[qb + e];
                        const float wt = __int_as_float(m.w);
                        // plain-kernel groups computed conj(V / W)
                        const float vi_ = (keys[qb + e] & 1) ? im : -im;
                        if (!SEPW_CHECKED || m.z >= 0)  // m.z < 0: skipped slot
                            vis_out[m.z] = make_float2(wt * v[0], wt * vi_);
                    }
                }
            };
            if (__all_sync(0xffffffffu, n == K))
                groups(std::false_type{});
            else
                groups(std::true_type{});
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// Gridding with a 4 x 8 lane grid, S = 8, 16.  Lane (rg, cg) =
// (lane >> 3, lane & 7) owns the cells at footprint rows rg + 4 r
// (r < RB = S / 4) and columns cg + 8 c (c < ceil(S / 8), column < S).  The
// inner loop runs over runs of equal keys found with one ballot per batch, so
// the flush and its branch sit outside it.
//
// The accumulators of the lane's rows 2q and 2q + 1 in one column form a
// pair, (re, re) and (im, im), so that the complex multiply-adds of the
// outer product run as paired FP32 FMAs (two FMAs per instruction): per row
// pair and column
//     re += (vr_2q, vr_2q+1) pr - (vi_2q, vi_2q+1) pi
//     im += (vi_2q, vi_2q+1) pr + (vr_2q, vr_2q+1) pi
// with the same rounding sequence per cell as scalar FMAs.  The v-tap pairs
// come straight from the lane-ordered planar copy of the table (see
// planar_taps_kernel: a lane's RB taps are adjacent); without it (PLANAR
// false) they are rearranged from the interleaved table in registers.
// ---------------------------------------------------------------------------
template <int S>
struct Blk2 {
    // S = 12 leaves half the lanes with one column: the column-per-lane
    // kernel was faster there (sparse batched grids, 11.1 vs 13.0 ms)
    static constexpr bool OK = S == 8 || S == 16;
    static constexpr int RB = S / 4;        // rows per lane
    static constexpr int RP = RB / 2;       // row pairs per lane
    static constexpr int CB = (S + 7) / 8;  // columns per lane
    static constexpr bool FULL = S % 8 == 0;
};

// five resident CTAs per SM (48 registers): the kernel is bound by load
// latency, and 40 warps hide it better than 32 (2.37 vs 2.44 ms on 32M
// visibilities; six CTAs at 40 registers spill and run slower, 2.56 ms)
constexpr int kGridBlkPerSM = 5;

template <int S, bool PLANAR>
__global__ void __launch_bounds__(kTiledThreads, kGridBlkPerSM) grid_tiled_block_kernel(
    DevParams p, const WorkItem *__restrict__ items, const int32_t *__restrict__ nitems,
    int32_t *counter, const uint64_t *__restrict__ rec, const int32_t *__restrict__ perm,
    const float2 *__restrict__ vis, const float *__restrict__ weight,
    const float2 *__restrict__ taps, const float *__restrict__ planar, float2 *grid,
    int parts)
{
    constexpr int RB = Blk2<S>::RB, RP = Blk2<S>::RP, CB = Blk2<S>::CB;
    constexpr bool FULL = Blk2<S>::FULL;
    static_assert(RB % 2 == 0, "rows come in pairs");
    __shared__ int4 s_meta[kTiledWarps * 32];
    __shared__ int s_key[kTiledWarps * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rg = lane >> 3, cg = lane & 7;
    int4 *const meta = s_meta + warp * 32;
    int *const keys = s_key + warp * 32;
    // this lane's u-tap column and first v-tap row within a table row; in
    // the planar copy its RB v-taps sit at RB rg .. RB rg + RB - 1
    const float2 *const tcol = taps + cg;
    const float2 *const trow = taps + p.voff + rg;
    const float *const prow = PLANAR ? planar + 2 * p.voff + RB * rg : nullptr;
    const int n_items = *nitems;

    for (;;) {
        // a warp takes one of `parts` consecutive parts of an item: on dense
        // plans whole 2048-visibility items per warp left the end of the
        // launch to few warps (parts: 1 -> 2.38 ms, 2 -> 2.24, 4 -> 2.16,
        // 8 -> 2.13, 16 -> 2.14 on 32M visibilities; runs break only at part
        // edges).  Sparse plans (many small items) keep parts = 1: split
        // units there only add atomics on the one counter.
        int unit = 0;
        if (lane == 0)
            unit = atomicAdd(counter, 1);
        unit = __shfl_sync(0xffffffffu, unit, 0);
        const int item = unit / parts, part = unit % parts;
        if (item >= n_items)
            break;
        const WorkItem it = items[item];
        if (!work_item_ok(p, it))
            continue;  // checked build only
        const int len = (it.count + parts - 1) / parts;
        const int b0 = it.start + part * len;
        const int b1 = min(it.start + it.count, b0 + len);
        if (b0 >= b1)
            continue;
        const TileOrigin o = tile_origin(p, it.tile);
        float2 *const tgrid = grid + o.base + (o.gy0 + rg) * p.N + o.gx0 + cg;

        // ar[q][c] = (re of rows 2q, 2q + 1) of column c (footprint rows
        // rg + 8 q, rg + 8 q + 4); ai likewise
        float2 ar[RP][CB], ai[RP][CB];
#pragma unroll
        for (int q = 0; q < RP; ++q)
#pragma unroll
            for (int c = 0; c < CB; ++c)
                ar[q][c] = ai[q][c] = make_float2(0.f, 0.f);
        int cur = -1;

        // adds the register block of key `cur` to the grid and clears it;
        // conj groups accumulated conj(W V) F1 F1 and are conjugated here
        auto flush = [&]() {
            if (cur >= 0) {
                const float sg = (cur & 1) ? -1.f : 1.f;
                float2 *g = tgrid + key_ly(cur) * p.N + key_lx(cur);
#pragma unroll
                for (int q = 0; q < RP; ++q) {
#pragma unroll
                    for (int c = 0; c < CB; ++c)
                        if (FULL || cg + 8 * c < S) {
                            atomicAdd(g + 8 * c, make_float2(ar[q][c].x, sg * ai[q][c].x));
                            atomicAdd(g + 4 * p.N + 8 * c,
                                      make_float2(ar[q][c].y, sg * ai[q][c].y));
                        }
                    g += 8 * p.N;
                }
            }
#pragma unroll
            for (int q = 0; q < RP; ++q)
#pragma unroll
                for (int c = 0; c < CB; ++c)
                    ar[q][c] = ai[q][c] = make_float2(0.f, 0.f);
        };

        for (int base = b0; base < b1; base += 32) {
            // lane q stages slot base + q: tap-row offsets, W V, key
            const int s = base + lane;
            int kq = -1;
            if (s < b1) {
                const uint64_t r = rec[s];
                const int i = perm[s];
                if (record_ok(p, r, i, o.gy0, o.gx0)) {
                    const float wt = weight ? __ldg(weight + i) : 1.0f;
                    const float2 x = __ldg(vis + i);
                    const bool cj = rec_conj(r);
                    const int row = rec_plane(r) * p.OS;
                    kq = ((rec_ly(r) * 64 + rec_lx(r)) << 1) | (cj ? 1 : 0);
                    meta[lane] = make_int4((row + rec_ou(r)) * S, (row + rec_ov(r)) * S,
                                           __float_as_int(wt * x.x),
                                           __float_as_int(cj ? -wt * x.y : wt * x.y));
                } else {
                    // checked build: a skipped slot adds zero under key -1,
                    // which the flush never writes
                    meta[lane] = make_int4(0, 0, 0, 0);
                }
                keys[lane] = kq;
            }
            __syncwarp();
            const int n = min(32, b1 - base);
            // runs of equal keys in this batch: bit q set where slot q starts one
            const int kp = __shfl_up_sync(0xffffffffu, kq, 1);
            const unsigned starts = __ballot_sync(0xffffffffu, lane < n && (lane == 0 || kq != kp));
            for (int q = 0; q < n;) {
                const unsigned later = starts & ~((2u << q) - 1u);
                const int q1 = later ? __ffs(later) - 1 : n;
                const int key = keys[q];
                if (key != cur) {
                    flush();
                    cur = key;
                }
                for (; q < q1; ++q) {
                    const int4 m = meta[q];
                    const float wx = __int_as_float(m.z), wy = __int_as_float(m.w);
                    const float2 *tu = tcol + m.x;
                    float pr[CB], pi[CB];
#pragma unroll
                    for (int c = 0; c < CB; ++c) {
                        float2 a = make_float2(0.f, 0.f);
                        if (FULL || cg + 8 * c < S)
                            a = __ldg(tu + 8 * c);
                        // partial product W V F1(u), Sec. 5
                        pr[c] = wx * a.x - wy * a.y;
                        pi[c] = wx * a.y + wy * a.x;
                    }
                    // v-tap pairs of this lane's rows: (vr_2q, vr_2q+1), (vi_2q, vi_2q+1)
                    float2 vr[RP], vi[RP];
                    if constexpr (PLANAR) {
                        const float *pv = prow + 2 * m.y;
                        if constexpr (RP == 2) {
                            const float4 re = __ldg(reinterpret_cast<const float4 *>(pv));
                            const float4 im = __ldg(reinterpret_cast<const float4 *>(pv + S));
                            vr[0] = make_float2(re.x, re.y);
                            vr[1] = make_float2(re.z, re.w);
                            vi[0] = make_float2(im.x, im.y);
                            vi[1] = make_float2(im.z, im.w);
                        } else {
#pragma unroll
                            for (int q2 = 0; q2 < RP; ++q2) {
                                vr[q2] = __ldg(reinterpret_cast<const float2 *>(pv) + q2);
                                vi[q2] = __ldg(reinterpret_cast<const float2 *>(pv + S) + q2);
                            }
                        }
                    } else {
                        const float2 *tv = trow + m.y;
#pragma unroll
                        for (int q2 = 0; q2 < RP; ++q2) {
                            const float2 t0 = __ldg(tv + 8 * q2), t1 = __ldg(tv + 8 * q2 + 4);
                            vr[q2] = make_float2(t0.x, t1.x);
                            vi[q2] = make_float2(t0.y, t1.y);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < CB; ++c) {
                        const float2 prr = make_float2(pr[c], pr[c]);
                        const float2 pii = make_float2(pi[c], pi[c]);
                        const float2 npi = make_float2(-pi[c], -pi[c]);
#pragma unroll
                        for (int q2 = 0; q2 < RP; ++q2) {
                            ar[q2][c] = __ffma2_rn(vr[q2], prr, ar[q2][c]);
                            ar[q2][c] = __ffma2_rn(vi[q2], npi, ar[q2][c]);
                            ai[q2][c] = __ffma2_rn(vi[q2], prr, ai[q2][c]);
                            ai[q2][c] = __ffma2_rn(vr[q2], pii, ai[q2][c]);
                        }
                    }
                }
            }
            __syncwarp();
        }
        flush();
    }
}

// Row stride of the shared window: the smallest WP >= W for which the row
// groups of a warp touch disjoint banks.
static int window_stride(int W, int S)
{
    const int RG = (32 / S) > 0 ? (32 / S) : 1;
    const int RPL = (S + RG - 1) / RG;
    for (int wp = W; wp < W + 32; ++wp) {
        unsigned used = 0;
        bool ok = true;
        for (int g = 0; g < RG && ok; ++g)
            for (int jj = 0; jj < S && ok; ++jj) {
                const unsigned b = 1u << ((g * RPL * wp + jj) & 31);
                if (used & b)
                    ok = false;
                used |= b;
            }
        if (ok)
            return wp;
    }
    return W;
}

static size_t tiled_smem(int W, int WP)
{
    // window (re + im), then per warp 32 int4 of metadata
    return sizeof(float4) * (size_t)((2 * W * WP + 3) / 4) +
           (size_t)kTiledWarps * 32 * sizeof(int4);
}

// Lane-ordered planar copy of a tap table: row j of S complex taps becomes
// S real parts followed by S imaginary parts (same bytes per row, same row
// order), with tap k at position (k mod 4) S/4 + floor(k / 4) when 4 divides
// S.  A lane of the block gridder owns rows g, g + 4, g + 8, ... (g = k mod 4),
// whose taps are then adjacent: one vector load gives its FP32 pairs.
__global__ void planar_taps_kernel(const float2 *__restrict__ taps, float *__restrict__ out,
                                   int64_t n, int S)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / S;
        const int k = (int)(e - row * S);
        const int pos = S % 4 == 0 ? (k & 3) * (S >> 2) + (k >> 2) : k;
        const float2 t = taps[e];
        out[row * 2 * S + pos] = t.x;
        out[row * 2 * S + S + pos] = t.y;
    }
}

static cudaError_t launch_planar_taps(const float2 *taps, float *out, int64_t n, int S,
                               cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    const int64_t blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    planar_taps_kernel<<<(unsigned)blocks, 256, 0, s>>>(taps, out, n, S);
    return cudaGetLastError();
}

template <int S>
static cudaError_t launch_grid_S(const DevParams &p, const Plan &plan, const float2 *vis,
                                 const float *weight, const float2 *taps, float *planar,
                                 float2 *grid, int num_sms, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(plan.d_item_counter, 0, sizeof(int32_t), s);
    if (e != cudaSuccess)
        return e;
    if constexpr (Blk2<S>::OK) {
        const unsigned nb = (unsigned)(num_sms * kGridBlkPerSM);
        const int parts =
            p.grid_parts > 0 ? p.grid_parts
            : plan.nvis >= (int64_t)kGridPartsMinDensity * plan.ntiles ? kGridParts : 1;
        if (planar) {  // rebuilt per call: the caller's table may have changed
            const int64_t n = (p.facet ? 2 : 1) * (int64_t)p.P * p.OS * S;
            if ((e = launch_planar_taps(taps, planar, n, S, s)) != cudaSuccess)
                return e;
        }
        if (planar)
            grid_tiled_block_kernel<S, true><<<nb, kTiledThreads, 0, s>>>(
                p, plan.d_items, plan.d_nitems, plan.d_item_counter, plan.d_rec, plan.d_perm,
                vis, weight, taps, planar, grid, parts);
        else
            grid_tiled_block_kernel<S, false><<<nb, kTiledThreads, 0, s>>>(
                p, plan.d_items, plan.d_nitems, plan.d_item_counter, plan.d_rec, plan.d_perm,
                vis, weight, taps, nullptr, grid, parts);
    } else
        grid_tiled_kernel<S><<<num_sms * kTiledBlocksPerSM, kTiledThreads, 0, s>>>(
            p, plan.d_items, plan.d_nitems, plan.d_item_counter, plan.d_rec, plan.d_perm, vis,
            weight, taps, grid);
    return cudaGetLastError();
}

template <int S>
static cudaError_t launch_degrid_S(const DevParams &p, const Plan &plan,
                                   const float2 *grid, const float *weight,
                                   const float2 *taps, float2 *vis, int num_sms,
                                   cudaStream_t s)
{
    const int W = p.T + S - 1;
    cudaError_t e = cudaMemsetAsync(plan.d_item_counter + 1, 0, sizeof(int32_t), s);
    if (e != cudaSuccess)
        return e;
    if constexpr (Blk<S>::OK) {
        // float2 window rows with stride = 4 (mod 8): the 4 x 4 patch read by a
        // virtual warp covers all 32 banks
        const int WP = W + ((4 - W % 8) + 8) % 8;
        const size_t shm = sizeof(float4) * (size_t)((W * WP + 1) / 2) +
                           (size_t)kTiledWarps * 2 * Blk<S>::MS * (sizeof(int4) + sizeof(int));
        degrid_tiled_block_kernel<S><<<num_sms * Blk<S>::BPS, kTiledThreads, shm, s>>>(
            p, WP, plan.d_items, plan.d_nitems, plan.d_item_counter + 1, plan.d_rec,
            plan.d_perm, grid, weight, taps, vis);
    } else {
        const int WP = window_stride(W, S);
        const size_t shm = tiled_smem(W, WP);
        degrid_tiled_kernel<S><<<num_sms * kTiledBlocksPerSM, kTiledThreads, shm, s>>>(
            p, WP, plan.d_items, plan.d_nitems, plan.d_item_counter + 1, plan.d_rec,
            plan.d_perm, grid, weight, taps, vis);
    }
    return cudaGetLastError();
}

#define SEPW_FOR_EACH_S(X) \
    X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(20) X(22) X(24) X(26) X(28) X(30) X(32)

// the plan's bounds for the checked build's checks (unused otherwise)
static DevParams with_plan_bounds(const DevParams &p, const Plan &plan)
{
    DevParams q = p;
    q.chk_nvis = plan.nvis;
    q.chk_tiles = (int64_t)p.ntx * p.ntx * plan.ngrids;
    return q;
}

cudaError_t launch_grid_tiled(const DevParams &p0, const Plan &plan, const float2 *vis,
                              const float *weight, const float2 *taps, float *planar,
                              float2 *grid, int num_sms, cudaStream_t s)
{
    const DevParams p = with_plan_bounds(p0, plan);
    switch (p.S) {
#define X(SS) \
    case SS: return launch_grid_S<SS>(p, plan, vis, weight, taps, planar, grid, num_sms, s);
        SEPW_FOR_EACH_S(X)
#undef X
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_degrid_tiled(const DevParams &p0, const Plan &plan,
                                const float2 *grid, const float *weight,
                                const float2 *taps, float2 *vis, int num_sms,
                                cudaStream_t s)
{
    const DevParams p = with_plan_bounds(p0, plan);
    switch (p.S) {
#define X(SS) \
    case SS: return launch_degrid_S<SS>(p, plan, grid, weight, taps, vis, num_sms, s);
        SEPW_FOR_EACH_S(X)
#undef X
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace sepw
