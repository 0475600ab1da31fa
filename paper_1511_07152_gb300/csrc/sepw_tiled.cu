// Tiled FP32 gridder and degridder (the separable update of Sec. 5, binned).
//
// Work items are <= kChunk visibilities of one T x T tile, sorted by
// (footprint origin, conj), taken from an atomic counter: by a whole warp in
// the gridder, by a whole CTA in the degridder.  The degridder keeps the
// tile's window of (T + S - 1)^2 cells in shared memory (separate re / im
// planes; row stride chosen so the row groups of a warp hit disjoint banks).
//
// Lane (rg, j) of a warp owns footprint column j and rows rg*RPL ..
// rg*RPL + RPL - 1.  Each warp walks a contiguous slice of the item.  Per
// block of 32 visibilities the warp first decodes the records once (one per
// lane: origin/conj key, tap-row offsets, W V) into one 16-byte shared-memory
// record each; the inner loop then reads them as broadcasts and loads the
// v-taps of its rows with 128-bit loads.
//
// Gridding: per visibility the lane forms the partial product W V F1(u - u_i)
// for its column once (Sec. 5: reused down every row) and accumulates RPL
// complex products with the v-taps into a register block.  A block of
// visibilities with one key shares the register block; for conj visibilities
// it accumulates conj(W V) F1 F1 and is conjugated when it is flushed, so the
// inner loop needs no sign handling.  The register block is added to the HBM
// grid with float2 atomics (native L2 reductions) when the key changes.  (A
// shared-memory window in between was slower: float adds to shared memory
// run as compare-and-swap loops, several instructions per add.)
//
// Degridding (the adjoint): the window is loaded from HBM; the lane keeps its
// RPL window values (conjugated for plain-kernel groups) in registers while
// the key is unchanged, forms sum_k F1_v(k) X'(k) and multiplies by F1_u(j).
// Eight visibilities are reduced over the 32 lanes together (reduce-scatter:
// 9 shuffles per component instead of 40), then conjugated back as needed and
// scaled by W.
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
                    load_vtaps<S>(tu + meta_dv(m.y), rg, tr, ti);
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
                            load_vtaps<S>(tu + meta_dv(m.y), rg, tr, ti);
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

template <int S>
static cudaError_t launch_grid_S(const DevParams &p, const Plan &plan, const float2 *vis,
                                 const float *weight, const float2 *taps, float2 *grid,
                                 int num_sms, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(plan.d_item_counter, 0, sizeof(int32_t), s);
    if (e != cudaSuccess)
        return e;
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
    const int WP = window_stride(W, S);
    const size_t shm = tiled_smem(W, WP);
    cudaError_t e = cudaMemsetAsync(plan.d_item_counter + 1, 0, sizeof(int32_t), s);
    if (e != cudaSuccess)
        return e;
    degrid_tiled_kernel<S><<<num_sms * kTiledBlocksPerSM, kTiledThreads, shm, s>>>(
        p, WP, plan.d_items, plan.d_nitems, plan.d_item_counter + 1, plan.d_rec,
        plan.d_perm, grid, weight, taps, vis);
    return cudaGetLastError();
}

#define SEPW_FOR_EACH_S(X) \
    X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(20) X(22) X(24) X(26) X(28) X(30) X(32)

cudaError_t launch_grid_tiled(const DevParams &p, const Plan &plan, const float2 *vis,
                              const float *weight, const float2 *taps, float2 *grid,
                              int num_sms, cudaStream_t s)
{
    switch (p.S) {
#define X(SS) \
    case SS: return launch_grid_S<SS>(p, plan, vis, weight, taps, grid, num_sms, s);
        SEPW_FOR_EACH_S(X)
#undef X
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_degrid_tiled(const DevParams &p, const Plan &plan,
                                const float2 *grid, const float *weight,
                                const float2 *taps, float2 *vis, int num_sms,
                                cudaStream_t s)
{
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
