// Tiled FP32 gridder and degridder (the separable update of Sec. 5, binned).
//
// A persistent CTA takes work items (<= kChunk visibilities of one T x T tile,
// sorted by footprint origin) from an atomic counter.  The tile's window of
// (T + S - 1)^2 cells lives in shared memory (separate re / im planes, row
// stride chosen so a warp's accesses are bank-conflict free).
//
// Gridding: each warp walks a contiguous range of the item's visibilities.
// Lane (rg, j) owns footprint column j and rows rg*RPL .. rg*RPL+RPL-1.  Per
// visibility it forms the partial product W V F1(u - u_i) for its column once
// (Sec. 5: reused down every row) and accumulates RPL complex products with
// the v-taps in registers.  While consecutive visibilities share a footprint
// origin the S x S block stays in registers; when the origin changes it is
// added into the shared window with shared-memory atomics.  At the end of the
// item the window is added to the HBM grid once with float2 atomics (windows
// of neighbouring tiles and other chunks of the same tile overlap).
//
// Degridding (the adjoint): the window is loaded from the HBM grid, each lane
// forms sum_k conj(tv[k]) X[y_k][x_j] for its rows (the block is re-read from
// shared memory only when the origin changes), multiplies by conj(tu[j]) and
// the warp sums the 32 lane partials with shuffles.
#include "sepw_internal.cuh"

namespace sepw {

template <int S>
struct Layout {
    static constexpr int RG = (32 / S) > 0 ? (32 / S) : 1;  // row groups per warp
    static constexpr int RPL = (S + RG - 1) / RG;            // rows per lane
};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

constexpr int kTiledThreads = 256;
constexpr int kTiledWarps = kTiledThreads / 32;

template <int S>
__global__ void __launch_bounds__(kTiledThreads, 2) grid_tiled_kernel(
    DevParams p, int WP, const WorkItem *__restrict__ items,
    const int32_t *__restrict__ nitems, int32_t *counter, const uint64_t *__restrict__ rec,
    const int32_t *__restrict__ perm, const float2 *__restrict__ vis,
    const float *__restrict__ weight, const float2 *__restrict__ taps, float2 *grid)
{
    constexpr int RG = Layout<S>::RG, RPL = Layout<S>::RPL;
    extern __shared__ float smem[];
    __shared__ int s_item;
    const int W = p.T + S - 1;
    float *wre = smem;
    float *wim = smem + W * WP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rg = lane / S, j = lane % S;
    const bool lane_ok = rg < RG;
    const int n_items = *nitems;

    for (int e = threadIdx.x; e < W * WP; e += kTiledThreads) {
        wre[e] = 0.f;
        wim[e] = 0.f;
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0)
            s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items)
            break;
        const WorkItem it = items[item];
        const int per = (it.count + kTiledWarps - 1) / kTiledWarps;
        const int b0 = it.start + min(it.count, warp * per);
        const int b1 = it.start + min(it.count, (warp + 1) * per);

        float2 acc[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            acc[q] = make_float2(0.f, 0.f);
        int cur_lx = -1, cur_ly = -1;

        for (int base = b0; base < b1; base += 32) {
            const int s = base + lane;
            uint64_t r = 0;
            float2 wv = make_float2(0.f, 0.f);
            if (s < b1) {
                r = rec[s];
                const int i = perm[s];
                const float wt = weight ? __ldg(weight + i) : 1.0f;
                const float2 x = __ldg(vis + i);
                wv = make_float2(wt * x.x, wt * x.y);
            }
            const int n = min(32, b1 - base);
            for (int q = 0; q < n; ++q) {
                const uint64_t rq = __shfl_sync(0xffffffffu, r, q);
                const float2 wq = make_float2(__shfl_sync(0xffffffffu, wv.x, q),
                                              __shfl_sync(0xffffffffu, wv.y, q));
                const int lx = rec_lx(rq), ly = rec_ly(rq);
                if (lx != cur_lx || ly != cur_ly) {
                    if (cur_lx >= 0 && lane_ok) {
#pragma unroll
                        for (int qq = 0; qq < RPL; ++qq) {
                            const int k = rg * RPL + qq;
                            if (k < S) {
                                const int a = (cur_ly + k) * WP + cur_lx + j;
                                atomicAdd(wre + a, acc[qq].x);
                                atomicAdd(wim + a, acc[qq].y);
                            }
                        }
                    }
#pragma unroll
                    for (int qq = 0; qq < RPL; ++qq)
                        acc[qq] = make_float2(0.f, 0.f);
                    cur_lx = lx;
                    cur_ly = ly;
                }
                const float sg = rec_conj(rq) ? -1.f : 1.f;
                const int64_t row = (int64_t)rec_plane(rq) * p.OS;
                const float2 *tu = taps + (row + rec_ou(rq)) * S;
                const float2 *tv = taps + (row + rec_ov(rq)) * S;
                if (lane_ok) {
                    float2 a = __ldg(tu + j);
                    a.y *= sg;
                    const float2 pu = cmulf(wq, a);
#pragma unroll
                    for (int qq = 0; qq < RPL; ++qq) {
                        const int k = rg * RPL + qq;
                        if (k < S) {
                            float2 b = __ldg(tv + k);
                            b.y *= sg;
                            acc[qq].x += pu.x * b.x - pu.y * b.y;
                            acc[qq].y += pu.x * b.y + pu.y * b.x;
                        }
                    }
                }
            }
        }
        if (cur_lx >= 0 && lane_ok) {
#pragma unroll
            for (int qq = 0; qq < RPL; ++qq) {
                const int k = rg * RPL + qq;
                if (k < S) {
                    const int a = (cur_ly + k) * WP + cur_lx + j;
                    atomicAdd(wre + a, acc[qq].x);
                    atomicAdd(wim + a, acc[qq].y);
                }
            }
        }
        __syncthreads();
        const int ty = it.tile / p.ntx, tx = it.tile - ty * p.ntx;
        const int64_t gy0 = (int64_t)ty * p.T, gx0 = (int64_t)tx * p.T;
        for (int e = threadIdx.x; e < W * W; e += kTiledThreads) {
            const int rr = e / W, cc = e - rr * W;
            const int a = rr * WP + cc;
            const float re = wre[a], im = wim[a];
            if (re != 0.f || im != 0.f) {
                atomicAdd(grid + (gy0 + rr) * p.N + gx0 + cc, make_float2(re, im));
                wre[a] = 0.f;
                wim[a] = 0.f;
            }
        }
    }
}

template <int S>
__global__ void __launch_bounds__(kTiledThreads, 2) degrid_tiled_kernel(
    DevParams p, int WP, const WorkItem *__restrict__ items,
    const int32_t *__restrict__ nitems, int32_t *counter, const uint64_t *__restrict__ rec,
    const int32_t *__restrict__ perm, const float2 *__restrict__ grid,
    const float *__restrict__ weight, const float2 *__restrict__ taps,
    float2 *__restrict__ vis_out)
{
    constexpr int RG = Layout<S>::RG, RPL = Layout<S>::RPL;
    extern __shared__ float smem[];
    __shared__ int s_item;
    const int W = p.T + S - 1;
    float *wre = smem;
    float *wim = smem + W * WP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rg = lane / S, j = lane % S;
    const bool lane_ok = rg < RG;
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
        const int ty = it.tile / p.ntx, tx = it.tile - ty * p.ntx;
        const int64_t gy0 = (int64_t)ty * p.T, gx0 = (int64_t)tx * p.T;
        for (int e = threadIdx.x; e < W * W; e += kTiledThreads) {
            const int rr = e / W, cc = e - rr * W;
            const int64_t gy = gy0 + rr, gx = gx0 + cc;
            float2 g = make_float2(0.f, 0.f);
            if (gy < p.N && gx < p.N)
                g = __ldg(grid + gy * p.N + gx);
            wre[rr * WP + cc] = g.x;
            wim[rr * WP + cc] = g.y;
        }
        __syncthreads();
        const int per = (it.count + kTiledWarps - 1) / kTiledWarps;
        const int b0 = it.start + min(it.count, warp * per);
        const int b1 = it.start + min(it.count, (warp + 1) * per);

        float xr[RPL], xi[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            xr[q] = xi[q] = 0.f;
        int cur_lx = -1, cur_ly = -1;

        for (int base = b0; base < b1; base += 32) {
            const int s = base + lane;
            uint64_t r = 0;
            int i = 0;
            if (s < b1) {
                r = rec[s];
                i = perm[s];
            }
            float2 outv = make_float2(0.f, 0.f);
            const int n = min(32, b1 - base);
            for (int q = 0; q < n; ++q) {
                const uint64_t rq = __shfl_sync(0xffffffffu, r, q);
                const int lx = rec_lx(rq), ly = rec_ly(rq);
                if (lx != cur_lx || ly != cur_ly) {
                    cur_lx = lx;
                    cur_ly = ly;
                    if (lane_ok) {
#pragma unroll
                        for (int qq = 0; qq < RPL; ++qq) {
                            const int k = rg * RPL + qq;
                            if (k < S) {
                                const int a = (ly + k) * WP + lx + j;
                                xr[qq] = wre[a];
                                xi[qq] = wim[a];
                            }
                        }
                    }
                }
                // conjugate of the gridding kernel: conj(tap) for w >= 0
                const float sg = rec_conj(rq) ? 1.f : -1.f;
                const int64_t row = (int64_t)rec_plane(rq) * p.OS;
                const float2 *tu = taps + (row + rec_ou(rq)) * S;
                const float2 *tv = taps + (row + rec_ov(rq)) * S;
                float tre = 0.f, tim = 0.f;
                if (lane_ok) {
                    float sre = 0.f, sim = 0.f;
#pragma unroll
                    for (int qq = 0; qq < RPL; ++qq) {
                        const int k = rg * RPL + qq;
                        if (k < S) {
                            float2 b = __ldg(tv + k);
                            b.y *= sg;
                            sre += b.x * xr[qq] - b.y * xi[qq];
                            sim += b.x * xi[qq] + b.y * xr[qq];
                        }
                    }
                    float2 a = __ldg(tu + j);
                    a.y *= sg;
                    tre = sre * a.x - sim * a.y;
                    tim = sre * a.y + sim * a.x;
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    tre += __shfl_xor_sync(0xffffffffu, tre, off);
                    tim += __shfl_xor_sync(0xffffffffu, tim, off);
                }
                if (lane == q)
                    outv = make_float2(tre, tim);
            }
            if (s < b1) {
                const float wt = weight ? __ldg(weight + i) : 1.0f;
                vis_out[i] = make_float2(wt * outv.x, wt * outv.y);
            }
        }
    }
}

template <int S>
static cudaError_t launch_grid_S(const DevParams &p, int WP, const Plan &plan,
                                 const float2 *vis, const float *weight,
                                 const float2 *taps, float2 *grid, int num_sms,
                                 cudaStream_t s)
{
    const int W = p.T + S - 1;
    size_t shm = (size_t)2 * W * WP * sizeof(float);
    cudaError_t e = cudaMemsetAsync(plan.d_item_counter, 0, sizeof(int32_t), s);
    if (e != cudaSuccess)
        return e;
    grid_tiled_kernel<S><<<num_sms * 2, kTiledThreads, shm, s>>>(
        p, WP, plan.d_items, plan.d_nitems, plan.d_item_counter, plan.d_rec, plan.d_perm,
        vis, weight, taps, grid);
    return cudaGetLastError();
}

template <int S>
static cudaError_t launch_degrid_S(const DevParams &p, int WP, const Plan &plan,
                                   const float2 *grid, const float *weight,
                                   const float2 *taps, float2 *vis, int num_sms,
                                   cudaStream_t s)
{
    const int W = p.T + S - 1;
    size_t shm = (size_t)2 * W * WP * sizeof(float);
    cudaError_t e = cudaMemsetAsync(plan.d_item_counter + 1, 0, sizeof(int32_t), s);
    if (e != cudaSuccess)
        return e;
    degrid_tiled_kernel<S><<<num_sms * 2, kTiledThreads, shm, s>>>(
        p, WP, plan.d_items, plan.d_nitems, plan.d_item_counter + 1, plan.d_rec,
        plan.d_perm, grid, weight, taps, vis);
    return cudaGetLastError();
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
                unsigned b = 1u << ((g * RPL * wp + jj) & 31);
                if (used & b)
                    ok = false;
                used |= b;
            }
        if (ok)
            return wp;
    }
    return W;
}

#define SEPW_FOR_EACH_S(X) \
    X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(20) X(22) X(24) X(26) X(28) X(30) X(32)

cudaError_t launch_grid_tiled(const DevParams &p, const Plan &plan, const float2 *vis,
                              const float *weight, const float2 *taps, float2 *grid,
                              int num_sms, cudaStream_t s)
{
    const int WP = window_stride(p.T + p.S - 1, p.S);
    switch (p.S) {
#define X(SS) \
    case SS: return launch_grid_S<SS>(p, WP, plan, vis, weight, taps, grid, num_sms, s);
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
    const int WP = window_stride(p.T + p.S - 1, p.S);
    switch (p.S) {
#define X(SS) \
    case SS: return launch_degrid_S<SS>(p, WP, plan, grid, weight, taps, vis, num_sms, s);
        SEPW_FOR_EACH_S(X)
#undef X
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace sepw
