// Stored correction of the separable kernel (Sec. 7): the difference
// F_w - F~_w between the exact 2-D W-projection kernel and the separable one,
// kept in a full 2-D table, and a second gridding / degridding pass that
// applies it on top of the separable pass.
//
// Table: res[p][ovr][our][k][j] for the Sr x Sr central footprint cells
// (first at k0 = (S - Sr)/2) and OSr oversample offsets per axis (coarse
// entry c stands for the fine offset c * OS / OSr).  Built in float64:
//   F_w(d_u, d_v) = (1/N^2) sum_{a,b} c1(nu_a) c1(nu_b) exp(2 pi i w (n_ab - 1))
//                   exp(-2 pi i (d_u nu_a + d_v nu_b))
// as two passes over the pixels (rows d_v first, then columns d_u), minus the
// outer product of the 1-D taps at the same offsets.  The DFT phases reuse
// the exact integer reduction of the taps kernel (twiddles of N*OS).
//
// Pass: each warp takes work items of the plan; per visibility the lanes
// cover the Sr^2 cells.  Gridding adds W V R (conj(R) for w < 0) with float2
// atomics; degridding adds W sum conj(kernel) X to the visibility (the
// separable degridding pass writes it first).
#include "sepw_internal.cuh"

namespace sepw {

constexpr int kResRows = 8;  // table rows accumulated per thread in pass A

// exp(-2 pi i d nu_b) with d * OS = dos (an integer) and nu_b = (b - N/2)/N
__device__ __forceinline__ double2 dft_tw(const double2 *tw, int64_t M, int64_t dos, int b,
                                          int N)
{
    int64_t m = (dos * (int64_t)(b - N / 2)) % M;
    if (m < 0)
        m += M;
    return tw[m];
}

// integer d * OS of table row r = (coarse offset c, tap t)
__device__ __forceinline__ int64_t row_dos(const DevParams &p, int Sr, int OSr, int r)
{
    const int c = r / Sr, t = r % Sr;
    const int kk = (p.S - Sr) / 2 + t;
    return (int64_t)(kk - p.S / 2 + 1) * p.OS - (int64_t)c * (p.OS / OSr);
}

// pass A: X[p][r][a] = sum_b E[r][b] c1(nu_a) c1(nu_b) exp(2 pi i w_p (n_ab - 1))
// grid (ceil(N / 256), P, ceil(R / kResRows)); block 256
__global__ void __launch_bounds__(256) residual_rows_kernel(DevParams p, int Sr, int OSr,
                                                            const double *taper64,
                                                            const double2 *tw, double2 *X)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int plane = blockIdx.y;
    const int R = OSr * Sr;
    const int r0 = blockIdx.z * kResRows;
    if (a >= p.N)
        return;
    const int64_t M = (int64_t)p.N * p.OS;
    const double wp = p.P > 1 ? (double)plane * p.w_max / (double)(p.P - 1) : 0.0;
    const double l = (double)(a - p.N / 2) / (double)p.N * p.fov;
    const double ca = taper64[a];
    int64_t dos[kResRows];
    double2 acc[kResRows];
#pragma unroll
    for (int q = 0; q < kResRows; ++q) {
        dos[q] = r0 + q < R ? row_dos(p, Sr, OSr, r0 + q) : 0;
        acc[q] = make_double2(0.0, 0.0);
    }
    for (int b = 0; b < p.N; ++b) {
        const double m = (double)(b - p.N / 2) / (double)p.N * p.fov;
        const double r2 = l * l + m * m;
        const double nm1 = -r2 / (1.0 + sqrt(1.0 - r2));
        double s, c;
        sincospi(2.0 * (wp * nm1), &s, &c);
        const double h = ca * taper64[b];
        const double hr = h * c, hi = h * s;
#pragma unroll
        for (int q = 0; q < kResRows; ++q) {
            const double2 e = dft_tw(tw, M, dos[q], b, p.N);
            acc[q].x += e.x * hr - e.y * hi;
            acc[q].y += e.x * hi + e.y * hr;
        }
    }
    const int64_t base = (int64_t)plane * R * p.N;
#pragma unroll
    for (int q = 0; q < kResRows; ++q)
        if (r0 + q < R)
            X[base + (int64_t)(r0 + q) * p.N + a] = acc[q];
}

// pass B: K[(rv, ru)] = (1/N^2) sum_a X[rv][a] E[ru][a], minus the separable
// product; writes the table.  grid (ceil(R*R / 256), P); block 256
__global__ void __launch_bounds__(256) residual_cols_kernel(DevParams p, int Sr, int OSr,
                                                            const double2 *tw, const double2 *X,
                                                            const double2 *taps64,
                                                            double2 *out64, float2 *out32)
{
    const int R = OSr * Sr;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int plane = blockIdx.y;
    if (e >= R * R)
        return;
    const int rv = e / R, ru = e % R;
    const int64_t M = (int64_t)p.N * p.OS;
    const int64_t dos = row_dos(p, Sr, OSr, ru);
    const double2 *x = X + ((int64_t)plane * R + rv) * p.N;
    double kr = 0.0, ki = 0.0;
    for (int a = 0; a < p.N; ++a) {
        const double2 t = dft_tw(tw, M, dos, a, p.N);
        const double2 v = x[a];
        kr += v.x * t.x - v.y * t.y;
        ki += v.x * t.y + v.y * t.x;
    }
    const double inv = 1.0 / ((double)p.N * (double)p.N);
    kr *= inv;
    ki *= inv;
    // separable product at the same offsets: taps[p][o][kk]
    const int step = p.OS / OSr, k0 = (p.S - Sr) / 2;
    const int cv = rv / Sr, k = rv % Sr, cu = ru / Sr, j = ru % Sr;
    const double2 tv = taps64[((int64_t)plane * p.OS + cv * step) * p.S + k0 + k];
    const double2 tu = taps64[((int64_t)plane * p.OS + cu * step) * p.S + k0 + j];
    kr -= tv.x * tu.x - tv.y * tu.y;
    ki -= tv.x * tu.y + tv.y * tu.x;
    const int64_t idx = (((int64_t)plane * OSr + cv) * OSr + cu) * Sr * Sr + k * Sr + j;
    if (out64)
        out64[idx] = make_double2(kr, ki);
    if (out32)
        out32[idx] = make_float2((float)kr, (float)ki);
}

cudaError_t launch_residual_table(const DevParams &p, int Sr, int OSr, const double *taper64,
                                  const double2 *tw, const double2 *taps64, double2 *X,
                                  double2 *out64, float2 *out32, cudaStream_t s)
{
    const int R = OSr * Sr;
    dim3 ga((p.N + 255) / 256, p.P, (R + kResRows - 1) / kResRows);
    residual_rows_kernel<<<ga, 256, 0, s>>>(p, Sr, OSr, taper64, tw, X);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    dim3 gb((R * R + 255) / 256, p.P);
    residual_cols_kernel<<<gb, 256, 0, s>>>(p, Sr, OSr, tw, X, taps64, out64, out32);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// correction passes over the plan's work items
// ---------------------------------------------------------------------------

constexpr int kResWarps = 8;

__global__ void __launch_bounds__(kResWarps * 32) grid_residual_kernel(
    DevParams p, int Sr, int OSr, const WorkItem *__restrict__ items,
    const int32_t *__restrict__ nitems, int32_t *counter, const uint64_t *__restrict__ rec,
    const int32_t *__restrict__ perm, const float2 *__restrict__ vis,
    const float *__restrict__ weight, const float2 *__restrict__ res, float2 *grid)
{
    const int lane = threadIdx.x & 31;
    const int n_items = *nitems;
    const int step = p.OS / OSr, k0 = (p.S - Sr) / 2, cells = Sr * Sr;
    for (;;) {
        int item = 0;
        if (lane == 0)
            item = atomicAdd(counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items)
            break;
        const WorkItem it = items[item];
        const TileOrigin o = tile_origin(p, it.tile);
        float2 *const tg = grid + o.base + (o.gy0 + k0) * p.N + o.gx0 + k0;
        for (int s = it.start; s < it.start + it.count; ++s) {
            const uint64_t r = rec[s];
            const int i = perm[s];
            const float wt = weight ? __ldg(weight + i) : 1.0f;
            const float2 x = __ldg(vis + i);
            const float wr = wt * x.x, wi = wt * x.y;
            const float sg = rec_conj(r) ? -1.f : 1.f;
            const float2 *R = res + (((int64_t)rec_plane(r) * OSr + rec_ov(r) / step) * OSr +
                                     rec_ou(r) / step) * cells;
            float2 *g = tg + (int64_t)rec_ly(r) * p.N + rec_lx(r);
            for (int c = lane; c < cells; c += 32) {
                const float2 t = __ldg(R + c);
                const float ti = sg * t.y;
                atomicAdd(g + (int64_t)(c / Sr) * p.N + (c % Sr),
                          make_float2(wr * t.x - wi * ti, wr * ti + wi * t.x));
            }
        }
    }
}

__global__ void __launch_bounds__(kResWarps * 32) degrid_residual_kernel(
    DevParams p, int Sr, int OSr, const WorkItem *__restrict__ items,
    const int32_t *__restrict__ nitems, int32_t *counter, const uint64_t *__restrict__ rec,
    const int32_t *__restrict__ perm, const float2 *__restrict__ grid,
    const float *__restrict__ weight, const float2 *__restrict__ res, float2 *vis_out)
{
    const int lane = threadIdx.x & 31;
    const int n_items = *nitems;
    const int step = p.OS / OSr, k0 = (p.S - Sr) / 2, cells = Sr * Sr;
    for (;;) {
        int item = 0;
        if (lane == 0)
            item = atomicAdd(counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items)
            break;
        const WorkItem it = items[item];
        const TileOrigin o = tile_origin(p, it.tile);
        const float2 *const tg = grid + o.base + (o.gy0 + k0) * p.N + o.gx0 + k0;
        for (int s = it.start; s < it.start + it.count; ++s) {
            const uint64_t r = rec[s];
            const float sg = rec_conj(r) ? 1.f : -1.f;  // conj of the gridding kernel
            const float2 *R = res + (((int64_t)rec_plane(r) * OSr + rec_ov(r) / step) * OSr +
                                     rec_ou(r) / step) * cells;
            const float2 *g = tg + (int64_t)rec_ly(r) * p.N + rec_lx(r);
            float ar = 0.f, ai = 0.f;
            for (int c = lane; c < cells; c += 32) {
                const float2 t = __ldg(R + c);
                const float ti = sg * t.y;
                const float2 x = __ldg(g + (int64_t)(c / Sr) * p.N + (c % Sr));
                ar += t.x * x.x - ti * x.y;
                ai += t.x * x.y + ti * x.x;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                ar += __shfl_xor_sync(0xffffffffu, ar, off);
                ai += __shfl_xor_sync(0xffffffffu, ai, off);
            }
            if (lane == 0) {
                const int i = perm[s];
                const float wt = weight ? __ldg(weight + i) : 1.0f;
                float2 v = vis_out[i];
                v.x += wt * ar;
                v.y += wt * ai;
                vis_out[i] = v;
            }
        }
    }
}

cudaError_t launch_grid_residual(const DevParams &p, int Sr, int OSr, const Plan &plan,
                                 const float2 *vis, const float *weight, const float2 *res,
                                 float2 *grid, int num_sms, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(plan.d_item_counter, 0, sizeof(int32_t), s);
    if (e != cudaSuccess)
        return e;
    grid_residual_kernel<<<num_sms * 4, kResWarps * 32, 0, s>>>(
        p, Sr, OSr, plan.d_items, plan.d_nitems, plan.d_item_counter, plan.d_rec, plan.d_perm,
        vis, weight, res, grid);
    return cudaGetLastError();
}

cudaError_t launch_degrid_residual(const DevParams &p, int Sr, int OSr, const Plan &plan,
                                   const float2 *grid, const float *weight, const float2 *res,
                                   float2 *vis_out, int num_sms, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(plan.d_item_counter + 1, 0, sizeof(int32_t), s);
    if (e != cudaSuccess)
        return e;
    degrid_residual_kernel<<<num_sms * 4, kResWarps * 32, 0, s>>>(
        p, Sr, OSr, plan.d_items, plan.d_nitems, plan.d_item_counter + 1, plan.d_rec,
        plan.d_perm, grid, weight, res, vis_out);
    return cudaGetLastError();
}

}  // namespace sepw
