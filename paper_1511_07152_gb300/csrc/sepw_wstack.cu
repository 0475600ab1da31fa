// Hybrid W stacking (Sec. 4.3): visibilities are partitioned by w into slices;
// each slice's mean w term is corrected in image space by the phase
// exp(2 pi i w_c (n - 1)) of its centre w_c, and the residual w - w_c by the
// separable W-projection kernel of the gridder.
//
// Planning: every visibility gets the slice with the nearest centre (ties to
// the lower centre, distances in IEEE double), then a counting sort by slice
// writes the slice-ordered (u, v, w - w_c) the batched plan is built on; the
// plan's slot -> visibility map is then composed with the sort, so gridding
// and degridding read V, W and write predictions in the caller's order.
//
// Image step: one batched inverse FFT of all slice grids between a sign pass
// and a combine pass that applies the grid correction n / (c c), the slice
// phase and the sum over slices; the prediction direction mirrors it.
#include "sepw_internal.cuh"

namespace sepw {

// Slice of w among the strictly increasing centres c[0..L): the nearest,
// ties to the lower index; non-finite w gets slice 0.
__device__ __forceinline__ int nearest_slice(double w, const double *__restrict__ c, int L)
{
    if (!isfinite(w))
        return 0;
    int lo = 0, hi = L;  // first index with c[j] > w
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (c[mid] > w)
            hi = mid;
        else
            lo = mid + 1;
    }
    int k;
    if (lo == 0)
        k = 0;
    else if (lo == L)
        k = L - 1;
    else
        k = (__dadd_rn(w, -c[lo - 1]) <= __dadd_rn(c[lo], -w)) ? lo - 1 : lo;
    // a lower centre at an equal rounded distance wins the tie
    while (k > 0 && fabs(__dadd_rn(w, -c[k - 1])) == fabs(__dadd_rn(w, -c[k])))
        --k;
    return k;
}

// Slice of every visibility and the slice histogram.  With L <= kSmemSlices
// the block counts in shared memory and adds one global atomic per slice it
// saw (a handful of slices hold most visibilities, so per-visibility global
// atomics would serialise on a few addresses).
constexpr int kWsThreads = 1024;
constexpr int kSmemSlices = 8192;

__global__ void __launch_bounds__(kWsThreads) wstack_assign_kernel(
    int64_t nvis, const double *__restrict__ w, const double *__restrict__ c, int L,
    int32_t *__restrict__ slice, int32_t *count)
{
    extern __shared__ int32_t s_cnt[];
    const bool smem = L <= kSmemSlices;
    if (smem) {
        for (int j = threadIdx.x; j < L; j += blockDim.x)
            s_cnt[j] = 0;
        __syncthreads();
    }
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nvis) {
        const int k = nearest_slice(w[i], c, L);
        slice[i] = k;
        atomicAdd(smem ? s_cnt + k : count + k, 1);
    }
    if (smem) {
        __syncthreads();
        for (int j = threadIdx.x; j < L; j += blockDim.x)
            if (s_cnt[j])
                atomicAdd(count + j, s_cnt[j]);
    }
}

// slice-ordered coordinates with the residual w - w_c; part[slot] = i.  The
// block ranks its visibilities per slice in shared memory and reserves one
// range per slice with a single global atomic.
__global__ void __launch_bounds__(kWsThreads) wstack_scatter_kernel(
    int64_t nvis, const double *__restrict__ u, const double *__restrict__ v,
    const double *__restrict__ w, const double *__restrict__ c, int L,
    const int32_t *__restrict__ slice, int32_t *cursor, int32_t *__restrict__ part,
    double *__restrict__ up, double *__restrict__ vp, double *__restrict__ wp)
{
    extern __shared__ int32_t s_cnt[];  // [L] counts, then [L] bases
    const bool smem = L <= kSmemSlices;
    int32_t *s_base = s_cnt + (smem ? L : 0);
    if (smem) {
        for (int j = threadIdx.x; j < L; j += blockDim.x)
            s_cnt[j] = 0;
        __syncthreads();
    }
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int k = 0, r = 0;
    if (i < nvis) {
        k = slice[i];
        r = atomicAdd(smem ? s_cnt + k : cursor + k, 1);
    }
    if (smem) {
        __syncthreads();
        for (int j = threadIdx.x; j < L; j += blockDim.x)
            if (s_cnt[j])
                s_base[j] = atomicAdd(cursor + j, s_cnt[j]);
        __syncthreads();
        r += s_base[k];
    }
    if (i >= nvis)
        return;
    part[r] = (int32_t)i;
    up[r] = u[i];
    vp[r] = v[i];
    wp[r] = __dadd_rn(w[i], -c[k]);
}

// plan slots and dropped indices refer to the slice order: map them back to
// the caller's visibility indices
__global__ void __launch_bounds__(256) wstack_compose_kernel(
    int64_t nvis, const unsigned long long *__restrict__ dropped,
    const int32_t *__restrict__ part, int32_t *perm, int32_t *drop_list)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nd = (int64_t)*dropped;
    if (i < nvis - nd)
        perm[i] = part[perm[i]];
    if (i < nd)
        drop_list[i] = part[drop_list[i]];
}

cudaError_t launch_wstack_assign(int64_t nvis, const double *w, const double *c, int L,
                                 int32_t *slice, int32_t *count, cudaStream_t s)
{
    if (nvis == 0)
        return cudaSuccess;
    const size_t shm = L <= kSmemSlices ? sizeof(int32_t) * L : 0;
    wstack_assign_kernel<<<(unsigned)((nvis + kWsThreads - 1) / kWsThreads), kWsThreads, shm,
                           s>>>(nvis, w, c, L, slice, count);
    return cudaGetLastError();
}

cudaError_t launch_wstack_scatter(int64_t nvis, const double *u, const double *v,
                                  const double *w, const double *c, int L, const int32_t *slice,
                                  int32_t *cursor, int32_t *part, double *up, double *vp,
                                  double *wp, cudaStream_t s)
{
    if (nvis == 0)
        return cudaSuccess;
    const size_t shm = L <= kSmemSlices ? 2 * sizeof(int32_t) * L : 0;
    if (shm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(wstack_scatter_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)shm);
        if (e != cudaSuccess)
            return e;
    }
    wstack_scatter_kernel<<<(unsigned)((nvis + kWsThreads - 1) / kWsThreads), kWsThreads, shm,
                            s>>>(nvis, u, v, w, c, L, slice, cursor, part, up, vp, wp);
    return cudaGetLastError();
}

cudaError_t launch_wstack_compose(int64_t nvis, const Plan &plan, const int32_t *part,
                                  cudaStream_t s)
{
    if (nvis == 0)
        return cudaSuccess;
    wstack_compose_kernel<<<(unsigned)((nvis + 255) / 256), 256, 0, s>>>(
        nvis, plan.d_dropped, part, plan.d_perm, plan.d_drop_list);
    return cudaGetLastError();
}

// n - 1 without cancellation, and the grid correction factors of pixel (a, b)
// (at l0 + l, m0 + m for a facet centred at (l0, m0))
__device__ __forceinline__ void pixel_terms(int N, float fov_over_n, float l0, float m0,
                                            const float *taper, int a, int b, float &nm1,
                                            float &n, float &cc)
{
    const float l = (float)(a - N / 2) * fov_over_n + l0;
    const float m = (float)(b - N / 2) * fov_over_n + m0;
    const float r2 = l * l + m * m;
    n = sqrtf(1.f - r2);
    nm1 = -r2 / (1.f + n);
    cc = taper[a] * taper[b];
}

// exp(sgn 2 pi i w_c (n - 1)) with the argument reduced to [-1/2, 1/2] turns
__device__ __forceinline__ float2 slice_phase(float wc, float nm1, float sgn)
{
    float x = wc * nm1;
    x -= rintf(x);
    float sn, cs;
    sincospif(2.f * x, &sn, &cs);
    return make_float2(cs, sgn * sn);
}

// checkerboard sign (-1)^(a+b) on every slice grid (the shift of the DFT)
__global__ void wstack_sign_kernel(int N, int L, float2 *g)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (a >= N)
        return;
    if (((a + b) & 1) == 0)
        return;
    const int64_t n2 = (int64_t)N * N;
    for (int c = 0; c < L; ++c) {
        float2 *p = g + c * n2 + (int64_t)b * N + a;
        const float2 x = *p;
        *p = make_float2(-x.x, -x.y);
    }
}

// image = sum_c sign n / (c c) exp(2 pi i w_c (n - 1)) IDFT(grid_c)
__global__ void wstack_combine_kernel(int N, int L, float fov_over_n, float l0, float m0,
                                      const float *taper,
                                      const float *__restrict__ wc, const float2 *__restrict__ g,
                                      float2 *__restrict__ image)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (a >= N)
        return;
    float nm1, n, cc;
    pixel_terms(N, fov_over_n, l0, m0, taper, a, b, nm1, n, cc);
    const float s = (((a + b) & 1) ? -1.f : 1.f) * n / cc;
    const int64_t n2 = (int64_t)N * N, idx = (int64_t)b * N + a;
    float re = 0.f, im = 0.f;
    for (int c = 0; c < L; ++c) {
        const float2 x = g[c * n2 + idx];
        const float2 e = slice_phase(wc[c], nm1, 1.f);
        re += x.x * e.x - x.y * e.y;
        im += x.x * e.y + x.y * e.x;
    }
    image[idx] = make_float2(s * re, s * im);
}

// grid_c (before the forward DFT) = sign / (n c c) exp(-2 pi i w_c (n - 1)) image
__global__ void wstack_split_kernel(int N, int L, float fov_over_n, float l0, float m0,
                                    const float *taper,
                                    const float *__restrict__ wc,
                                    const float2 *__restrict__ image, float2 *__restrict__ g)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (a >= N)
        return;
    float nm1, n, cc;
    pixel_terms(N, fov_over_n, l0, m0, taper, a, b, nm1, n, cc);
    const float s = (((a + b) & 1) ? -1.f : 1.f) / (n * cc);
    const int64_t n2 = (int64_t)N * N, idx = (int64_t)b * N + a;
    const float2 x = image[idx];
    for (int c = 0; c < L; ++c) {
        const float2 e = slice_phase(wc[c], nm1, -1.f);
        g[c * n2 + idx] = make_float2(s * (x.x * e.x - x.y * e.y), s * (x.x * e.y + x.y * e.x));
    }
}

cudaError_t launch_wstack_sign(const DevParams &p, int L, float2 *g, cudaStream_t s)
{
    dim3 grid((p.N + 255) / 256, p.N);
    wstack_sign_kernel<<<grid, 256, 0, s>>>(p.N, L, g);
    return cudaGetLastError();
}

cudaError_t launch_wstack_combine(const DevParams &p, int L, const float *taper,
                                  const float *wc, const float2 *g, float2 *image,
                                  cudaStream_t s)
{
    dim3 grid((p.N + 255) / 256, p.N);
    wstack_combine_kernel<<<grid, 256, 0, s>>>(p.N, L, (float)(p.fov / p.N), (float)p.l0,
                                               (float)p.m0, taper, wc, g, image);
    return cudaGetLastError();
}

cudaError_t launch_wstack_split(const DevParams &p, int L, const float *taper, const float *wc,
                                const float2 *image, float2 *g, cudaStream_t s)
{
    dim3 grid((p.N + 255) / 256, p.N);
    wstack_split_kernel<<<grid, 256, 0, s>>>(p.N, L, (float)(p.fov / p.N), (float)p.l0,
                                             (float)p.m0, taper, wc, image, g);
    return cudaGetLastError();
}

}  // namespace sepw
