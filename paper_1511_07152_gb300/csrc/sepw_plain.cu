// Locate kernel and the plain FP32 gridder / degridder.
//
// The plain form is the straightforward scatter/gather of Sec. 5: each
// visibility forms its partial products W V F1(u - u_i) once per footprint
// column and updates every cell of its S x S footprint directly in the HBM
// grid with a float2 atomic add (degridding: reads the footprint from HBM).
// No binning, no reuse across visibilities: the in-library comparator for the
// tiled forms.
#include "sepw_internal.cuh"

namespace sepw {

__global__ void locate_kernel(DevParams p, int64_t nvis, const double *__restrict__ u,
                              const double *__restrict__ v, const double *__restrict__ w,
                              int32_t *cu, int32_t *cv, int32_t *ou, int32_t *ov,
                              int32_t *plane, uint8_t *conj, uint8_t *keep)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvis)
        return;
    Loc L = locate(u[i], v[i], w[i], p);
    if (cu) cu[i] = L.cu;
    if (cv) cv[i] = L.cv;
    if (ou) ou[i] = L.ou;
    if (ov) ov[i] = L.ov;
    if (plane) plane[i] = L.plane;
    if (conj) conj[i] = L.conj ? 1 : 0;
    if (keep) keep[i] = L.keep ? 1 : 0;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Block = 256 threads = VB visibilities x S columns (VB = 256 / S).
__global__ void __launch_bounds__(256) grid_plain_kernel(
    DevParams p, int64_t nvis, const double *__restrict__ u, const double *__restrict__ v,
    const double *__restrict__ w, const float2 *__restrict__ vis,
    const float *__restrict__ weight, const float2 *__restrict__ taps, float2 *grid,
    unsigned long long *dropped)
{
    __shared__ Loc sloc[256];
    __shared__ float2 swv[256];
    const int S = p.S;
    const int VB = 256 / S;
    const int64_t base = (int64_t)blockIdx.x * VB;
    int t = threadIdx.x;
    if (t < VB) {
        int64_t i = base + t;
        Loc L;
        L.keep = false;
        float2 wv = make_float2(0.f, 0.f);
        if (i < nvis) {
            L = locate(u[i], v[i], w[i], p);
            if (!L.keep && dropped)
                atomicAdd(dropped, 1ull);
            float wt = weight ? weight[i] : 1.0f;
            float2 x = vis[i];
            wv = make_float2(wt * x.x, wt * x.y);
        }
        sloc[t] = L;
        swv[t] = wv;
    }
    __syncthreads();
    int vs = t / S, j = t % S;
    if (vs >= VB)
        return;
    Loc L = sloc[vs];
    if (!L.keep)
        return;
    const float2 *tu = taps + ((int64_t)L.plane * p.OS + L.ou) * S;
    const float2 *tv = taps + p.voff + ((int64_t)L.plane * p.OS + L.ov) * S;
    float sg = L.conj ? -1.f : 1.f;
    float2 a = __ldg(tu + j);
    a.y *= sg;
    float2 pu = cmul(swv[vs], a);
    int64_t x = L.cu - S / 2 + 1 + j;
    int64_t y0 = L.cv - S / 2 + 1;
    for (int k = 0; k < S; ++k) {
        float2 b = __ldg(tv + k);
        b.y *= sg;
        atomicAdd(grid + (y0 + k) * p.N + x, cmul(pu, b));
    }
}

__global__ void __launch_bounds__(256) degrid_plain_kernel(
    DevParams p, int64_t nvis, const double *__restrict__ u, const double *__restrict__ v,
    const double *__restrict__ w, const float2 *__restrict__ grid,
    const float *__restrict__ weight, const float2 *__restrict__ taps,
    float2 *__restrict__ vis, unsigned long long *dropped)
{
    __shared__ Loc sloc[256];
    __shared__ float2 part[256];
    const int S = p.S;
    const int VB = 256 / S;
    const int64_t base = (int64_t)blockIdx.x * VB;
    int t = threadIdx.x;
    if (t < VB) {
        int64_t i = base + t;
        Loc L;
        L.keep = false;
        if (i < nvis) {
            L = locate(u[i], v[i], w[i], p);
            if (!L.keep && dropped)
                atomicAdd(dropped, 1ull);
        }
        sloc[t] = L;
    }
    __syncthreads();
    int vs = t / S, j = t % S;
    float2 acc = make_float2(0.f, 0.f);
    if (vs < VB) {
        Loc L = sloc[vs];
        if (L.keep) {
            const float2 *tu = taps + ((int64_t)L.plane * p.OS + L.ou) * S;
            const float2 *tv = taps + p.voff + ((int64_t)L.plane * p.OS + L.ov) * S;
            // conj of the gridding kernel: conj(tap) if w >= 0, tap if w < 0
            float sg = L.conj ? 1.f : -1.f;
            int64_t x = L.cu - S / 2 + 1 + j;
            int64_t y0 = L.cv - S / 2 + 1;
            for (int k = 0; k < S; ++k) {
                float2 b = __ldg(tv + k);
                b.y *= sg;
                float2 g = __ldg(grid + (y0 + k) * p.N + x);
                float2 m = cmul(b, g);
                acc.x += m.x;
                acc.y += m.y;
            }
            float2 a = __ldg(tu + j);
            a.y *= sg;
            acc = cmul(acc, a);
        }
    }
    part[t] = acc;
    __syncthreads();
    if (t < VB) {
        int64_t i = base + t;
        if (i < nvis) {
            float2 s = make_float2(0.f, 0.f);
            for (int jj = 0; jj < S; ++jj) {
                s.x += part[t * S + jj].x;
                s.y += part[t * S + jj].y;
            }
            float wt = weight ? weight[i] : 1.0f;
            vis[i] = make_float2(wt * s.x, wt * s.y);
        }
    }
}

// Number of visibilities that locate() drops (plain-form plans).
__global__ void count_dropped_kernel(DevParams p, int64_t nvis, const double *__restrict__ u,
                                     const double *__restrict__ v,
                                     const double *__restrict__ w,
                                     unsigned long long *dropped)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool drop = i < nvis && !locate(u[i], v[i], w[i], p).keep;
    unsigned m = __ballot_sync(0xffffffffu, drop);
    if (m && (threadIdx.x & 31) == __ffs(m) - 1)
        atomicAdd(dropped, (unsigned long long)__popc(m));
}

cudaError_t launch_count_dropped(const DevParams &p, int64_t nvis, const double *u,
                                 const double *v, const double *w,
                                 unsigned long long *dropped, cudaStream_t s)
{
    if (nvis == 0)
        return cudaSuccess;
    count_dropped_kernel<<<(unsigned)((nvis + 255) / 256), 256, 0, s>>>(p, nvis, u, v, w,
                                                                         dropped);
    return cudaGetLastError();
}

cudaError_t launch_locate(const DevParams &p, int64_t nvis, const double *u,
                          const double *v, const double *w, int32_t *cu, int32_t *cv,
                          int32_t *ou, int32_t *ov, int32_t *plane, uint8_t *conj,
                          uint8_t *keep, cudaStream_t s)
{
    if (nvis == 0)
        return cudaSuccess;
    locate_kernel<<<(unsigned)((nvis + 255) / 256), 256, 0, s>>>(
        p, nvis, u, v, w, cu, cv, ou, ov, plane, conj, keep);
    return cudaGetLastError();
}

cudaError_t launch_grid_plain(const DevParams &p, int64_t nvis, const double *u,
                              const double *v, const double *w, const float2 *vis,
                              const float *weight, const float2 *taps, float2 *grid,
                              unsigned long long *dropped, cudaStream_t s)
{
    if (nvis == 0)
        return cudaSuccess;
    int VB = 256 / p.S;
    grid_plain_kernel<<<(unsigned)((nvis + VB - 1) / VB), 256, 0, s>>>(
        p, nvis, u, v, w, vis, weight, taps, grid, dropped);
    return cudaGetLastError();
}

cudaError_t launch_degrid_plain(const DevParams &p, int64_t nvis, const double *u,
                                const double *v, const double *w, const float2 *grid,
                                const float *weight, const float2 *taps, float2 *vis,
                                unsigned long long *dropped, cudaStream_t s)
{
    if (nvis == 0)
        return cudaSuccess;
    int VB = 256 / p.S;
    degrid_plain_kernel<<<(unsigned)((nvis + VB - 1) / VB), 256, 0, s>>>(
        p, nvis, u, v, w, grid, weight, taps, vis, dropped);
    return cudaGetLastError();
}

}  // namespace sepw
