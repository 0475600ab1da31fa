// Image step with grid correction (Sec. 2: I_D / n = F^-1[grid] / c), around
// an in-place cuFFT C2C transform of the N x N buffer.
//
// With the u = 0 column at N/2, the shifted transform
//   sum_c G[c] exp(2 pi i (c - N/2)(a - N/2) / N)
// equals (-1)^a times the unshifted inverse DFT of (-1)^c G[c] (N even), so
// both shifts become checkerboard sign flips folded into the pre- and
// post-scaling passes:
//   GRID_TO_IMAGE:  buf *= (-1)^(a+b);  inverse FFT;  buf *= (-1)^(a+b) n/(c c)
//   IMAGE_TO_GRID:  buf *= (-1)^(a+b)/(n c c);  forward FFT;  buf *= (-1)^(a+b)
//   IMAGE_TO_GRID_ADJOINT:
//                   buf *= (-1)^(a+b);  inverse FFT;  buf *= (-1)^(a+b)/(n c c)
#include "sepw_internal.cuh"

namespace sepw {

// mode: 0 = sign only, 1 = sign * n / (c_a c_b), 2 = sign / (n c_a c_b)
// (l0, m0): facet centre (Sec. 4.1), n is taken at the pixel's position
// l0 + l, m0 + m in the original image plane
__global__ void image_scale_kernel(int N, float fov_over_n, float l0, float m0,
                                   const float *__restrict__ taper, float2 *buf, int mode)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (a >= N)
        return;
    float s = ((a + b) & 1) ? -1.f : 1.f;
    if (mode != 0) {
        const float l = (float)(a - N / 2) * fov_over_n + l0;
        const float m = (float)(b - N / 2) * fov_over_n + m0;
        const float n = sqrtf(1.f - (l * l + m * m));
        const float cc = taper[a] * taper[b];
        s = mode == 1 ? s * n / cc : s / (n * cc);
    }
    const int64_t idx = (int64_t)b * N + a;
    float2 x = buf[idx];
    buf[idx] = make_float2(x.x * s, x.y * s);
}

static cudaError_t scale(const DevParams &p, int mode, const float *taper, float2 *buf,
                         cudaStream_t s)
{
    dim3 grid((p.N + 255) / 256, p.N);
    image_scale_kernel<<<grid, 256, 0, s>>>(p.N, (float)(p.fov / p.N), (float)p.l0,
                                            (float)p.m0, taper, buf, mode);
    return cudaGetLastError();
}

// The inverse transform (GRID_TO_IMAGE and the adjoint of IMAGE_TO_GRID)
// scales after the FFT; the forward transform (IMAGE_TO_GRID) before it.
cudaError_t launch_image_pre(const DevParams &p, int direction, const float *taper,
                             float2 *buf, cudaStream_t s)
{
    return scale(p, direction == SEPW_IMAGE_TO_GRID ? 2 : 0, taper, buf, s);
}

cudaError_t launch_image_post(const DevParams &p, int direction, const float *taper,
                              float2 *buf, cudaStream_t s)
{
    if (direction == SEPW_GRID_TO_IMAGE)
        return scale(p, 1, taper, buf, s);
    if (direction == SEPW_IMAGE_TO_GRID_ADJOINT)
        return scale(p, 2, taper, buf, s);
    return scale(p, 0, taper, buf, s);
}

}  // namespace sepw
