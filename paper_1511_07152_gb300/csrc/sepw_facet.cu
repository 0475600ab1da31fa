// Image-plane faceting (Sec. 4.1): the visibilities of a facet centred at
// (l0, m0).  The linear term of the Taylor expansion of h about the facet
// centre is absorbed by u' = u - w l0 / n0, v' = v - w m0 / n0 (IEEE double,
// each operation rounded, in this order, so that locating u' agrees with the
// FP64 oracle bit for bit), and the phase centre moves to the facet centre:
// V' = V exp(2 pi i (u l0 + v m0 + w (n0 - 1))) (out of the facet: the
// conjugate phase).  The phase is summed in FP64, reduced to [-1/2, 1/2]
// turns, and applied in FP32.
#include "sepw_internal.cuh"

namespace sepw {

__global__ void __launch_bounds__(256) facet_shift_kernel(
    int64_t nvis, double l0, double m0, double n0, float sgn, const double *__restrict__ u,
    const double *__restrict__ v, const double *__restrict__ w, const float2 *__restrict__ vin,
    double *__restrict__ uo, double *__restrict__ vo, float2 *__restrict__ vout)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvis)
        return;
    const double ui = u[i], vi = v[i], wi = w[i];
    if (uo) {
        uo[i] = __dadd_rn(ui, -__ddiv_rn(__dmul_rn(wi, l0), n0));
        vo[i] = __dadd_rn(vi, -__ddiv_rn(__dmul_rn(wi, m0), n0));
    }
    if (vout) {
        double ph = __dadd_rn(__dadd_rn(__dmul_rn(ui, l0), __dmul_rn(vi, m0)),
                              __dmul_rn(wi, n0 - 1.0));
        ph -= rint(ph);
        float s, c;
        sincospif(2.f * (float)ph, &s, &c);
        s *= sgn;
        const float2 x = vin[i];
        vout[i] = make_float2(x.x * c - x.y * s, x.x * s + x.y * c);
    }
}

cudaError_t launch_facet_shift(int64_t nvis, double l0, double m0, int direction,
                               const double *u, const double *v, const double *w,
                               const float2 *vin, double *uo, double *vo, float2 *vout,
                               cudaStream_t s)
{
    if (nvis == 0)
        return cudaSuccess;
    const double n0 = sqrt(1.0 - l0 * l0 - m0 * m0);
    facet_shift_kernel<<<(unsigned)((nvis + 255) / 256), 256, 0, s>>>(
        nvis, l0, m0, n0, direction == 0 ? 1.f : -1.f, u, v, w, vin, uo, vo, vout);
    return cudaGetLastError();
}

}  // namespace sepw
