// 1-D GCF table generation in float64 (Eq. gt; Sec. 2: the GCF is the
// Fourier transform of the antialiasing taper times the w screen).
//
//   taps[p][o][j] = F1_{w_p}(d),  d = j - S/2 + 1 - o/OS
//   F1_w(d) = (1/N) sum_a c1(nu_a) g1_w(l_a) exp(-2 pi i d nu_a)
//
// The DFT phase d*nu_a = k (a - N/2) / (N OS) with the integer k = d*OS, so it
// is reduced exactly in integers and looked up in a table of N*OS twiddles
// exp(-2 pi i m / (N OS)), each computed once with sincospi.  The screen
// g1_w(l) = exp(2 pi i w (-l^2/2 - gamma l^4)) (or a facet screen of Eq.
// gt-facet, Sec. 4.1) is evaluated once per pixel and plane.  Off the hot
// path.
#include "sepw_internal.cuh"

namespace sepw {

// c1(nu): Kaiser-Bessel window transform S sinh(z)/z, z = sqrt(beta^2 -
// (pi S nu)^2) (sin form for imaginary z), normalised to c1(0) = 1 and
// evaluated without overflow.
__device__ double kb_taper_dev(double nu, int S, double beta)
{
    const double pi = 3.141592653589793238462643383279502884;
    double x = pi * (double)S * nu;
    double z2 = beta * beta - x * x;
    double den = -expm1(-2.0 * beta);
    if (z2 > 0.0) {
        double z = sqrt(z2);
        return (beta / z) * exp(z - beta) * (-expm1(-2.0 * z)) / den;
    }
    if (z2 < 0.0) {
        double z = sqrt(-z2);
        return (beta / z) * sin(z) * 2.0 * exp(-beta) / den;
    }
    return beta * 2.0 * exp(-beta) / den;
}

__global__ void taper_kernel(DevParams p, double *taper64, float *taper32)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= p.N)
        return;
    double nu = (double)(a - p.N / 2) / (double)p.N;
    double c = kb_taper_dev(nu, p.S, p.beta);
    taper64[a] = c;
    taper32[a] = (float)c;
}

__global__ void twiddle_kernel(int64_t M, double2 *tw)
{
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M)
        return;
    double s, c;
    sincospi(2.0 * (double)m / (double)M, &s, &c);
    tw[m] = make_double2(c, -s);  // exp(-2 pi i m / M)
}

constexpr int kTapWarps = 8;
constexpr int kTapsPerWarp = 4;
constexpr int kTapsPerBlock = kTapWarps * kTapsPerWarp;
constexpr int kPixChunk = 1024;

// grid = (ceil(OS*S / 32), P, tables); block = 256 threads.  Table 0 is the
// u-direction table (the only one unless p.facet), table 1 the v-direction
// table of a facet; the screen is exp(2 pi i w (a2 l^2 + a4 l^4)) with
// (a2, a4) = (-1/2, -gamma) (Eq. gt) or (a2u or a2v, 0) (Eq. gt-facet).
__global__ void __launch_bounds__(256) taps_kernel(DevParams p, const double *taper64,
                                                   const double2 *tw, double2 *out64,
                                                   float2 *out32)
{
    __shared__ double2 h[kPixChunk];
    const int plane = blockIdx.y;
    const int table = blockIdx.z;
    const double a2 = p.facet ? (table ? p.a2v : p.a2u) : -0.5;
    const double a4 = p.facet ? 0.0 : -p.gamma;
    const int ntap = p.OS * p.S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t M = (int64_t)p.N * p.OS;
    const double wp = p.P > 1 ? (double)plane * p.w_max / (double)(p.P - 1) : 0.0;

    int kk[kTapsPerWarp];
    bool valid[kTapsPerWarp];
    double2 acc[kTapsPerWarp];
#pragma unroll
    for (int q = 0; q < kTapsPerWarp; ++q) {
        int t = blockIdx.x * kTapsPerBlock + warp * kTapsPerWarp + q;
        valid[q] = t < ntap;
        int o = valid[q] ? t / p.S : 0;
        int j = valid[q] ? t % p.S : 0;
        kk[q] = (j - p.S / 2 + 1) * p.OS - o;  // d * OS
        acc[q] = make_double2(0.0, 0.0);
    }

    for (int a0 = 0; a0 < p.N; a0 += kPixChunk) {
        __syncthreads();
        for (int i = threadIdx.x; i < kPixChunk; i += blockDim.x) {
            int a = a0 + i;
            double2 hv = make_double2(0.0, 0.0);
            if (a < p.N) {
                double nu = (double)(a - p.N / 2) / (double)p.N;
                double l = nu * p.fov;
                double l2 = l * l;
                double turns = wp * (a2 * l2 + a4 * l2 * l2);
                double s, c;
                sincospi(2.0 * turns, &s, &c);
                double t = taper64[a];
                hv = make_double2(t * c, t * s);
            }
            h[i] = hv;
        }
        __syncthreads();
        int lim = min(kPixChunk, p.N - a0);
        for (int i = lane; i < lim; i += 32) {
            int64_t ac = (int64_t)(a0 + i) - p.N / 2;
            double2 hv = h[i];
#pragma unroll
            for (int q = 0; q < kTapsPerWarp; ++q) {
                int64_t m = ((int64_t)kk[q] * ac) % M;
                if (m < 0)
                    m += M;
                double2 e = tw[m];
                acc[q].x += hv.x * e.x - hv.y * e.y;
                acc[q].y += hv.x * e.y + hv.y * e.x;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kTapsPerWarp; ++q) {
        double re = acc[q].x, im = acc[q].y;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, off);
            im += __shfl_xor_sync(0xffffffffu, im, off);
        }
        if (lane == 0 && valid[q]) {
            int t = blockIdx.x * kTapsPerBlock + warp * kTapsPerWarp + q;
            int64_t idx = ((int64_t)table * p.P + plane) * ntap + t;
            double2 v = make_double2(re / (double)p.N, im / (double)p.N);
            if (out64)
                out64[idx] = v;
            if (out32)
                out32[idx] = make_float2((float)v.x, (float)v.y);
        }
    }
}

cudaError_t launch_taper(const DevParams &p, double *taper64, float *taper32,
                         cudaStream_t s)
{
    taper_kernel<<<(p.N + 255) / 256, 256, 0, s>>>(p, taper64, taper32);
    return cudaGetLastError();
}

cudaError_t launch_twiddles(const DevParams &p, double2 *tw, cudaStream_t s)
{
    int64_t M = (int64_t)p.N * p.OS;
    twiddle_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(M, tw);
    return cudaGetLastError();
}

cudaError_t launch_taps(const DevParams &p, const double *taper64, const double2 *tw,
                        double2 *out64, float2 *out32, cudaStream_t s)
{
    dim3 grid((p.OS * p.S + kTapsPerBlock - 1) / kTapsPerBlock, p.P, p.facet ? 2 : 1);
    taps_kernel<<<grid, 256, 0, s>>>(p, taper64, tw, out64, out32);
    return cudaGetLastError();
}

}  // namespace sepw
