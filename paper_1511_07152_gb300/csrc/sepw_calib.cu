// sepw_fma_probe: the FP32 FMA rate of this GPU, measured.
//
// The scatter-form gridder and degridder (tiled FP32) are bound by FP32
// fused multiply-adds, and their roofline is stated against the FMA peak.
// The peak derived from unit counts (SMs x FP32 lanes x 2 flop x clock) is
// checked here against a kernel that does nothing else: every thread runs
// kChains independent FMA chains (scalar FFMA, or paired FFMA2 on float2
// operands), so the pipes never wait on a dependence, and one CTA group per
// SM keeps all of them busy.  The caller times the launch (CUDA events on the
// stream) and divides the flop count this function reports by the time.
#include <cuda_fp16.h>

#include "sepw_internal.cuh"

namespace sepw {
namespace {

constexpr int kChains = 8;     // independent accumulators per thread
constexpr int kThreads = 256;  // threads per CTA
constexpr int kCtasPerSm = 4;

__global__ void __launch_bounds__(kThreads) fma_kernel(int64_t iters, float a, float b,
                                                        float *out)
{
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc[c] = (float)(threadIdx.x + c);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            acc[c] = fmaf(acc[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += acc[c];
    out[blockIdx.x * kThreads + threadIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(kThreads) fma2_kernel(int64_t iters, float a, float b,
                                                         float *out)
{
    float2 acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc[c] = make_float2((float)(threadIdx.x + c), (float)(threadIdx.x - c));
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            acc[c] = __ffma2_rn(acc[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += acc[c].x + acc[c].y;
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace sepw

extern "C" SEPW_API int sepw_fma_probe(int paired, int64_t iters, float *out, int64_t out_len,
                                       int64_t *flops, sepw_stream_t stream)
{
    using namespace sepw;
    if (iters < 1 || iters > ((int64_t)1 << 30) || !out || !flops)
        return SEPW_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SEPW_ECUDA;
    const int64_t ctas = (int64_t)sms * kCtasPerSm;
    if (out_len < ctas * kThreads)
        return SEPW_EINVAL;
    // a, b keep the chains bounded (|a| < 1): no overflow, no denormals
    const float a = 0.999f, b = 0.001f;
    cudaStream_t s = (cudaStream_t)stream;
    if (paired)
        fma2_kernel<<<(unsigned)ctas, kThreads, 0, s>>>(iters, a, b, out);
    else
        fma_kernel<<<(unsigned)ctas, kThreads, 0, s>>>(iters, a, b, out);
    if (cudaGetLastError() != cudaSuccess)
        return SEPW_ECUDA;
    // one FMA = 2 flop; a paired FMA does two
    *flops = ctas * kThreads * iters * kChains * 2 * (paired ? 2 : 1);
    return SEPW_OK;
}
