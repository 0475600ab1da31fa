// Tensor-core (tcgen05) contraction form of the separable gridder.
//
// Sec. 5 writes the update of a visibility as the separable product
// W V F1(u - u_i) F1(v - v_i).  Summed over the n visibilities of one tile
// this is a dense complex contraction: with Bv[i][y] the v-taps of visibility
// i placed at its row offset inside the tile's window and P[i][x] = W_i V_i
// times its u-taps placed at its column offset,
//     G[y][x] = sum_i Bv[i][y] P[i][x]                      (G = Bv^T P).
// In real arithmetic, with K = (visibility, re/im component):
//     [G_r; G_i] (128 x 64) = A (128 x 2n) * B (2n x 64),
//     A[(0,y)][(i,0)] =  Bv_r    A[(0,y)][(i,1)] = -Bv_i
//     A[(1,y)][(i,0)] =  Bv_i    A[(1,y)][(i,1)] =  Bv_r
//     B[(i,0)][x]     =  P_r     B[(i,1)][x]     =  P_i
// which is one tcgen05.mma shape M = 128, N = 64 per K = 16 (8 visibilities).
// The window is 64 x 64 (tile edge T with T + S - 1 <= 64).
//
// Operands: BF16 or FP16 (taps, and W V times the taps), FP32 accumulation in
// tensor memory.  They are built in shared memory in the no-swizzle K-major
// canonical layout (8-row x 16-byte core matrices; K-adjacent cores 128 bytes
// apart, 8-row groups 2048 bytes apart).  Only the non-zero entries of a
// stage are written, and cleared again once the tensor core has consumed the
// stage, so the buffers stay zero elsewhere: each of the 512 producer threads
// owns one (visibility, tap pair) unit of every stage, reads its visibility's
// record itself, and clears its entries of a buffer when the buffer comes
// round again.  Two stages of 64 visibilities are in flight.  Producer warps
// arrive on the stage's "full" mbarrier; a separate warp waits on it, issues
// the MMAs and commits them to the stage's "empty" mbarrier, so no CTA-wide
// barrier is needed inside a work item.
//
// After the last stage of a work item the accumulator is read back with
// tcgen05.ld, staged in shared memory and added to the HBM grid with float2
// atomics (windows overlap).  Every wait on an mbarrier is bounded in time;
// on expiry the kernel records SEPW_ETIMEOUT in the device status word, stops
// issuing work, waits (bounded) for its own MMAs and frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sepw_internal.cuh"

namespace sepw {
namespace {

constexpr int kTcThreads = 512;
constexpr int kStageVis = 64;                 // visibilities per stage (K = 128)
constexpr int kStages = 3;                    // stages in flight
constexpr int kWin = 64;                      // padded window edge
constexpr int kM = 128, kN = 64;              // MMA shape
constexpr int kKStage = 2 * kStageVis;        // K elements per stage
constexpr int kSBO = (kKStage / 8) * 128;     // bytes between 8-row core groups
constexpr int kABytes = kM * kKStage * 2;     // 32 KiB
constexpr int kBBytes = kN * kKStage * 2;     // 16 KiB
constexpr uint32_t kTmemCols = 64;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = globaltimer();
    while (globaltimer() - t0 < kWaitNs)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: no swizzle, K-major canonical layout.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(kSBO >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D = F32, A/B = BF16 (fmt 1) or F16 (0),
// both K-major, N = 64, M = 128.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t ab_fmt)
{
    return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(kN >> 3) << 17) |
           ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

#define SEPW_TMEM_LD32(taddr, r)                                                          \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "                                \
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"                \
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];" \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), \
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]),             \
                   "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),         \
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),         \
                   "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),         \
                   "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),         \
                   "=r"(r[31])                                                              \
                 : "r"(taddr)                                                               \
                 : "memory")

#define SEPW_TMEM_LD16(taddr, r)                                                          \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "                                \
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"          \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), \
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]),             \
                   "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])          \
                 : "r"(taddr)                                                               \
                 : "memory")

template <bool FP16>
__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    if constexpr (FP16) {
        __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

// byte offset of element pair (row, visibility ii) in a stage operand
__device__ __forceinline__ uint32_t op_off(int row, int ii)
{
    return (uint32_t)((row >> 3) * kSBO + (ii >> 2) * 128 + (row & 7) * 16 + (ii & 3) * 4);
}

// One producer thread's unit of a stage: visibility ii = 4 * warp + (lane & 3)
// and the taps k, k + 8 with k = lane >> 2.  The 32 four-byte stores of a
// warp instruction land in 32 distinct banks (row & 7 differs across k,
// ii & 3 across the lane quads).  Rows k and k + 8 are one 8-row core group
// (kSBO bytes) apart, and the second block of A (row + 64) eight groups, so a
// unit needs two offsets: offA = op_off(ly + k, ii), offB = op_off(lx + k, ii).
template <int S, bool FP16>
__device__ __forceinline__ void unit_set(unsigned char *A, unsigned char *B, uint32_t offA,
                                         uint32_t offB, int k, const float2 *tv,
                                         const float2 *tu, float wr, float wi, bool cj)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int kk = k + 8 * h;
        if (kk >= S)
            continue;
        float2 v = __ldg(tv + kk);
        float2 u = __ldg(tu + kk);
        if (cj) {
            v.y = -v.y;
            u.y = -u.y;
        }
        *reinterpret_cast<uint32_t *>(A + offA + h * kSBO) = pack2<FP16>(v.x, -v.y);
        *reinterpret_cast<uint32_t *>(A + offA + (8 + h) * kSBO) = pack2<FP16>(v.y, v.x);
        *reinterpret_cast<uint32_t *>(B + offB + h * kSBO) =
            pack2<FP16>(wr * u.x - wi * u.y, wr * u.y + wi * u.x);
    }
}

template <int S>
__device__ __forceinline__ void unit_clear(unsigned char *A, unsigned char *B, uint32_t offA,
                                           uint32_t offB, int k)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (k + 8 * h >= S)
            continue;
        *reinterpret_cast<uint32_t *>(A + offA + h * kSBO) = 0u;
        *reinterpret_cast<uint32_t *>(A + offA + (8 + h) * kSBO) = 0u;
        *reinterpret_cast<uint32_t *>(B + offB + h * kSBO) = 0u;
    }
}

constexpr int kProducerWarps = kTcThreads / 32;  // 16
constexpr int kTcBlock = kTcThreads + 32;        // + one MMA-issuing warp

template <int S, bool FP16>
__global__ void __launch_bounds__(kTcBlock, 1) grid_tc_kernel(
    DevParams p, const WorkItem *__restrict__ items, const int32_t *__restrict__ nitems,
    int32_t *counter, const uint64_t *__restrict__ rec, const int32_t *__restrict__ perm,
    const float2 *__restrict__ vis, const float *__restrict__ weight,
    const float2 *__restrict__ taps, float2 *grid, int32_t *status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Abuf = smem;                      // kStages x 32 KiB
    unsigned char *Bbuf = smem + kStages * kABytes;  // kStages x 16 KiB
    uint64_t *full = reinterpret_cast<uint64_t *>(Bbuf + kStages * kBBytes);
    uint64_t *empty = full + kStages;
    uint64_t *accf = empty + kStages;
    __shared__ uint32_t s_tmem;
    __shared__ int s_item;
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == kProducerWarps;
    constexpr uint32_t idesc = instr_desc(FP16 ? 0u : 1u);

    for (int e = tid; e < kStages * (kABytes + kBBytes) / 16; e += kTcBlock)
        reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int b = 0; b < kStages; ++b) {
            mbar_init(full + b, kProducerWarps);
            mbar_init(empty + b, 1);
        }
        mbar_init(accf, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const int n_items = *nitems;

    // producer unit of this thread; operand offsets of its last two stages
    // (0xffffffff: nothing written) for the clears
    const int ii = 4 * warp + (lane & 3);
    const int k = lane >> 2;
    uint32_t oldA[kStages], oldB[kStages];
#pragma unroll
    for (int q = 0; q < kStages; ++q) {
        oldA[q] = 0xffffffffu;
        oldB[q] = 0;
    }

    int t_global = 0;  // stages of this CTA so far (buffer t % kStages)
    int n_done = 0;    // items of this CTA so far (accf parity)

    for (;;) {
        if (tid == 0)
            s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items || s_abort)
            break;
        const WorkItem it = items[item];
        const int nst = (it.count + kStageVis - 1) / kStageVis;

        if (!mma_warp) {
            // records of the unit's visibility, one stage ahead
            uint64_t r_next = 0;
            int i_next = -1;
            if (ii < it.count) {
                r_next = rec[it.start + ii];
                i_next = perm[it.start + ii];
            }
            for (int st = 0; st < nst; ++st) {
                const int t = t_global + st;
                const int b = t % kStages;
                unsigned char *A = Abuf + b * kABytes;
                unsigned char *B = Bbuf + b * kBBytes;
                const uint64_t r = r_next;
                const int i = i_next;
                float2 x = make_float2(0.f, 0.f);
                float wt = 1.0f;
                if (i >= 0) {
                    x = __ldg(vis + i);
                    if (weight)
                        wt = __ldg(weight + i);
                }
                const int vn = it.start + (st + 1) * kStageVis + ii;
                i_next = -1;
                if (st + 1 < nst && vn < it.start + it.count) {
                    r_next = rec[vn];
                    i_next = perm[vn];
                }
                uint32_t pa = 0xffffffffu, pb = 0;
#pragma unroll
                for (int q = 0; q < kStages; ++q)
                    if (q == b) {
                        pa = oldA[q];
                        pb = oldB[q];
                    }
                if (t >= kStages) {
                    // buffer b held stage t - kStages: wait (lane 0) for its
                    // MMAs, then clear the entries this unit wrote there
                    if (lane == 0 && !s_abort &&
                        !mbar_wait(empty + b, ((t - kStages) / kStages) & 1))
                        s_abort = 1;
                    __syncwarp();
                    tc_fence_after();
                    if (pa != 0xffffffffu)
                        unit_clear<S>(A, B, pa, pb, k);
                }
                pa = 0xffffffffu;
                if (i >= 0) {
                    const int row = rec_plane(r) * p.OS;
                    const uint32_t offA = op_off(rec_ly(r) + k, ii);
                    const uint32_t offB = op_off(rec_lx(r) + k, ii);
                    unit_set<S, FP16>(A, B, offA, offB, k, taps + (row + rec_ov(r)) * S,
                                      taps + (row + rec_ou(r)) * S, wt * x.x, wt * x.y,
                                      rec_conj(r));
                    pa = offA;
                    pb = offB;
                }
#pragma unroll
                for (int q = 0; q < kStages; ++q)
                    if (q == b) {
                        oldA[q] = pa;
                        oldB[q] = pb;
                    }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                     smem_u32(full + b))
                                 : "memory");
            }
        } else if (lane == 0) {
            for (int st = 0; st < nst; ++st) {
                const int t = t_global + st;
                const int b = t % kStages;
                if (!s_abort && !mbar_wait(full + b, (t / kStages) & 1))
                    s_abort = 1;
                if (s_abort)
                    continue;
                tc_fence_after();
                const int v0 = it.start + st * kStageVis;
                const int nv = min(kStageVis, it.start + it.count - v0);
                const uint32_t a0 = smem_u32(Abuf + b * kABytes);
                const uint32_t b0 = smem_u32(Bbuf + b * kBBytes);
                const int nk = (nv + 7) / 8;  // K = 16 steps holding visibilities
                for (int q = 0; q < nk; ++q)
                    mma_f16(tmem, smem_desc(a0 + 256 * q), smem_desc(b0 + 256 * q), idesc,
                            (st > 0 || q > 0) ? 1u : 0u);
                mma_commit(empty + b);
            }
            if (!s_abort)
                mma_commit(accf);
        }
        t_global += nst;

        // epilogue: wait for the accumulator, TMEM -> shared staging (the B
        // buffers, re-zeroed afterwards) -> float2 atomics into the HBM grid
        if (lane == 0 && !s_abort && !mbar_wait(accf, n_done & 1))
            s_abort = 1;
        __syncwarp();
        ++n_done;
        tc_fence_after();
        float *stg = reinterpret_cast<float *>(Bbuf);  // [128][64], xor-swizzled
        if (!mma_warp && !s_abort) {
            const int q = warp & 3, h = warp >> 2;  // lane quarter, 16-column group
            const int m = 32 * q + lane;
            uint32_t r[16];
            SEPW_TMEM_LD16(tmem + ((uint32_t)(32 * q) << 16) + 16 * h, r);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int x = 16 * h + c;
                stg[m * kWin + (x ^ (m & 31))] = __uint_as_float(r[c]);
            }
        }
        tc_fence_before();
        __syncthreads();
        if (!s_abort) {
            const int W = p.T + S - 1;
            const TileOrigin o = tile_origin(p, it.tile);
            for (int e = tid; e < W * kWin; e += kTcBlock) {
                const int y = e >> 6, x = e & 63;
                if (x >= W)
                    continue;
                const float re = stg[y * kWin + (x ^ (y & 31))];
                const float im = stg[(kWin + y) * kWin + (x ^ ((kWin + y) & 31))];
                if (re != 0.f || im != 0.f)
                    atomicAdd(grid + o.base + (o.gy0 + y) * p.N + o.gx0 + x,
                              make_float2(re, im));
            }
        }
        __syncthreads();
        for (int e = tid; e < kStages * kBBytes / 16; e += kTcBlock)
            reinterpret_cast<uint4 *>(Bbuf)[e] = make_uint4(0, 0, 0, 0);
        fence_proxy_async();
    }

    if (s_abort) {
        if (tid == 0)
            atomicExch(status, SEPW_ETIMEOUT);
        // bounded wait for this CTA's own MMAs before releasing TMEM
        if (mma_warp && lane == 0 && n_done > 0)
            mbar_wait(accf, (n_done - 1) & 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
}

size_t tc_smem_bytes()
{
    return (size_t)kStages * (kABytes + kBBytes) + sizeof(uint64_t) * (2 * kStages + 1);
}

template <int S, bool FP16>
cudaError_t launch_tc_S(const DevParams &p, const Plan &plan, const float2 *vis,
                        const float *weight, const float2 *taps, float2 *grid, int num_sms,
                        int32_t *status, cudaStream_t s)
{
    const size_t shm = tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(grid_tc_kernel<S, FP16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess)
        return e;
    e = cudaMemsetAsync(plan.d_item_counter, 0, sizeof(int32_t), s);
    if (e != cudaSuccess)
        return e;
    grid_tc_kernel<S, FP16><<<num_sms, kTcBlock, shm, s>>>(
        p, plan.d_items, plan.d_nitems, plan.d_item_counter, plan.d_rec, plan.d_perm, vis,
        weight, taps, grid, status);
    return cudaGetLastError();
}

}  // namespace

int tc_tile_for_support(int S)
{
    int T = kWin - S + 1;
    return T & ~1;
}

cudaError_t launch_grid_tc(const DevParams &p, const Plan &plan, const float2 *vis,
                           const float *weight, const float2 *taps, float2 *grid,
                           int num_sms, bool fp16, int32_t *status, cudaStream_t s)
{
    if (p.T + p.S - 1 > kWin)
        return cudaErrorInvalidValue;
#define SEPW_TC_CASE(SS)                                                                   \
    case SS:                                                                               \
        return fp16 ? launch_tc_S<SS, true>(p, plan, vis, weight, taps, grid, num_sms,     \
                                            status, s)                                     \
                    : launch_tc_S<SS, false>(p, plan, vis, weight, taps, grid, num_sms,    \
                                             status, s);
    switch (p.S) {
        SEPW_TC_CASE(2) SEPW_TC_CASE(4) SEPW_TC_CASE(6) SEPW_TC_CASE(8) SEPW_TC_CASE(10)
        SEPW_TC_CASE(12) SEPW_TC_CASE(14) SEPW_TC_CASE(16)
    default:
        return cudaErrorInvalidValue;
    }
#undef SEPW_TC_CASE
}

}  // namespace sepw
