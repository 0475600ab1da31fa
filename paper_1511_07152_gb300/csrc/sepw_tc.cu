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
// Operand precisions (FP32 accumulation in tensor memory throughout):
//   * BF16: one product per K step;
//   * FP16: one product, with a power-of-two scale 2^-a per work item on B
//     so that the largest |W V| of the item is below 1 (FP16's range), and
//     2^a applied to the accumulator when it is read back;
//   * FP16 hi + lo: each operand x is split into hi = fp16(x) and
//     lo = fp16(x - hi) (22 significant bits together) and the tile update
//     takes the three products hi*hi + hi*lo + lo*hi, scaled as for FP16.
//     The dropped lo*lo term and the two roundings leave about 2^-21 of the
//     largest operand in each product: FP32-class accuracy.
//
// The operands are built in shared memory in the no-swizzle K-major canonical
// layout.  Only the non-zero entries of a stage are written, and cleared
// again once the tensor core has consumed the stage, so the buffers stay zero
// elsewhere.  Eight producer threads share a visibility (taps k = q, q + 8):
// each reads the record, loads its taps, forms its part of P and writes its
// entries; the 32 four-byte stores of a warp instruction (four visibilities,
// eight consecutive rows each) land in 32 distinct banks.  Producer warps arrive on the
// stage's "full" mbarrier; a separate warp waits on it, issues the MMAs and
// commits them to the stage's "empty" mbarrier, so no CTA-wide barrier is
// needed inside a work item.
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

constexpr int kProducers = 512;                 // 16 warps, 8 threads per visibility
constexpr int kProducerWarps = kProducers / 32;
constexpr int kTcBlock = kProducers + 32;       // + one MMA-issuing warp
constexpr int kStageVis = kProducers / 8;       // 64 visibilities per stage
constexpr int kWin = 64;                        // padded window edge
constexpr int kM = 128, kN = 64;                // MMA shape
constexpr int kKStage = 2 * kStageVis;          // K elements per stage
constexpr int kSBO = (kKStage / 8) * 128;       // bytes between 8-row core groups
constexpr int kABytes = kM * kKStage * 2;       // 32 KiB
constexpr int kBBytes = kN * kKStage * 2;       // 16 KiB
constexpr uint32_t kTmemCols = 64;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

// PREC: 0 = BF16, 1 = FP16, 2 = FP16 hi + lo
template <int PREC>
struct Prec {
    static constexpr int TERMS = PREC == 2 ? 2 : 1;   // operand copies (hi, lo)
    static constexpr int STAGES = PREC == 2 ? 2 : 3;  // stages in flight
    static constexpr bool SCALED = PREC != 0;         // per-item power-of-two scale
};

template <int PREC>
constexpr size_t tc_smem_bytes_for()
{
    return (size_t)Prec<PREC>::STAGES * Prec<PREC>::TERMS * (kABytes + kBBytes) +
           sizeof(uint64_t) * (2 * Prec<PREC>::STAGES + 1);
}

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

// Shared-memory matrix descriptor: no swizzle, K-major canonical layout
// (K-adjacent core matrices 128 bytes apart, 8-row groups kSBO bytes apart).
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

// Packs (x, y) for an operand: the rounded pair, and for the split form the
// rounded remainder.
template <int PREC>
__device__ __forceinline__ void split2(float x, float y, uint32_t &hi, uint32_t &lo)
{
    if constexpr (PREC == 0) {
        __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
        hi = *reinterpret_cast<uint32_t *>(&h);
        lo = 0u;
    } else {
        __half2 h = __floats2half2_rn(x, y);
        hi = *reinterpret_cast<uint32_t *>(&h);
        if constexpr (PREC == 2) {
            const float2 f = __half22float2(h);
            __half2 l = __floats2half2_rn(x - f.x, y - f.y);
            lo = *reinterpret_cast<uint32_t *>(&l);
        } else {
            lo = 0u;
        }
    }
}

// (a, b) -> (a, -b) and (b, a) on packed 16-bit pairs (sign flip is exact)
__device__ __forceinline__ uint32_t pair_conj(uint32_t v) { return v ^ 0x80000000u; }
__device__ __forceinline__ uint32_t pair_swap(uint32_t v) { return (v >> 16) | (v << 16); }

// byte offset of the element pair of visibility ii in operand row `row`
__device__ __forceinline__ uint32_t op_off(int row, int ii)
{
    return (uint32_t)((row >> 3) * kSBO + (ii >> 2) * 128 + (row & 7) * 16 + (ii & 3) * 4);
}

// What a producer thread holds of one stage: its visibility's value and
// weight, its taps, and the footprint origin (ly | lx << 8 | conj << 16), or
// pos = -1 for no visibility.
template <int NT>
struct StageData {
    int pos;
    float2 x;
    float wt;
    float2 tv[NT], tu[NT];
};

// Byte offsets of the rows r0, r0 + 8 (visibility ii): a step of 8 rows is
// one core group, kSBO bytes.
template <int NT>
__device__ __forceinline__ void row_offsets(int r0, int ii, uint32_t (&o)[NT])
{
    const uint32_t o0 = op_off(r0, ii);
#pragma unroll
    for (int j = 0; j < NT; ++j)
        o[j] = o0 + j * kSBO;
}

template <int S, int PREC>
__global__ void __launch_bounds__(kTcBlock, 1) grid_tc_kernel(
    DevParams p, const WorkItem *__restrict__ items, const int32_t *__restrict__ nitems,
    int32_t *counter, const uint64_t *__restrict__ rec, const int32_t *__restrict__ perm,
    const float2 *__restrict__ vis, const float *__restrict__ weight,
    const float2 *__restrict__ taps, float2 *grid, int32_t *status)
{
    constexpr int TERMS = Prec<PREC>::TERMS, STAGES = Prec<PREC>::STAGES;
    constexpr int NT = (S + 7) / 8;  // taps per producer thread
    extern __shared__ __align__(1024) unsigned char smem[];
    // operand buffers: A[stage][term], then B[stage][term]
    unsigned char *const Abuf = smem;
    unsigned char *const Bbuf = smem + STAGES * TERMS * kABytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(Bbuf + STAGES * TERMS * kBBytes);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;
    __shared__ uint32_t s_tmem;
    __shared__ int s_item;
    __shared__ volatile int s_abort;
    __shared__ float s_red[kProducerWarps];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == kProducerWarps;
    constexpr uint32_t idesc = instr_desc(PREC == 0 ? 1u : 0u);

    for (int e = tid; e < STAGES * TERMS * (kABytes + kBBytes) / 16; e += kTcBlock)
        reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int b = 0; b < STAGES; ++b) {
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

    // producer unit: visibility ii of each stage, taps k = q + 8 j
    const int ii = tid >> 3, q = tid & 7;
    // footprint origin (ly | lx << 8) this thread wrote into each buffer, or -1
    int oldpos[STAGES];
#pragma unroll
    for (int b = 0; b < STAGES; ++b)
        oldpos[b] = -1;

    int t_global = 0;  // stages of this CTA so far (buffer t % STAGES)
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
        int a_exp = 0;  // accumulator holds G * 2^-a_exp

        if (!mma_warp) {
            float scale = 1.0f;
            if constexpr (Prec<PREC>::SCALED) {
                // largest |W V| component of the item -> power-of-two scale
                float m = 0.f;
                for (int e = tid; e < it.count; e += kProducers) {
                    const int i = perm[it.start + e];
                    const float2 x = __ldg(vis + i);
                    const float wt = weight ? __ldg(weight + i) : 1.0f;
                    m = fmaxf(m, fmaxf(fabsf(wt * x.x), fabsf(wt * x.y)));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (lane == 0)
                    s_red[warp] = m;
                asm volatile("bar.sync 1, %0;" ::"n"(kProducers) : "memory");
                m = s_red[0];
#pragma unroll
                for (int w = 1; w < kProducerWarps; ++w)
                    m = fmaxf(m, s_red[w]);
                if (m > 0.f && m <= 3.0e38f) {
                    frexpf(m, &a_exp);  // m = f 2^a_exp, f in [0.5, 1)
                    // 2^-a_exp and 2^a_exp both normal floats
                    a_exp = max(-126, min(126, a_exp));
                    scale = ldexpf(1.0f, -a_exp);
                }
            }
            // The record is read one stage ahead; the visibility, weight and
            // taps at the start of the stage, so that their latency overlaps
            // the wait for the buffer.
            auto rec_at = [&](int st_, uint64_t &r_, int &i_) {
                const int e = st_ * kStageVis + ii;
                i_ = -1;
                if (st_ < nst && e < it.count) {
                    r_ = rec[it.start + e];
                    i_ = perm[it.start + e];
                }
            };
            uint64_t rn = 0;
            int in = -1;
            rec_at(0, rn, in);
            for (int st = 0; st < nst; ++st) {
                const int t = t_global + st;
                const int b = t % STAGES;
                const uint64_t r = rn;
                const int i = in;
                rec_at(st + 1, rn, in);
                StageData<NT> cur;
                cur.pos = -1;
                if (i >= 0) {
                    cur.x = __ldg(vis + i);
                    cur.wt = weight ? __ldg(weight + i) : 1.0f;
                    const int row = rec_plane(r) * p.OS;
                    const float2 *pv = taps + p.voff + (row + rec_ov(r)) * S + q;
                    const float2 *pu = taps + (row + rec_ou(r)) * S + q;
#pragma unroll
                    for (int j = 0; j < NT; ++j) {
                        cur.tv[j] = make_float2(0.f, 0.f);
                        cur.tu[j] = make_float2(0.f, 0.f);
                        if (q + 8 * j < S) {
                            cur.tv[j] = __ldg(pv + 8 * j);
                            cur.tu[j] = __ldg(pu + 8 * j);
                        }
                    }
                    cur.pos = rec_ly(r) | (rec_lx(r) << 8) | (rec_conj(r) ? 1 << 16 : 0);
                }
                int old = -1;
#pragma unroll
                for (int c = 0; c < STAGES; ++c)
                    if (c == b)
                        old = oldpos[c];
                if (t >= STAGES) {
                    // buffer b held stage t - STAGES: wait (lane 0) for its
                    // MMAs, then clear the entries this thread wrote there
                    if (lane == 0 && !s_abort &&
                        !mbar_wait(empty + b, ((t - STAGES) / STAGES) & 1))
                        s_abort = 1;
                    __syncwarp();
                    tc_fence_after();
                    if (old >= 0) {
                        uint32_t oa[NT], ob[NT];
                        row_offsets<NT>((old & 255) + q, ii, oa);
                        row_offsets<NT>(((old >> 8) & 255) + q, ii, ob);
#pragma unroll
                        for (int h = 0; h < TERMS; ++h) {
                            unsigned char *A = Abuf + (b * TERMS + h) * kABytes;
                            unsigned char *B = Bbuf + (b * TERMS + h) * kBBytes;
#pragma unroll
                            for (int j = 0; j < NT; ++j) {
                                if (q + 8 * j >= S)
                                    continue;
                                *reinterpret_cast<uint32_t *>(A + oa[j]) = 0u;
                                *reinterpret_cast<uint32_t *>(A + oa[j] + 8 * kSBO) = 0u;
                                *reinterpret_cast<uint32_t *>(B + ob[j]) = 0u;
                            }
                        }
                    }
                }
                const int pos = cur.pos;
                if (pos >= 0) {
                    const bool cj = pos >> 16;
                    const float wr = (cur.wt * cur.x.x) * scale;  // exact power-of-two scaling
                    const float wi = (cur.wt * cur.x.y) * scale;
                    uint32_t oa[NT], ob[NT];
                    row_offsets<NT>((pos & 255) + q, ii, oa);
                    row_offsets<NT>(((pos >> 8) & 255) + q, ii, ob);
                    unsigned char *A0 = Abuf + (b * TERMS) * kABytes;
                    unsigned char *B0 = Bbuf + (b * TERMS) * kBBytes;
#pragma unroll
                    for (int j = 0; j < NT; ++j) {
                        if (q + 8 * j >= S)
                            continue;
                        const float vr = cur.tv[j].x, vi = cj ? -cur.tv[j].y : cur.tv[j].y;
                        const float ur = cur.tu[j].x, ui = cj ? -cur.tu[j].y : cur.tu[j].y;
                        const float pr = wr * ur - wi * ui;
                        const float pi = wr * ui + wi * ur;
                        uint32_t vh, vl, ph, pl;
                        split2<PREC>(vr, vi, vh, vl);
                        split2<PREC>(pr, pi, ph, pl);
                        // rows y: (Bv_r, -Bv_i); rows 64 + y: (Bv_i, Bv_r)
                        *reinterpret_cast<uint32_t *>(A0 + oa[j]) = pair_conj(vh);
                        *reinterpret_cast<uint32_t *>(A0 + oa[j] + 8 * kSBO) = pair_swap(vh);
                        *reinterpret_cast<uint32_t *>(B0 + ob[j]) = ph;
                        if constexpr (TERMS == 2) {
                            *reinterpret_cast<uint32_t *>(A0 + kABytes + oa[j]) = pair_conj(vl);
                            *reinterpret_cast<uint32_t *>(A0 + kABytes + oa[j] + 8 * kSBO) =
                                pair_swap(vl);
                            *reinterpret_cast<uint32_t *>(B0 + kBBytes + ob[j]) = pl;
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < STAGES; ++c)
                    if (c == b)
                        oldpos[c] = pos;
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
                const int b = t % STAGES;
                if (!s_abort && !mbar_wait(full + b, (t / STAGES) & 1))
                    s_abort = 1;
                if (s_abort)
                    continue;
                tc_fence_after();
                const int v0 = it.start + st * kStageVis;
                const int nv = min(kStageVis, it.start + it.count - v0);
                const uint32_t ah = smem_u32(Abuf + (b * TERMS) * kABytes);
                const uint32_t bh = smem_u32(Bbuf + (b * TERMS) * kBBytes);
                const int nk = (nv + 7) / 8;  // K = 16 steps holding visibilities
                for (int kq = 0; kq < nk; ++kq) {
                    const uint32_t acc = (st > 0 || kq > 0) ? 1u : 0u;
                    mma_f16(tmem, smem_desc(ah + 256 * kq), smem_desc(bh + 256 * kq), idesc,
                            acc);
                    if constexpr (TERMS == 2) {
                        mma_f16(tmem, smem_desc(ah + 256 * kq),
                                smem_desc(bh + kBBytes + 256 * kq), idesc, 1u);
                        mma_f16(tmem, smem_desc(ah + kABytes + 256 * kq),
                                smem_desc(bh + 256 * kq), idesc, 1u);
                    }
                }
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
            const int qq = warp & 3, h = warp >> 2;  // lane quarter, 16-column group
            const int m = 32 * qq + lane;
            const float back = ldexpf(1.0f, a_exp);
            uint32_t rr[16];
            SEPW_TMEM_LD16(tmem + ((uint32_t)(32 * qq) << 16) + 16 * h, rr);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int x = 16 * h + c;
                stg[m * kWin + (x ^ (m & 31))] = __uint_as_float(rr[c]) * back;
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
        for (int e = tid; e < STAGES * TERMS * kBBytes / 16; e += kTcBlock)
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

template <int S, int PREC>
cudaError_t launch_tc_S(const DevParams &p, const Plan &plan, const float2 *vis,
                        const float *weight, const float2 *taps, float2 *grid, int num_sms,
                        int32_t *status, cudaStream_t s)
{
    constexpr size_t shm = tc_smem_bytes_for<PREC>();
    cudaError_t e = cudaFuncSetAttribute(grid_tc_kernel<S, PREC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess)
        return e;
    e = cudaMemsetAsync(plan.d_item_counter, 0, sizeof(int32_t), s);
    if (e != cudaSuccess)
        return e;
    grid_tc_kernel<S, PREC><<<num_sms, kTcBlock, shm, s>>>(
        p, plan.d_items, plan.d_nitems, plan.d_item_counter, plan.d_rec, plan.d_perm, vis,
        weight, taps, grid, status);
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_tc_prec(int prec, const DevParams &p, const Plan &plan, const float2 *vis,
                           const float *weight, const float2 *taps, float2 *grid,
                           int num_sms, int32_t *status, cudaStream_t s)
{
    switch (prec) {
    case 0: return launch_tc_S<S, 0>(p, plan, vis, weight, taps, grid, num_sms, status, s);
    case 1: return launch_tc_S<S, 1>(p, plan, vis, weight, taps, grid, num_sms, status, s);
    case 2: return launch_tc_S<S, 2>(p, plan, vis, weight, taps, grid, num_sms, status, s);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Tensor-core contraction form of the degridder (the adjoint, Sec. 2).
//
// Per tile window X (64 x 64 cells) and 128 visibilities of a stage,
//     Q[i][x] = sum_y conj(Av[i][y]) X[y][x]
// with Av[i][y] the v-taps of visibility i at its row offset (conjugated for
// w < 0), then V_i = W_i sum_j tu'[j] Q[i][lx_i + j] with tu' = conj(tu)
// (tu for w < 0).  In real arithmetic with K = (y, re/im) and N = (x, re/im):
//     A[i][(y,0)] = Av_r, A[i][(y,1)] = Av_i;
//     B[(y,0)][(x,0)] = X_r, B[(y,1)][(x,0)] = X_i,
//     B[(y,0)][(x,1)] = X_i, B[(y,1)][(x,1)] = -X_r,
// one tcgen05.mma shape M = 128 (visibilities), N = 128, K = 16 per step,
// eight steps per stage; a stage inside one sub-block of the tile contracts
// only the 32 window columns its footprints reach (N = 64).  B (the window) is built once per work item in one
// of two buffers; A (2 S values per visibility, cleared after use) in one of
// two stage buffers; a window buffer is rebuilt only after the epilogue has
// finished the item before last.  Roles: 8 producer warps (two threads per
// visibility), one MMA warp (two TMEM accumulators of 128 columns), 4 epilogue warps,
// one thread per visibility: each reads its accumulator row, stages it in
// shared memory and takes the u-direction dot product at its own column
// offset.  FP16 operands take a power-of-two scale per item so that the
// window's largest component is below 1.  Work items are assigned to CTAs
// statically (item = CTA, CTA + grid, ...), so every role walks the same
// sequence without a shared counter.  All mbarrier waits are bounded.
// ---------------------------------------------------------------------------
constexpr int kDgProducers = 256;
constexpr int kDgProdWarps = kDgProducers / 32;
constexpr int kDgVis = 128;
constexpr int kDgEpiWarps = 4;
constexpr int kDgMmaWarp = kDgProdWarps;
constexpr int kDgBlock = kDgProducers + 32 + 32 * kDgEpiWarps;
constexpr int kDgK = 128, kDgN = 128;
constexpr int kDgABytes = kDgVis * kDgK * 2;  // 32 KiB
constexpr int kDgBBytes = kDgN * kDgK * 2;    // 32 KiB
constexpr int kDgStgBytes = kDgVis * kDgN * 4;  // 64 KiB
constexpr uint32_t kDgTmemCols = 256;

constexpr size_t degrid_tc_smem_bytes()
{
    return 2 * (size_t)kDgABytes + 2 * (size_t)kDgBBytes + kDgStgBytes + 12 * sizeof(uint64_t);
}

__host__ __device__ constexpr uint32_t instr_desc_n(uint32_t ab_fmt, int n)
{
    return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kM >> 4) << 24);
}

// byte offset of element pair k, k + 1 (k even) of row `row` in a K = 128
// K-major operand
__device__ __forceinline__ uint32_t dg_off(int row, int k)
{
    return (uint32_t)((row >> 3) * kSBO + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <int PREC>
__device__ __forceinline__ uint32_t pack_pair(float x, float y)
{
    uint32_t hi, lo;
    split2<PREC>(x, y, hi, lo);
    return hi;
}

// First window column x0 of a stage whose visibilities all lie in one column
// of sub-blocks of the tile (the plan keeps the bins of a column consecutive
// inside an item, so the first and last slot decide), when their footprints
// fit the 32 columns x0 .. x0 + 31: the stage then contracts only those
// (N = 64).  -1: the whole window (N = 128).  x0 is a multiple of 4 (the
// operand's 8-row core-matrix groups) and at most 32.
__device__ __forceinline__ int dg_stage_x0(const DevParams &p, const WorkItem &it, int st,
                                           const uint64_t *__restrict__ rec, int S)
{
    const int first = it.start + st * kDgVis;
    const int last = min(first + kDgVis, it.start + it.count) - 1;
    const uint64_t r0 = __ldg(reinterpret_cast<const unsigned long long *>(rec) + first);
    const uint64_t r1 = __ldg(reinterpret_cast<const unsigned long long *>(rec) + last);
    const int sx = sub_bin(rec_lx(r0), rec_ly(r0), rec_conj(r0), p) >> 3;
    if (sx != sub_bin(rec_lx(r1), rec_ly(r1), rec_conj(r1), p) >> 3)
        return -1;
    const int lo = (sx * p.T + 3) >> 2;            // first column of the sub-block
    const int hi = (((sx + 1) * p.T + 3) >> 2) - 1;  // last column
    const int x0 = min(lo & ~3, 32);
    return hi + S <= x0 + 32 ? x0 : -1;
}

template <int S, int PREC>
__global__ void __launch_bounds__(kDgBlock, 1) degrid_tc_kernel(
    DevParams p, const WorkItem *__restrict__ items, const int32_t *__restrict__ nitems,
    const uint64_t *__restrict__ rec, const int32_t *__restrict__ perm,
    const float2 *__restrict__ grid, const float *__restrict__ weight,
    const float2 *__restrict__ taps, float2 *__restrict__ vis_out, int32_t *status)
{
    constexpr int NT = (S + 1) / 2 < 8 ? (S + 1) / 2 : 8;  // taps per producer thread
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *const Abuf = smem;                          // [2] stage operands
    unsigned char *const Bbuf = smem + 2 * kDgABytes;          // [2] window operands
    float *const stg = reinterpret_cast<float *>(Bbuf + 2 * kDgBBytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(Bbuf + 2 * kDgBBytes + kDgStgBytes);
    uint64_t *full = bars, *empty = bars + 2, *accf = bars + 4, *tfree = bars + 6,
             *efree = bars + 8, *bready = bars + 10;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ int s_aexp[2];
    __shared__ float s_red[kDgProdWarps];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr uint32_t idesc = instr_desc_n(PREC == 0 ? 1u : 0u, kDgN);
    constexpr uint32_t idesc64 = instr_desc_n(PREC == 0 ? 1u : 0u, kDgN / 2);
    const int n_items = *nitems;
    const int W = p.T + S - 1;

    for (int e = tid; e < (2 * kDgABytes + 2 * kDgBBytes) / 16; e += kDgBlock)
        reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(full + b, kDgProdWarps);
            mbar_init(empty + b, 1);
            mbar_init(accf + b, 1);
            mbar_init(tfree + b, kDgEpiWarps);
            mbar_init(efree + b, kDgEpiWarps);
            mbar_init(bready + b, kDgProdWarps);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kDgTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // lane 0 waits (bounded), the warp follows
    auto warp_wait = [&](uint64_t *bar, uint32_t parity) {
        if (lane == 0 && !s_abort && !mbar_wait(bar, parity))
            s_abort = 1;
        __syncwarp();
    };

    if (warp < kDgProdWarps) {
        // ---------------- producers: window operand per item, A per stage
        const int ii = tid >> 1, h = tid & 1;
        int oldly[2] = {-1, -1};
        int tg = 0;
        for (int n = 0;; ++n) {
            const int item = blockIdx.x + n * gridDim.x;
            if (item >= n_items || s_abort)
                break;
            const WorkItem it = items[item];
            const int nst = (it.count + kDgVis - 1) / kDgVis;
            const int ib = n & 1;
            // window buffer ib and its scale are free once the epilogue has
            // finished item n - 2 (all of whose MMAs it has waited for)
            if (n >= 2)
                warp_wait(efree + ib, ((n - 2) >> 1) & 1);
            tc_fence_after();
            // the window, scaled by 2^-a for FP16
            const TileOrigin o = tile_origin(p, it.tile);
            float2 xv[16];
            float m = 0.f;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int e = tid + q * kDgProducers;  // 4096 cells
                const int y = e >> 6, x = e & 63;
                float2 g = make_float2(0.f, 0.f);
                if (y < W && x < W && o.gy0 + y < p.N && o.gx0 + x < p.N)
                    g = __ldg(grid + o.base + (o.gy0 + y) * p.N + o.gx0 + x);
                xv[q] = g;
                m = fmaxf(m, fmaxf(fabsf(g.x), fabsf(g.y)));
            }
            int a_exp = 0;
            float scale = 1.f;
            if constexpr (PREC == 1) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
                if (lane == 0)
                    s_red[warp] = m;
                asm volatile("bar.sync 1, %0;" ::"n"(kDgProducers) : "memory");
                m = s_red[0];
#pragma unroll
                for (int w2 = 1; w2 < kDgProdWarps; ++w2)
                    m = fmaxf(m, s_red[w2]);
                if (m > 0.f && m <= 3.0e38f) {
                    frexpf(m, &a_exp);
                    a_exp = max(-126, min(126, a_exp));
                    scale = ldexpf(1.0f, -a_exp);
                }
            }
            unsigned char *B = Bbuf + ib * kDgBBytes;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int e = tid + q * kDgProducers;
                const int y = e >> 6, x = e & 63;
                const float xr = xv[q].x * scale, xi = xv[q].y * scale;
                // row (x, re): (X_r, X_i) at K = (y, 0), (y, 1); row (x, im): (X_i, -X_r)
                *reinterpret_cast<uint32_t *>(B + dg_off(2 * x, 2 * y)) = pack_pair<PREC>(xr, xi);
                *reinterpret_cast<uint32_t *>(B + dg_off(2 * x + 1, 2 * y)) =
                    pack_pair<PREC>(xi, -xr);
            }
            if (tid == 0)
                s_aexp[ib] = a_exp;
            fence_proxy_async();
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bready + ib))
                             : "memory");
            // records and taps run one stage ahead of the operand writes, so
            // their load latency overlaps the wait for the stage buffer
            auto stage_rec = [&](int st) -> uint64_t {
                return st < nst && st * kDgVis + ii < it.count
                           ? __ldg(reinterpret_cast<const unsigned long long *>(rec) +
                                   it.start + st * kDgVis + ii)
                           : ~0ull;
            };
            float2 tv[NT];
            auto stage_taps = [&](uint64_t r) {
                if (r != ~0ull) {
                    const float2 *pv = taps + p.voff + (rec_plane(r) * p.OS + rec_ov(r)) * S;
#pragma unroll
                    for (int j = 0; j < NT; ++j) {
                        const int k = NT * h + j;
                        tv[j] = k < S ? __ldg(pv + k) : make_float2(0.f, 0.f);
                    }
                }
            };
            uint64_t rcur = stage_rec(0);
            stage_taps(rcur);
            for (int st = 0; st < nst; ++st) {
                const int t = tg + st, b = t & 1;
                const uint64_t rnext = stage_rec(st + 1);
                const bool valid = rcur != ~0ull;
                const int ly = valid ? rec_ly(rcur) : -1;
                const bool cj = valid && rec_conj(rcur);
                if (t >= 2)
                    warp_wait(empty + b, ((t - 2) >> 1) & 1);
                tc_fence_after();
                unsigned char *A = Abuf + b * kDgABytes;
                if (oldly[b] >= 0) {
#pragma unroll
                    for (int j = 0; j < NT; ++j) {
                        const int k = NT * h + j;
                        if (k < S)
                            *reinterpret_cast<uint32_t *>(A + dg_off(ii, 2 * (oldly[b] + k))) = 0u;
                    }
                }
                if (valid) {
#pragma unroll
                    for (int j = 0; j < NT; ++j) {
                        const int k = NT * h + j;
                        if (k < S)
                            *reinterpret_cast<uint32_t *>(A + dg_off(ii, 2 * (ly + k))) =
                                pack_pair<PREC>(tv[j].x, cj ? -tv[j].y : tv[j].y);
                    }
                }
                oldly[b] = ly;
                fence_proxy_async();
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(full + b))
                                 : "memory");
                rcur = rnext;
                stage_taps(rcur);
            }
            tg += nst;
        }
    } else if (warp == kDgMmaWarp) {
        // ---------------- MMA issue (one thread)
        int tg = 0;
        int last_t = -1;  // last stage whose MMAs were committed
        for (int n = 0;; ++n) {
            const int item = blockIdx.x + n * gridDim.x;
            if (item >= n_items || s_abort)
                break;
            const WorkItem it = items[item];
            const int nst = (it.count + kDgVis - 1) / kDgVis;
            if (lane == 0) {
                for (int st = 0; st < nst && !s_abort; ++st) {
                    const int t = tg + st, b = t & 1;
                    const int x0 = dg_stage_x0(p, it, st, rec, S);
                    if (!mbar_wait(full + b, (t >> 1) & 1) ||
                        (t >= 2 && !mbar_wait(tfree + b, ((t - 2) >> 1) & 1))) {
                        s_abort = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(Abuf + b * kDgABytes);
                    // rows 2 x0 .. 2 x0 + 63 of the window operand: x0 / 4
                    // groups of 8 rows (kSBO bytes each) in
                    const uint32_t b0 = smem_u32(Bbuf + (n & 1) * kDgBBytes) +
                                        (x0 >= 0 ? (uint32_t)(x0 / 4) * kSBO : 0u);
                    const uint32_t id = x0 >= 0 ? idesc64 : idesc;
                    const uint32_t d = tmem + (uint32_t)(b * kDgN);
#pragma unroll
                    for (int kq = 0; kq < kDgK / 16; ++kq)
                        mma_f16(d, smem_desc(a0 + 256 * kq), smem_desc(b0 + 256 * kq), id,
                                kq > 0 ? 1u : 0u);
                    mma_commit(empty + b);
                    mma_commit(accf + b);
                    last_t = t;
                }
            }
            __syncwarp();
            tg += nst;
        }
        // after a timeout, wait (bounded) for this CTA's own MMAs before the
        // tensor memory is released
        if (s_abort && lane == 0 && last_t >= 0)
            mbar_wait(accf + (last_t & 1), (last_t >> 1) & 1);
    } else {
        // ---------------- epilogue: one thread per visibility of a stage
        const int qq = warp & 3;  // TMEM lane quarter this warp may read
        const int ii = 32 * qq + lane;
        float *const row = stg + ii * kDgN;
        int tg = 0;
        for (int n = 0;; ++n) {
            const int item = blockIdx.x + n * gridDim.x;
            if (item >= n_items || s_abort)
                break;
            const WorkItem it = items[item];
            const int nst = (it.count + kDgVis - 1) / kDgVis;
            const int ib = n & 1;
            // the records, output index and u-taps of a stage are loaded one
            // stage ahead, before the wait for its accumulator
            auto stage_rec = [&](int st, int &io) -> uint64_t {
                if (st < nst && st * kDgVis + ii < it.count) {
                    const int slot = it.start + st * kDgVis + ii;
                    io = __ldg(perm + slot);
                    return __ldg(reinterpret_cast<const unsigned long long *>(rec) + slot);
                }
                return ~0ull;
            };
            float2 tu[S];
            float wcur = 1.f;
            auto stage_taps = [&](uint64_t r, int io) {
                if (r != ~0ull) {
                    const float2 *pu = taps + (rec_plane(r) * p.OS + rec_ou(r)) * S;
#pragma unroll
                    for (int j = 0; j < S; ++j)
                        tu[j] = __ldg(pu + j);
                    wcur = weight ? __ldg(weight + io) : 1.0f;
                }
            };
            int iout = 0;
            uint64_t rcur = stage_rec(0, iout);
            stage_taps(rcur, iout);
            warp_wait(bready + ib, (n >> 1) & 1);
            const float back = ldexpf(1.0f, s_aexp[ib]);
            for (int st = 0; st < nst; ++st) {
                const int t = tg + st, b = t & 1;
                int inext = 0;
                const uint64_t rnext = stage_rec(st + 1, inext);
                const int x0 = dg_stage_x0(p, it, st, rec, S);
                const int nc = x0 >= 0 ? kDgN / 64 : kDgN / 32;  // accumulator chunks
                const int xb = x0 >= 0 ? x0 : 0;                  // window column of chunk 0
                warp_wait(accf + b, (t >> 1) & 1);
                if (s_abort)
                    break;
                tc_fence_after();
#pragma unroll
                for (int c = 0; c < kDgN / 32; ++c) {
                    if (c >= nc)
                        break;
                    uint32_t rr[32];
                    SEPW_TMEM_LD32(tmem + ((uint32_t)(32 * qq) << 16) + (uint32_t)(b * kDgN + 32 * c),
                                   rr);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int x = 0; x < 32; ++x)
                        row[(32 * c + x) ^ lane] = __uint_as_float(rr[x]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tfree + b))
                                 : "memory");
                if (rcur != ~0ull) {
                    const uint64_t r = rcur;
                    const int i = iout;
                    const float sg = rec_conj(r) ? 1.f : -1.f;  // tu' = conj(tu) unless w < 0
                    const int lx = rec_lx(r);
                    float vr = 0.f, vi = 0.f;
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        const float ur = tu[j].x, ui = sg * tu[j].y;
                        const int col = 2 * (lx - xb + j);
                        const float qr = row[col ^ lane], qi = row[(col + 1) ^ lane];
                        vr += ur * qr - ui * qi;
                        vi += ur * qi + ui * qr;
                    }
                    const float wt = wcur * back;
                    vis_out[i] = make_float2(wt * vr, wt * vi);
                }
                rcur = rnext;
                iout = inext;
                stage_taps(rcur, iout);
            }
            __syncwarp();
            if (lane == 0 && !s_abort)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(efree + ib))
                             : "memory");
            tg += nst;
        }
    }

    if (s_abort && tid == 0)
        atomicExch(status, SEPW_ETIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kDgTmemCols)
                     : "memory");
}

template <int S, int PREC>
cudaError_t launch_degrid_tc_S(const DevParams &p, const Plan &plan, const float2 *grid,
                               const float *weight, const float2 *taps, float2 *vis,
                               int num_sms, int32_t *status, cudaStream_t s)
{
    constexpr size_t shm = degrid_tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(degrid_tc_kernel<S, PREC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess)
        return e;
    degrid_tc_kernel<S, PREC><<<num_sms, kDgBlock, shm, s>>>(
        p, plan.d_items, plan.d_nitems, plan.d_rec, plan.d_perm, grid, weight, taps, vis,
        status);
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
                           int num_sms, int prec, int32_t *status, cudaStream_t s)
{
    if (p.T + p.S - 1 > kWin)
        return cudaErrorInvalidValue;
#define SEPW_TC_CASE(SS) \
    case SS: return launch_tc_prec<SS>(prec, p, plan, vis, weight, taps, grid, num_sms, status, s);
    switch (p.S) {
        SEPW_TC_CASE(2) SEPW_TC_CASE(4) SEPW_TC_CASE(6) SEPW_TC_CASE(8) SEPW_TC_CASE(10)
        SEPW_TC_CASE(12) SEPW_TC_CASE(14) SEPW_TC_CASE(16)
    default:
        return cudaErrorInvalidValue;
    }
#undef SEPW_TC_CASE
}

cudaError_t launch_degrid_tc(const DevParams &p, const Plan &plan, const float2 *grid,
                             const float *weight, const float2 *taps, float2 *vis,
                             int num_sms, int prec, int32_t *status, cudaStream_t s)
{
    if (p.T + p.S - 1 > kWin || (prec != 0 && prec != 1))
        return cudaErrorInvalidValue;
#define SEPW_DG_CASE(SS)                                                                     \
    case SS:                                                                                 \
        return prec ? launch_degrid_tc_S<SS, 1>(p, plan, grid, weight, taps, vis, num_sms,   \
                                                status, s)                                   \
                    : launch_degrid_tc_S<SS, 0>(p, plan, grid, weight, taps, vis, num_sms,   \
                                                status, s);
    switch (p.S) {
        SEPW_DG_CASE(2) SEPW_DG_CASE(4) SEPW_DG_CASE(6) SEPW_DG_CASE(8) SEPW_DG_CASE(10)
        SEPW_DG_CASE(12) SEPW_DG_CASE(14) SEPW_DG_CASE(16)
    default:
        return cudaErrorInvalidValue;
    }
#undef SEPW_DG_CASE
}

}  // namespace sepw
