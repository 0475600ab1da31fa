// Tensor-core (tcgen05) contraction form of the degridder (the adjoint of the
// contraction gridder of sepw_tc_grid.cu), for BF16 and FP16 operands with
// FP32 accumulation in tensor memory.  Every mbarrier wait is bounded; on
// expiry the kernel records SEPW_ETIMEOUT in the device status word, stops
// issuing work, waits (bounded) for its own MMAs and frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sepw_internal.cuh"
#include "sepw_tc_ptx.cuh"

namespace sepw {
namespace {

using namespace tcx;

constexpr int kM = 128;                         // MMA rows (visibilities)
// K-major canonical layout of a K = 128 operand: K-adjacent core matrices 128
// bytes apart, 8-row groups kSBO bytes apart
constexpr int kSBO = (128 / 8) * 128;

// Packs (x, y) as a BF16 (PREC 0) or FP16 (PREC 1) pair.
template <int PREC>
__device__ __forceinline__ uint32_t pack_pair(float x, float y)
{
    if constexpr (PREC == 0) {
        __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(x, y);
        return *reinterpret_cast<uint32_t *>(&h);
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
constexpr int kDgWin = 64;  // window edge, T + S - 1 <= 64
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

// Instruction descriptor: A and B K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t instr_desc_n(uint32_t ab_fmt, int n)
{
    return instr_desc(ab_fmt, false, false, kM, n);
}

// K-major no-swizzle descriptor of a K = 128 operand
__device__ __forceinline__ uint64_t kdesc(uint32_t addr) { return smem_desc(addr, 128, kSBO); }

// byte offset of element pair k, k + 1 (k even) of row `row` in a K = 128
// K-major operand
__device__ __forceinline__ uint32_t dg_off(int row, int k)
{
    return (uint32_t)((row >> 3) * kSBO + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
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
    if (p.T + S - 1 <= 32)
        return 0;  // the whole window fits the 32 columns
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
    const float2 *__restrict__ taps, float2 *__restrict__ vis_out, int32_t *status,
    TcControl ctl)
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
        if (lane == 0 && !s_abort && !mbar_wait(bar, parity, ctl.wait_ns))
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
                    if (!mbar_wait(full + b, (t >> 1) & 1, ctl.wait_ns) ||
                        (t >= 2 && !mbar_wait(tfree + b, ((t - 2) >> 1) & 1, ctl.wait_ns))) {
                        s_abort = 1;
                        break;
                    }
                    if (ctl.stall)
                        continue;  // test hook: issue and signal nothing
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
                        mma_f16(d, kdesc(a0 + 256 * kq), kdesc(b0 + 256 * kq), id,
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
            mbar_wait(accf + (last_t & 1), (last_t >> 1) & 1, ctl.wait_ns);
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
                               int num_sms, int32_t *status, TcControl ctl, cudaStream_t s)
{
    constexpr size_t shm = degrid_tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(degrid_tc_kernel<S, PREC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess)
        return e;
    degrid_tc_kernel<S, PREC><<<num_sms, kDgBlock, shm, s>>>(
        p, plan.d_items, plan.d_nitems, plan.d_rec, plan.d_perm, grid, weight, taps, vis,
        status, ctl);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_degrid_tc(const DevParams &p, const Plan &plan, const float2 *grid,
                             const float *weight, const float2 *taps, float2 *vis,
                             int num_sms, int prec, int32_t *status, TcControl ctl,
                             cudaStream_t s)
{
    if (p.T + p.S - 1 > kDgWin || (prec != 0 && prec != 1))
        return cudaErrorInvalidValue;
#define SEPW_DG_CASE(SS)                                                                     \
    case SS:                                                                                 \
        return prec ? launch_degrid_tc_S<SS, 1>(p, plan, grid, weight, taps, vis, num_sms,   \
                                                status, ctl, s)                              \
                    : launch_degrid_tc_S<SS, 0>(p, plan, grid, weight, taps, vis, num_sms,   \
                                                status, ctl, s);
    switch (p.S) {
        SEPW_DG_CASE(2) SEPW_DG_CASE(4) SEPW_DG_CASE(6) SEPW_DG_CASE(8) SEPW_DG_CASE(10)
        SEPW_DG_CASE(12) SEPW_DG_CASE(14) SEPW_DG_CASE(16)
    default:
        return cudaErrorInvalidValue;
    }
#undef SEPW_DG_CASE
}

}  // namespace sepw
