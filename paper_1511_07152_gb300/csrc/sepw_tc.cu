// Tensor-core (tcgen05) contraction form of the degridder (the adjoint of the
// contraction gridder of sepw_tc_grid.cu), for BF16 and FP16 operands with
// FP32 accumulation in tensor memory.
//
// Per work item (one tile; its window X of W = T + S - 1 <= 32 cells a side)
// and stage of 128 visibilities (Sec. 2, the adjoint of gridding):
//     Q[i][x] = sum_y conj(a_i[y]) X[y][x]           (tcgen05.mma)
//     V_i = W_i sum_j tu'_i[j] Q[i][lx_i + j]         (epilogue, FP32)
// with a_i the v-taps of visibility i at its row offset (conjugated for
// w < 0) and tu' = conj(tu) (tu for w < 0).  In real arithmetic with
// K = (y, re/im) and N = (x, re/im), 32 window cells a side:
//     A[i][(y,0)] = a_r    A[i][(y,1)] = a_i
//     B[(y,0)][(x,0)] = X_r    B[(y,1)][(x,0)] = X_i
//     B[(y,0)][(x,1)] = X_i    B[(y,1)][(x,1)] = -X_r
// one MMA of M = 128 (visibilities), N = 64, K = 16, four per stage.  FP16
// operands take a power-of-two scale per item so that the window's largest
// component is below 1 (the producers find it while they load the window).
//
// Operands are K-major (8 K elements, one row of a core matrix, in 16 bytes):
//   - A, per stage, from a table built per call: per (plane, oversample)
//     the S v-taps as (re, im) pairs in the 16-bit format (64 bytes), shifted
//     in registers by ly mod 4 words into five 16-byte chunks, chunk j holding
//     rows 4 j .. 4 j + 3 of the footprint relative to 4 (ly / 4).  A
//     visibility's row of A is eight 16-byte stores: chunk j at K chunk
//     j + ly / 4, zeros elsewhere, so no row needs clearing.  Slot i of a stage is row i; the 8 lanes of a
//     quarter warp write 8 different rows of one core matrix column: no bank
//     conflicts, whatever chunk each lane writes.
//   - B, the window, once per item, two 4-byte (re, im) pairs per cell.
//
// Roles (work items assigned to CTAs round robin, so every role walks the
// same items and stages without a shared counter):
//   - eight producer warps in two groups of four, group g owning stage buffer
//     g: it writes the CTA's stages t = g, g + 2, ... (one lane per
//     visibility).  Owning its buffer, a group has itself filled the
//     buffer's previous stage, so its wait for that stage's MMAs is never two
//     mbarrier phases behind.  All eight build each item's window (two
//     buffers, item n in buffer n mod 2) and wait until it is complete
//     before they declare a stage full;
//   - one MMA thread: per stage it waits for "full" and for the accumulator,
//     issues the four MMAs and commits them to the stage's "done" barrier,
//     which both the producers (buffer free) and the epilogue (accumulator
//     ready) wait on: one commit per stage;
//   - four epilogue warps (one per tensor-memory lane quarter), one thread
//     per visibility: it reads its accumulator row into registers, releases
//     the accumulator, shifts the row to its column offset with a barrel
//     shift in registers and takes the u-direction dot product with the
//     u-taps of a second 16-bit table.
// Every mbarrier wait is bounded; on expiry the kernel records SEPW_ETIMEOUT
// in the device status word, every role leaves its loop, the MMA thread waits
// (bounded) for its own MMAs and the tensor memory is freed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "sepw_internal.cuh"
#include "sepw_tc_ptx.cuh"

namespace sepw {
namespace {

using namespace tcx;

constexpr int kDgWin = 32;                               // window edge
constexpr int kDgVis = 128;                              // visibilities per stage (M)
constexpr int kDgK = 2 * kDgWin;                         // K = (y, re/im)
constexpr int kDgN = 2 * kDgWin;                         // N = (x, re/im)
constexpr int kDgGroups = 2;                             // producer groups = buffers
constexpr int kDgGroupWarps = kDgVis / 32;               // warps per group
constexpr int kDgProdWarps = kDgGroups * kDgGroupWarps;  // 8
constexpr int kDgProducers = 32 * kDgProdWarps;          // 256
constexpr int kDgMmaWarp = kDgProdWarps;
constexpr int kDgEpiWarps = 4;
constexpr int kDgBlock = kDgProducers + 32 + 32 * kDgEpiWarps;  // 416
constexpr uint32_t kDgLbo = 128;                 // K-adjacent core matrices
constexpr uint32_t kDgSbo = (kDgK / 8) * 128;    // 8-row groups
constexpr int kDgABytes = kDgVis * kDgK * 2;     // 16 KiB
constexpr int kDgBBytes = kDgN * kDgK * 2;       // 8 KiB
constexpr uint32_t kDgTmemCols = kDgGroups * kDgN;  // two accumulators
constexpr int kDgVChunks = 4;   // v-table chunks per row: 16 (re, im) pairs, unshifted
constexpr int kDgUChunks = 4;   // u-table chunks per row: 16 (re, im) pairs
constexpr size_t kDgSmem = 2 * (size_t)kDgABytes + 2 * (size_t)kDgBBytes + 16 * sizeof(uint64_t);
static_assert(kDgSmem <= 227 * 1024, "shared memory per CTA");

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Packs (x, y) as a BF16 (PREC 0) or FP16 (PREC 1) pair, x in the low half.
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

template <int PREC>
__device__ __forceinline__ float2 unpack_pair(uint32_t w)
{
    if constexpr (PREC == 0) {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    } else {
        return __half22float2(*reinterpret_cast<const __half2 *>(&w));
    }
}

__device__ __forceinline__ void st16(unsigned char *p, uint4 v)
{
    *reinterpret_cast<uint4 *>(p) = v;
}

__device__ __forceinline__ void ldg32(const void *p, uint4 &a, uint4 &b)
{
    asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z),
                   "=r"(b.w)
                 : "l"(p));
}

// byte offset of the element pair k, k + 1 (k even) of row `row` of a K = 64
// K-major operand
__device__ __forceinline__ uint32_t dg_off(int row, int k)
{
    return (uint32_t)((row >> 3) * kDgSbo + (k >> 3) * kDgLbo + (row & 7) * 16 + (k & 7) * 2);
}

// Workspace layout (from the start of the degridder's part): v-table, then
// u-table.
struct DgTables {
    uint4 *vtab;
    uint4 *utab;
};

DgTables dg_tables(const DevParams &p, void *base)
{
    const int64_t nrow = (int64_t)p.P * p.OS;
    unsigned char *b = reinterpret_cast<unsigned char *>(base);
    DgTables t;
    t.vtab = reinterpret_cast<uint4 *>(b);
    t.utab = t.vtab + nrow * kDgVChunks;
    return t;
}

// Per-call tables from the caller's complex64 taps (v taps at p.voff).
template <int PREC>
__global__ void dg_tables_kernel(DevParams p, const float2 *__restrict__ taps, uint4 *vtab,
                                 uint4 *utab)
{
    const int64_t nrow = (int64_t)p.P * p.OS;
    const int64_t nv = nrow * kDgVChunks, nu = nrow * kDgUChunks;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nv + nu; e += stride) {
        uint32_t w[4];
        if (e < nv) {
            const int j = (int)(e % kDgVChunks);
            const int64_t row = e / kDgVChunks;
            const float2 *tv = taps + p.voff + row * p.S;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = 4 * j + q;
                const float2 t = k < p.S ? tv[k] : make_float2(0.f, 0.f);
                w[q] = pack_pair<PREC>(t.x, t.y);
            }
            vtab[e] = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
            const int64_t q0 = e - nv;
            const int j = (int)(q0 % kDgUChunks);
            const int64_t row = q0 / kDgUChunks;
            const float2 *tu = taps + row * p.S;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = 4 * j + q;
                const float2 t = k < p.S ? tu[k] : make_float2(0.f, 0.f);
                w[q] = pack_pair<PREC>(t.x, t.y);
            }
            utab[q0] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// bits of the footprint column offset lx (0 .. T - 1, T <= 33 - S)
template <int S>
constexpr int kShiftBits = ((33 - S) & ~1) > 16 ? 5 : ((33 - S) & ~1) > 8 ? 4 : 3;

// q[k] <- q[k + 2 lx] for k < 2 S: levels BIT .. 0 of a barrel shift, level
// b moving by 2^(b+1) entries when bit b of lx is set and keeping only the
// entries the lower levels and the taps read.
template <int S, int BIT>
__device__ __forceinline__ void barrel_shift(float (&q)[kDgN], int lx)
{
    if constexpr (BIT >= 0) {
        constexpr int kSh = 2 << BIT;
        constexpr int kLen = 2 * S + 2 * ((1 << BIT) - 1);
        const bool on = (lx >> BIT) & 1;
#pragma unroll
        for (int k = 0; k < kLen; ++k)
            q[k] = on ? (k + kSh < kDgN ? q[k + kSh] : 0.f) : q[k];
        barrel_shift<S, BIT - 1>(q, lx);
    }
}

// Power-of-two exponent a with the window's largest component (the maximum
// of the producer warps' maxima) below 2^a: the FP16 form's scale 2^-a.
__device__ __forceinline__ int window_exp(const float *wm)
{
    float m = 0.f;
#pragma unroll
    for (int w = 0; w < kDgProdWarps; ++w)
        m = fmaxf(m, wm[w]);
    int a = 0;
    if (m > 0.f && m <= 3.0e38f) {
        frexpf(m, &a);  // m = f 2^a, f in [0.5, 1)
        a = max(-126, min(126, a));
    }
    return a;
}

template <int S, int PREC>
__global__ void __launch_bounds__(kDgBlock, 1) degrid_tc_kernel(
    DevParams p, const WorkItem *__restrict__ items, const int32_t *__restrict__ nitems,
    const uint64_t *__restrict__ rec, const int32_t *__restrict__ perm,
    const float2 *__restrict__ grid, const float *__restrict__ weight,
    const uint4 *__restrict__ vtab, const uint4 *__restrict__ utab,
    float2 *__restrict__ vis_out, int32_t *status, TcControl ctl)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *const Abuf = smem;                      // [2] stage operands
    unsigned char *const Bbuf = smem + 2 * kDgABytes;      // [2] window operands
    uint64_t *const bars = reinterpret_cast<uint64_t *>(Bbuf + 2 * kDgBBytes);
    uint64_t *const full = bars, *const done = bars + 2, *const tfree = bars + 4,
                    *const efree = bars + 6, *const bready = bars + 8, *const drain = bars + 10,
                    *const wmax = bars + 11;  // [2]
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ float s_wmax[2][kDgProdWarps];  // FP16: per-warp window maxima

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_items = *nitems;
    const int W = p.T + S - 1;

    for (int e = tid; e < (2 * kDgABytes + 2 * kDgBBytes) / 16; e += kDgBlock)
        reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(full + b, kDgGroupWarps);
            mbar_init(done + b, 1);
            mbar_init(tfree + b, kDgEpiWarps);
            mbar_init(efree + b, kDgEpiWarps);
            mbar_init(bready + b, kDgProdWarps);
            mbar_init(wmax + b, kDgProdWarps);
        }
        mbar_init(drain, 1);
        s_abort = 0;
        mbar_init_fence();
    }
    if (warp == 0)
        tmem_alloc(&s_tmem, kDgTmemCols);
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
        // ------------------------------------------------------------ producers
        const int grp = warp / kDgGroupWarps;  // the stage buffer this group owns
        const int ii = tid & (kDgVis - 1);     // slot of a stage (row of A)
        unsigned char *const A = Abuf + grp * kDgABytes;
        const uint32_t arow = (uint32_t)((ii >> 3) * kDgSbo + (ii & 7) * 16);
        int tg = 0;
        for (int n = 0;; ++n) {
            const int item = blockIdx.x + n * gridDim.x;
            if (item >= n_items || s_abort)
                break;
            const WorkItem it = items[item];
            const int nst = (it.count + kDgVis - 1) / kDgVis;
            const int ib = n & 1;
            // window buffer ib is free once the epilogue has finished item
            // n - 2, all of whose MMAs it has waited for
            if (n >= 2)
                warp_wait(efree + ib, ((n - 2) >> 1) & 1);
            tc_fence_after();
            const TileOrigin o = tile_origin(p, it.tile);
            constexpr int kCells = kDgWin * kDgWin / kDgProducers;
            float2 gv[kCells];
#pragma unroll
            for (int q = 0; q < kCells; ++q) {
                const int e = tid + q * kDgProducers;
                const int y = e >> 5, x = e & 31;
                gv[q] = make_float2(0.f, 0.f);
                if (y < W && x < W && o.gy0 + y < p.N && o.gx0 + x < p.N)
                    gv[q] = __ldg(grid + o.base + (o.gy0 + y) * p.N + o.gx0 + x);
            }
            float scale = 1.f;
            if constexpr (PREC == 1) {
                // the window's largest component, over the eight producer
                // warps: scale 2^-a with that maximum below 2^a
                float m = 0.f;
#pragma unroll
                for (int q = 0; q < kCells; ++q)
                    m = fmaxf(m, fmaxf(fabsf(gv[q].x), fabsf(gv[q].y)));
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
                if (lane == 0) {
                    s_wmax[ib][warp] = m;
                    mbar_arrive(wmax + ib);
                }
                warp_wait(wmax + ib, (n >> 1) & 1);
                scale = ldexpf(1.0f, -window_exp(s_wmax[ib]));
            }
            unsigned char *const B = Bbuf + ib * kDgBBytes;
#pragma unroll
            for (int q = 0; q < kCells; ++q) {
                const int e = tid + q * kDgProducers;
                const int y = e >> 5, x = e & 31;
                const float xr = gv[q].x * scale, xi = gv[q].y * scale;
                // row (x, re): (X_r, X_i) at K = (y, 0), (y, 1); row (x, im): (X_i, -X_r)
                *reinterpret_cast<uint32_t *>(B + dg_off(2 * x, 2 * y)) = pack_pair<PREC>(xr, xi);
                *reinterpret_cast<uint32_t *>(B + dg_off(2 * x + 1, 2 * y)) =
                    pack_pair<PREC>(xi, -xr);
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(bready + ib);
            // the whole window is written (and fenced) before any stage of
            // the item is declared full
            warp_wait(bready + ib, (n >> 1) & 1);
            // the slot's record of the group's next stage is loaded one stage
            // ahead (records stream from HBM; the table rows are L2 hits)
            auto rec_of = [&](int st) -> uint64_t {
                const int e = st * kDgVis + ii;
                return st < nst && e < it.count
                           ? __ldg(reinterpret_cast<const unsigned long long *>(rec) + it.start + e)
                           : ~0ull;
            };
            int st0 = grp ^ (tg & 1);
            uint64_t rcur = rec_of(st0);
            for (int st = st0; st < nst && !s_abort; st += 2) {
                const int t = tg + st;  // t mod 2 == grp
                const uint64_t rnext = rec_of(st + 2);
                const bool valid = rcur != ~0ull;  // no record has its top bits set
                uint4 c4[4];  // the 16 unshifted (re, im) v-tap words
                int ly = 0;
                uint32_t cjm = 0;
                if (valid) {
                    const uint64_t r = rcur;
                    ly = rec_ly(r);
                    cjm = rec_conj(r) ? 0x80000000u : 0u;  // conj(a): the im halves
                    const uint4 *pv =
                        vtab + ((int64_t)rec_plane(r) * p.OS + rec_ov(r)) * kDgVChunks;
                    ldg32(pv, c4[0], c4[1]);
                    ldg32(pv + 2, c4[2], c4[3]);
                }
                // buffer grp held stage t - 2: wait for its MMAs
                if (t >= 2)
                    warp_wait(done + grp, ((t - 2) >> 1) & 1);
                tc_fence_after();
                const int oy4 = valid ? (ly >> 2) : 8;
                // shift the words by ly mod 4: word q of chunk j holds the tap
                // of window row 4 (j + ly / 4) + q
                uint32_t tw[20];
#pragma unroll
                for (int k = 0; k < 20; ++k)
                    tw[k] = k < 16 ? (&c4[k >> 2].x)[k & 3] : 0u;
#pragma unroll
                for (int k = 19; k >= 0; --k)
                    tw[k] = (ly & 2) ? (k >= 2 ? tw[k - 2] : 0u) : tw[k];
#pragma unroll
                for (int k = 19; k >= 0; --k)
                    tw[k] = (ly & 1) ? (k >= 1 ? tw[k - 1] : 0u) : tw[k];
                uint4 c[5];
#pragma unroll
                for (int j = 0; j < 5; ++j)
                    c[j] = make_uint4(tw[4 * j], tw[4 * j + 1], tw[4 * j + 2], tw[4 * j + 3]);
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    const int ca = j + oy4;  // K chunk of table chunk j
                    if (ca < 8)
                        st16(A + arow + ca * kDgLbo,
                             make_uint4(c[j].x ^ cjm, c[j].y ^ cjm, c[j].z ^ cjm, c[j].w ^ cjm));
                }
#pragma unroll
                for (int ca = 0; ca < 8; ++ca)
                    if (ca < oy4 || ca > oy4 + 4)
                        st16(A + arow + ca * kDgLbo, make_uint4(0, 0, 0, 0));
                fence_proxy_async();
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(full + grp);
                rcur = rnext;
            }
            tg += nst;
        }
    } else if (warp == kDgMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc(PREC == 0 ? 1u : 0u, false, false, kDgVis, kDgN);
            const uint64_t da0 = smem_desc(smem_u32(Abuf), kDgLbo, kDgSbo);
            const uint64_t db0 = smem_desc(smem_u32(Bbuf), kDgLbo, kDgSbo);
            constexpr uint64_t kStep = (2 * kDgLbo) >> 4;  // K = 16: two core matrices
            int tg = 0;
            bool ok = true, issued = false;
            for (int n = 0; ok; ++n) {
                const int item = blockIdx.x + n * gridDim.x;
                if (item >= n_items)
                    break;
                const int nst = (items[item].count + kDgVis - 1) / kDgVis;
                const uint64_t db = db0 + (uint64_t)((n & 1) * kDgBBytes >> 4);
                for (int st = 0; st < nst; ++st) {
                    const int t = tg + st, b = t & 1;
                    if (!mbar_wait(full + b, (t >> 1) & 1, ctl.wait_ns) ||
                        (t >= 2 && !mbar_wait(tfree + b, ((t - 2) >> 1) & 1, ctl.wait_ns))) {
                        ok = false;
                        break;
                    }
                    if (ctl.stall)
                        continue;  // test hook: issue and signal nothing
                    tc_fence_after();
                    const uint64_t da = da0 + (uint64_t)((b * kDgABytes) >> 4);
                    const uint32_t d = tmem + (uint32_t)(b * kDgN);
#pragma unroll
                    for (int kq = 0; kq < kDgK / 16; ++kq)
                        mma_f16(d, da + kStep * kq, db + kStep * kq, idesc, kq > 0 ? 1u : 0u);
                    mma_commit(done + b);
                    issued = true;
                }
                tg += nst;
            }
            if (!ok) {
                s_abort = 1;
                // bounded wait for every MMA this thread issued before the
                // tensor memory is released
                if (issued) {
                    mma_commit(drain);
                    mbar_wait(drain, 0, ctl.wait_ns);
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int qq = warp & 3;  // tensor-memory lane quarter of this warp
        const int ii = 32 * qq + lane;
        int tg = 0;
        for (int n = 0;; ++n) {
            const int item = blockIdx.x + n * gridDim.x;
            if (item >= n_items || s_abort)
                break;
            const WorkItem it = items[item];
            const int nst = (it.count + kDgVis - 1) / kDgVis;
            const int ib = n & 1;
            float back = 1.0f;
            if constexpr (PREC == 1) {
                // every producer warp writes its maximum before it arrives on
                // wmax; s_wmax[ib] is rewritten only for item n + 2, after
                // this warp has finished item n
                warp_wait(wmax + ib, (n >> 1) & 1);
                back = ldexpf(1.0f, window_exp(s_wmax[ib]));
            }
            // the slot's record and output index one stage ahead; its weight
            // and u-taps (which depend on them) before the accumulator wait
            auto rec_of = [&](int st, int &io) -> uint64_t {
                const int e = st * kDgVis + ii;
                if (st < nst && e < it.count) {
                    io = __ldg(perm + it.start + e);
                    return __ldg(reinterpret_cast<const unsigned long long *>(rec) + it.start + e);
                }
                return ~0ull;
            };
            int inext = 0;
            uint64_t rnext = rec_of(0, inext);
            for (int st = 0; st < nst; ++st) {
                const int t = tg + st, b = t & 1;
                const uint64_t r = rnext;
                const int io = inext;
                rnext = rec_of(st + 1, inext);
                const bool valid = r != ~0ull;
                int iout = 0, lx = 0;
                float wt = 0.f, sg = 1.f;
                uint4 u0, u1, u2, u3;
                if (valid) {
                    iout = io;
                    wt = (weight ? __ldg(weight + iout) : 1.0f) * back;
                    lx = rec_lx(r);
                    sg = rec_conj(r) ? 1.f : -1.f;  // tu' = conj(tu) unless w < 0
                    const uint4 *pu = utab + ((int64_t)rec_plane(r) * p.OS + rec_ou(r)) * kDgUChunks;
                    ldg32(pu, u0, u1);
                    ldg32(pu + 2, u2, u3);
                }
                warp_wait(done + b, (t >> 1) & 1);
                if (s_abort)
                    break;
                tc_fence_after();
                // this row's 64 accumulator columns (x, re/im)
                float q[kDgN];
#pragma unroll
                for (int h = 0; h < kDgN / 32; ++h) {
                    uint32_t rr[32];
                    SEPW_TMEM_LD32(tmem + ((uint32_t)(32 * qq) << 16) + (uint32_t)(b * kDgN + 32 * h),
                                   rr);
                    tmem_wait_ld();
#pragma unroll
                    for (int xx = 0; xx < 32; ++xx)
                        q[32 * h + xx] = __uint_as_float(rr[xx]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(tfree + b);
                if (valid) {
                    // q[k] <- q[k + 2 lx]: a barrel shift in registers, one
                    // level per bit of lx, each keeping only the entries the
                    // later levels and the 2 S taps still read
                    barrel_shift<S, kShiftBits<S> - 1>(q, lx);
                    const uint32_t uw[16] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w,
                                             u2.x, u2.y, u2.z, u2.w, u3.x, u3.y, u3.z, u3.w};
                    float vr = 0.f, vi = 0.f;
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        const float2 u = unpack_pair<PREC>(uw[j]);
                        const float ur = u.x, ui = sg * u.y;
                        const float qr = q[2 * j], qi = q[2 * j + 1];
                        vr += ur * qr - ui * qi;
                        vi += ur * qi + ui * qr;
                    }
                    vis_out[iout] = make_float2(wt * vr, wt * vi);
                }
            }
            __syncwarp();
            if (lane == 0 && !s_abort)
                mbar_arrive(efree + ib);
            tg += nst;
        }
    }

    __syncthreads();
    if (s_abort && tid == 0)
        atomicExch(status, SEPW_ETIMEOUT);
    tc_fence_after();
    if (warp == 0)
        tmem_dealloc(tmem, kDgTmemCols);
}

template <int S, int PREC>
cudaError_t launch_degrid_tc_S(const DevParams &p, const Plan &plan, const float2 *grid,
                               const float *weight, const float2 *taps, void *tables,
                               float2 *vis, int num_sms, int32_t *status, TcControl ctl,
                               cudaStream_t s)
{
    const DgTables t = dg_tables(p, tables);
    const int64_t nrow = (int64_t)p.P * p.OS;
    const int64_t n = nrow * (kDgVChunks + kDgUChunks);
    dg_tables_kernel<PREC><<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(
        p, taps, t.vtab, t.utab);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(degrid_tc_kernel<S, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kDgSmem);
    if (e != cudaSuccess)
        return e;
    degrid_tc_kernel<S, PREC><<<num_sms, kDgBlock, kDgSmem, s>>>(
        p, plan.d_items, plan.d_nitems, plan.d_rec, plan.d_perm, grid, weight, t.vtab, t.utab,
        vis, status, ctl);
    return cudaGetLastError();
}

}  // namespace

size_t tc_degrid_tables_bytes(const DevParams &p, int64_t items_capacity)
{
    (void)items_capacity;
    const size_t nrow = (size_t)p.P * p.OS;
    return align256(nrow * (kDgVChunks + kDgUChunks) * 16);
}

cudaError_t launch_degrid_tc(const DevParams &p, const Plan &plan, const float2 *grid,
                             const float *weight, const float2 *taps, void *tables, float2 *vis,
                             int num_sms, int prec, int32_t *status, TcControl ctl,
                             cudaStream_t s)
{
    if (p.T + p.S - 1 > kDgWin || p.S > 16 || (prec != 0 && prec != 1))
        return cudaErrorInvalidValue;
#define SEPW_DG_CASE(SS)                                                                     \
    case SS:                                                                                 \
        return prec ? launch_degrid_tc_S<SS, 1>(p, plan, grid, weight, taps, tables, vis,    \
                                                num_sms, status, ctl, s)                     \
                    : launch_degrid_tc_S<SS, 0>(p, plan, grid, weight, taps, tables, vis,    \
                                                num_sms, status, ctl, s);
    switch (p.S) {
        SEPW_DG_CASE(2) SEPW_DG_CASE(4) SEPW_DG_CASE(6) SEPW_DG_CASE(8) SEPW_DG_CASE(10)
        SEPW_DG_CASE(12) SEPW_DG_CASE(14) SEPW_DG_CASE(16)
    default:
        return cudaErrorInvalidValue;
    }
#undef SEPW_DG_CASE
}

}  // namespace sepw
