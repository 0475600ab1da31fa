// Tensor-core (tcgen05) contraction form of the degridder (the adjoint of the
// contraction gridder of sepw_tc_grid.cu), for BF16 and FP16 operands with
// FP32 accumulation in tensor memory, one-part or split hi + lo.
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
// Hi + lo forms (SPLIT): a = a_hi + a_lo and X = X_hi + X_lo, each part the
// 16-bit rounding of what the higher parts leave (hi = rn(x), lo = rn(x - hi)),
// and Q takes three of the four products, a_hi X_hi + a_hi X_lo + a_lo X_hi,
// as twelve MMAs per stage into the same FP32 accumulator (the dropped
// a_lo X_lo is below 2^-16 (BF16) or 2^-22 (FP16) of |a| |X|).  The
// epilogue's u-taps are then FP32.
//
// Operands are K-major:
//   - A, per stage: row i (slot i) is 128 bytes of K in the 128-byte swizzle
//     layout (16-byte chunk c of row i stored at chunk c ^ (i mod 8) of it,
//     8-row atoms of 1024 bytes).  A per-call table holds, per (plane,
//     oversample, ly mod 4, conj) and split part, the visibility's row
//     relative to its first K chunk ly / 4: five chunks of (re, im) 16-bit
//     pairs and three zero chunks, conjugated for w < 0.  A quarter warp
//     builds one row: lane c copies table chunk c - ly / 4 (zero outside
//     0 .. 4) to K chunk c, so the eight lanes read one 128-byte line and
//     store to eight different bank groups.
//   - B, the window, once per item: each producer takes four cells of one
//     column x (a 16-byte K chunk) and writes the chunk of row (x, re) and of
//     row (x, im) in an order that keeps a quarter warp's stores in distinct
//     bank groups.
//
// Roles (work items assigned to CTAs round robin, so every role walks the
// same items and stages without a shared counter):
//   - eight producer warps in two groups of four, group g owning stage buffer
//     g: it writes the CTA's stages t = g, g + 2, ... (a lane loads the
//     record of one slot, a quarter warp builds one slot's A row at a time).
//     Owning its buffer, a group has itself filled the
//     buffer's previous stage, so its wait for that stage's MMAs is never two
//     mbarrier phases behind.  All eight build each item's window (two
//     buffers, item n in buffer n mod 2) and wait until it is complete
//     before they declare a stage full;
//   - one MMA thread: per stage it waits for "full" and for the accumulator,
//     issues the stage's MMAs (four, twelve for SPLIT) and commits them to
//     the stage's "done" barrier,
//     which both the producers (buffer free) and the epilogue (accumulator
//     ready) wait on: one commit per stage;
//   - four epilogue warps (one per tensor-memory lane quarter), one thread
//     per visibility: it reads its accumulator row into registers, releases
//     the accumulator, shifts the row to its column offset with a barrel
//     shift in registers and takes the u-direction dot product with the
//     u-taps of a second table (16-bit pairs, or complex64 for SPLIT).
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
constexpr int kDgShifts = 4;    // v-table entries per (plane, oversample): ly mod 4 ...
constexpr int kDgConj = 2;      // ... times conj (w < 0) or not
constexpr int kDgUChunks = 4;   // u-table chunks per row: 16 (re, im) 16-bit pairs
constexpr int kDgUChunksF = 8;  // u-table chunks per row: 16 complex64 taps (SPLIT)

// table strides (uint4) and shared memory: [2 buffers][parts] of A (1024-byte
// aligned at run time: 128-byte swizzle), then [2 windows][parts] of B, then
// the barriers
template <int SPLIT>
struct DgCfg {
    static constexpr int kParts = 1 + SPLIT;
    static constexpr int kVEntry = 8 * kParts;  // one 128-byte A row per part
    static constexpr int kVRow = kDgShifts * kDgConj * kVEntry;
    static constexpr int kURow = SPLIT ? kDgUChunksF : kDgUChunks;
    static constexpr size_t kOperandBytes = 2 * kParts * ((size_t)kDgABytes + kDgBBytes);
    static constexpr size_t kSmem = 1024 + kOperandBytes + 16 * sizeof(uint64_t);
    static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
};

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

// part h of the split of (x, y): 0 = hi = rn(v), 1 = lo = rn(v - hi)
template <int PREC>
__device__ __forceinline__ uint32_t pack_part(float x, float y, int h)
{
    const uint32_t hi = pack_pair<PREC>(x, y);
    if (!h)
        return hi;
    const float2 f = unpack_pair<PREC>(hi);
    return pack_pair<PREC>(x - f.x, y - f.y);
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
// u-table, rows of DgCfg<SPLIT>::kVRow and kURow uint4 per (plane, oversample).
struct DgTables {
    uint4 *vtab;
    uint4 *utab;
};

template <int SPLIT>
DgTables dg_tables(const DevParams &p, void *base)
{
    const int64_t nrow = (int64_t)p.P * p.OS;
    unsigned char *b = reinterpret_cast<unsigned char *>(base);
    DgTables t;
    t.vtab = reinterpret_cast<uint4 *>(b);
    t.utab = t.vtab + nrow * DgCfg<SPLIT>::kVRow;
    return t;
}

// Per-call tables from the caller's complex64 taps (v taps at p.voff).  A v
// entry per (plane, oversample, r = ly mod 4, conj) holds per split part the
// 128-byte A row of a visibility with row offset r, relative to its first
// K chunk 4 (ly / 4): chunk j, word q is the (re, im) 16-bit pair of tap
// 4 j + q - r (conjugated for conj; zero outside 0 .. S - 1; chunks 5 .. 7
// zero).  A u row is 16 (re, im) 16-bit pairs, or 16 complex64 taps for the
// split forms; zero beyond S.
template <int PREC, int SPLIT>
__global__ void dg_tables_kernel(DevParams p, const float2 *__restrict__ taps, uint4 *vtab,
                                 uint4 *utab)
{
    using C = DgCfg<SPLIT>;
    constexpr int kV = C::kVRow, kU = C::kURow;
    const int64_t nrow = (int64_t)p.P * p.OS;
    const int64_t nv = nrow * kV, nu = nrow * kU;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nv + nu; e += stride) {
        uint32_t w[4];
        if (e < nv) {
            const int64_t row = e / kV;
            const int rem = (int)(e % kV);
            const int ent = rem / C::kVEntry;  // (r, conj) = (ent / 2, ent % 2)
            const int r = ent >> 1, cj = ent & 1;
            const int h = (rem % C::kVEntry) / 8, j = rem % 8;
            const float2 *tv = taps + p.voff + row * p.S;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = 4 * j + q - r;
                const float2 t = k >= 0 && k < p.S ? tv[k] : make_float2(0.f, 0.f);
                w[q] = pack_part<PREC>(t.x, cj ? -t.y : t.y, h);
            }
            vtab[e] = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
            const int64_t q0 = e - nv;
            const int j = (int)(q0 % kU);
            const int64_t row = q0 / kU;
            const float2 *tu = taps + row * p.S;
            if constexpr (SPLIT) {
                const float2 t0 = 2 * j < p.S ? tu[2 * j] : make_float2(0.f, 0.f);
                const float2 t1 = 2 * j + 1 < p.S ? tu[2 * j + 1] : make_float2(0.f, 0.f);
                w[0] = __float_as_uint(t0.x);
                w[1] = __float_as_uint(t0.y);
                w[2] = __float_as_uint(t1.x);
                w[3] = __float_as_uint(t1.y);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k = 4 * j + q;
                    const float2 t = k < p.S ? tu[k] : make_float2(0.f, 0.f);
                    w[q] = pack_pair<PREC>(t.x, t.y);
                }
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

template <int S, int PREC, int SPLIT>
__global__ void __launch_bounds__(kDgBlock, 1) degrid_tc_kernel(
    DevParams p, const WorkItem *__restrict__ items, const int32_t *__restrict__ nitems,
    const uint64_t *__restrict__ rec, const int32_t *__restrict__ perm,
    const float2 *__restrict__ grid, const float *__restrict__ weight,
    const uint4 *__restrict__ vtab, const uint4 *__restrict__ utab,
    float2 *__restrict__ vis_out, int32_t *status, TcControl ctl)
{
    constexpr int kParts = DgCfg<SPLIT>::kParts;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the 128-byte-swizzle atoms of A need a 1024-byte aligned base (the
    // swizzle is a function of the address); the launch adds 1024 bytes
    unsigned char *const smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *const Abuf = smem;                              // [2][parts] stages
    unsigned char *const Bbuf = smem + 2 * kParts * kDgABytes;     // [2][parts] windows
    uint64_t *const bars = reinterpret_cast<uint64_t *>(smem + DgCfg<SPLIT>::kOperandBytes);
    uint64_t *const full = bars, *const done = bars + 2, *const tfree = bars + 4,
                    *const efree = bars + 6, *const bready = bars + 8, *const drain = bars + 10,
                    *const wmax = bars + 11;  // [2]
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ float s_wmax[2][kDgProdWarps];  // FP16: per-warp window maxima

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_items = *nitems;
    const int W = p.T + S - 1;

    for (int e = tid; e < (int)(DgCfg<SPLIT>::kOperandBytes / 16); e += kDgBlock)
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
        const int wg = warp % kDgGroupWarps;   // slots 32 wg .. 32 wg + 31 of its stages
        const int ii = tid & (kDgVis - 1);     // the slot whose record this lane loads
        const int qd = lane >> 3, c = lane & 7;  // quarter warp, K chunk of a row
        unsigned char *const A = Abuf + grp * kParts * kDgABytes;  // part h at + h kDgABytes
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
            // cells (x, 4 yq + q), q = 0 .. 3: one 16-byte K chunk of the
            // window rows (x, re) and (x, im)
            constexpr int kCells = 4;
            static_assert(kDgWin * kDgWin == kCells * kDgProducers, "window cells per producer");
            const int wx = tid & 31, yq = tid >> 5;
            float2 gv[kCells];
#pragma unroll
            for (int q = 0; q < kCells; ++q) {
                const int y = 4 * yq + q;
                gv[q] = make_float2(0.f, 0.f);
                if (y < W && wx < W && o.gy0 + y < p.N && o.gx0 + wx < p.N)
                    gv[q] = __ldg(grid + o.base + (o.gy0 + y) * p.N + o.gx0 + wx);
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
            unsigned char *const B = Bbuf + ib * kParts * kDgBBytes;
            // row (x, re): (X_r, X_i) at K = (y, 0), (y, 1); row (x, im):
            // (X_i, -X_r); part h of the split in B + h kDgBBytes.  Lanes
            // with x mod 8 >= 4 write their im row first, so that the eight
            // rows a quarter warp writes fall in eight different 16-byte
            // bank groups
            const int pf = (wx >> 2) & 1;
#pragma unroll
            for (int h = 0; h < kParts; ++h) {
                uint32_t wre[kCells], wim[kCells];
#pragma unroll
                for (int q = 0; q < kCells; ++q) {
                    wre[q] = pack_part<PREC>(gv[q].x * scale, gv[q].y * scale, h);
                    const float2 f = unpack_pair<PREC>(wre[q]);
                    wim[q] = pack_pair<PREC>(f.y, -f.x);  // exact: a part negated
                }
                const uint4 vre = make_uint4(wre[0], wre[1], wre[2], wre[3]);
                const uint4 vim = make_uint4(wim[0], wim[1], wim[2], wim[3]);
                unsigned char *const Bh = B + h * kDgBBytes;
                st16(Bh + dg_off(2 * wx + pf, 8 * yq), pf ? vim : vre);
                st16(Bh + dg_off(2 * wx + 1 - pf, 8 * yq), pf ? vre : vim);
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
                // this lane's slot: its table entry (plane, oversample,
                // ly mod 4, conj) and first K chunk ly / 4, or 8 for an empty
                // slot (every chunk zero); no record has its top bits set
                uint32_t info = 8u;
                if (rcur != ~0ull) {
                    const uint64_t r = rcur;
                    const int ly = rec_ly(r);
                    const uint32_t ent =
                        ((uint32_t)(rec_plane(r) * p.OS + rec_ov(r)) * kDgShifts + (ly & 3)) *
                            kDgConj + (rec_conj(r) ? 1u : 0u);
                    info = (ent << 4) | (uint32_t)(ly >> 2);
                }
                // quarter warp qd builds the rows of slots 32 wg + 4 k + qd,
                // lane c of it K chunk c: table chunk c - ly / 4 (zero outside
                // 0 .. 4), one 128-byte line per row and part
                uint4 val[8][kParts];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t inf = __shfl_sync(0xffffffffu, info, 4 * k + qd);
                    const int j = c - (int)(inf & 15u);
                    const uint4 *src = vtab + (size_t)(inf >> 4) * DgCfg<SPLIT>::kVEntry;
#pragma unroll
                    for (int h = 0; h < kParts; ++h)
                        val[k][h] = (unsigned)j <= 4u ? __ldg(src + 8 * h + j) : make_uint4(0, 0, 0, 0);
                }
                // buffer grp held stage t - 2: wait for its MMAs
                if (t >= 2)
                    warp_wait(done + grp, ((t - 2) >> 1) & 1);
                tc_fence_after();
                // 128-byte swizzle: chunk c of row `slot` at chunk c ^ (slot mod 8)
                // of the row, so a quarter warp's eight stores hit eight bank groups
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int slot = 32 * wg + 4 * k + qd;
                    const uint32_t off =
                        (uint32_t)((slot >> 3) * 1024 + (slot & 7) * 128 + ((c ^ (slot & 7)) << 4));
#pragma unroll
                    for (int h = 0; h < kParts; ++h)
                        st16(A + h * kDgABytes + off, val[k][h]);
                }
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
            const uint64_t da0 = smem_desc_sw128k(smem_u32(Abuf));
            const uint64_t db0 = smem_desc(smem_u32(Bbuf), kDgLbo, kDgSbo);
            constexpr uint64_t kStepA = 32 >> 4;            // K = 16: 32 bytes of the row
            constexpr uint64_t kStep = (2 * kDgLbo) >> 4;   // K = 16: two core matrices
            int tg = 0;
            bool ok = true, issued = false;
            for (int n = 0; ok; ++n) {
                const int item = blockIdx.x + n * gridDim.x;
                if (item >= n_items)
                    break;
                const int nst = (items[item].count + kDgVis - 1) / kDgVis;
                const uint64_t db = db0 + (uint64_t)((n & 1) * kParts * kDgBBytes >> 4);
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
                    const uint64_t da = da0 + (uint64_t)((b * kParts * kDgABytes) >> 4);
                    const uint32_t d = tmem + (uint32_t)(b * kDgN);
#pragma unroll
                    for (int kq = 0; kq < kDgK / 16; ++kq) {
                        mma_f16(d, da + kStepA * kq, db + kStep * kq, idesc, kq > 0 ? 1u : 0u);
                        if constexpr (SPLIT) {
                            // a_hi X_lo and a_lo X_hi (the lo parts kDgABytes /
                            // kDgBBytes above the hi parts)
                            constexpr uint64_t kLoA = kDgABytes >> 4, kLoB = kDgBBytes >> 4;
                            mma_f16(d, da + kStepA * kq, db + kLoB + kStep * kq, idesc, 1u);
                            mma_f16(d, da + kLoA + kStepA * kq, db + kStep * kq, idesc, 1u);
                        }
                    }
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
                // the u-taps: 16 (re, im) 16-bit words, or for the split
                // forms kUq 32-byte loads of four complex64 taps
                constexpr int kUq = SPLIT ? (S + 3) / 4 : 2;
                uint4 uu[2 * kUq];
#pragma unroll
                for (int k = 0; k < 2 * kUq; ++k)
                    uu[k] = make_uint4(0, 0, 0, 0);
                if (valid) {
                    iout = io;
                    wt = (weight ? __ldg(weight + iout) : 1.0f) * back;
                    lx = rec_lx(r);
                    sg = rec_conj(r) ? 1.f : -1.f;  // tu' = conj(tu) unless w < 0
                    const uint4 *pu =
                        utab + ((int64_t)rec_plane(r) * p.OS + rec_ou(r)) * DgCfg<SPLIT>::kURow;
#pragma unroll
                    for (int k = 0; k < kUq; ++k)
                        ldg32(pu + 2 * k, uu[2 * k], uu[2 * k + 1]);
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
                    float vr = 0.f, vi = 0.f;
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        float2 u;
                        if constexpr (SPLIT) {
                            const uint4 &w4 = uu[j >> 1];
                            u = (j & 1) ? make_float2(__uint_as_float(w4.z), __uint_as_float(w4.w))
                                        : make_float2(__uint_as_float(w4.x), __uint_as_float(w4.y));
                        } else {
                            u = unpack_pair<PREC>((&uu[j >> 2].x)[j & 3]);
                        }
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

template <int S, int PREC, int SPLIT>
cudaError_t launch_degrid_tc_S(const DevParams &p, const Plan &plan, const float2 *grid,
                               const float *weight, const float2 *taps, void *tables,
                               float2 *vis, int num_sms, int32_t *status, TcControl ctl,
                               cudaStream_t s)
{
    using C = DgCfg<SPLIT>;
    const DgTables t = dg_tables<SPLIT>(p, tables);
    const int64_t nrow = (int64_t)p.P * p.OS;
    const int64_t n = nrow * (C::kVRow + C::kURow);
    dg_tables_kernel<PREC, SPLIT><<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(
        p, taps, t.vtab, t.utab);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(degrid_tc_kernel<S, PREC, SPLIT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmem);
    if (e != cudaSuccess)
        return e;
    degrid_tc_kernel<S, PREC, SPLIT><<<num_sms, kDgBlock, C::kSmem, s>>>(
        p, plan.d_items, plan.d_nitems, plan.d_rec, plan.d_perm, grid, weight, t.vtab, t.utab,
        vis, status, ctl);
    return cudaGetLastError();
}

}  // namespace

size_t tc_degrid_tables_bytes(const DevParams &p, int64_t items_capacity)
{
    (void)items_capacity;
    // rows sized for the split forms (the larger)
    const size_t nrow = (size_t)p.P * p.OS;
    return align256(nrow * (DgCfg<1>::kVRow + DgCfg<1>::kURow) * 16);
}

cudaError_t launch_degrid_tc(const DevParams &p, const Plan &plan, const float2 *grid,
                             const float *weight, const float2 *taps, void *tables, float2 *vis,
                             int num_sms, int prec, int32_t *status, TcControl ctl,
                             cudaStream_t s)
{
    if (p.T + p.S - 1 > kDgWin || p.S > 16 || prec < 0 || prec > 3)
        return cudaErrorInvalidValue;
    // prec 0 = BF16, 1 = FP16, 2 = FP16 hi + lo, 3 = BF16 hi + lo
#define SEPW_DG_CASE(SS)                                                                     \
    case SS:                                                                                 \
        switch (prec) {                                                                      \
        case 0:                                                                              \
            return launch_degrid_tc_S<SS, 0, 0>(p, plan, grid, weight, taps, tables, vis,    \
                                                num_sms, status, ctl, s);                    \
        case 1:                                                                              \
            return launch_degrid_tc_S<SS, 1, 0>(p, plan, grid, weight, taps, tables, vis,    \
                                                num_sms, status, ctl, s);                    \
        case 2:                                                                              \
            return launch_degrid_tc_S<SS, 1, 1>(p, plan, grid, weight, taps, tables, vis,    \
                                                num_sms, status, ctl, s);                    \
        default:                                                                             \
            return launch_degrid_tc_S<SS, 0, 1>(p, plan, grid, weight, taps, tables, vis,    \
                                                num_sms, status, ctl, s);                    \
        }
    switch (p.S) {
        SEPW_DG_CASE(2) SEPW_DG_CASE(4) SEPW_DG_CASE(6) SEPW_DG_CASE(8) SEPW_DG_CASE(10)
        SEPW_DG_CASE(12) SEPW_DG_CASE(14) SEPW_DG_CASE(16)
    default:
        return cudaErrorInvalidValue;
    }
#undef SEPW_DG_CASE
}

}  // namespace sepw
