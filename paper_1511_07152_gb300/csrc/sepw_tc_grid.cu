// Tensor-core (tcgen05) contraction form of the separable gridder with
// MN-major operands built by 16-byte stores from unshifted tap tables.
//
// Sec. 5 writes the update of a visibility as the separable product
// W V F1(u - u_i) F1(v - v_i).  Summed over the visibilities of one tile it is
// a dense complex contraction over the tile's window (T + S - 1 <= 32 cells a
// side): with a_i[y] the v-taps of visibility i at its row offset and
// b'_i[x] = W_i V_i times its u-taps at its column offset,
//     G[y][x] = sum_i a_i[y] b'_i[x].
// In real arithmetic the 16-bit forms take K = visibility and put the real
// and imaginary parts of both factors in M and N, one tcgen05.mma of shape
// M = 64 H, N = 64 H per K = 16 visibilities:
//     rows    m = 64 h + 32 c + y    (h: split part of a, c: re/im of a, y: row)
//     columns n = 64 g + 32 d + x    (g: split part of b', d: re/im of b', x)
//     A[(h,c,y)][i] = a_h,c[y]       B[i][(g,d,x)] = b'_g,d[x]
// so the accumulator holds the four real products summed over the
// visibilities, D[(h,c,y)][(g,d,x)], and the epilogue forms
//     Re G = sum_h,g D[(h,0,y)][(g,0,x)] - D[(h,1,y)][(g,1,x)]
//     Im G = sum_h,g D[(h,0,y)][(g,1,x)] + D[(h,1,y)][(g,0,x)].
// a_h (b'_g) is the h-th (g-th) part of the 16-bit split of the taps (of W V
// times the taps): H = 1 for the one-part forms, H = 2 for the hi + lo forms,
// where one MMA yields all four products of the splits.  The TF32 form uses
// the same embedding (H = 1, K = 8 visibilities per MMA) with K-major
// operands, since MN-major TF32 operands gave zeros on the GB300: a
// visibility's column of A and row of B are one 4-byte element in each of 64
// rows, so every lane shifts its taps to absolute rows (columns) in registers
// and the warp stores one row at a time.
//
// The 16-bit operands are MN-major: a visibility's column of A (and its row
// of B) is contiguous along M (N) in 16-byte pieces of 8 values, so it is
// written as whole 16-byte chunks.  They come from tables built per call from
// the caller's complex64 taps, one unshifted row per (plane, oversample):
//   vtab: the S v-taps as 16-bit pairs (2 w, 2 w + 1) per split part and
//         component (zero beyond S);
//   utab: the S u-taps, as (re, im) 16-bit pairs (one-part forms) or
//         complex64 (hi + lo forms), multiplied by W V in FP32 before
//         rounding.
// A lane moves its 16 v values to the row offset ly mod 8 within three
// 8-value chunks in registers (shift16: two word shifts and a half-word step),
// and likewise its W V u products to the column offset lx mod 8.  Chunk j of a
// visibility whose footprint starts at row ly goes to chunk row j + ly / 8 of
// its column: the placement is a computed store address, and the chunk rows
// its footprint misses get zeros, so each stage overwrites every byte its
// visibilities own and no buffer ever needs clearing.
//
// One lane per visibility: a stage is 64 visibilities, written by a pair of
// producer warps (32 each).  Slot i is K row i % 8 of core-matrix group i / 8,
// so the 8 lanes of a quarter warp write the 8 rows of one aligned 128-byte
// core matrix: no bank conflicts, whatever chunk row each lane writes, and no
// padding between the core matrices the MMA reads.
//
// Roles (static round-robin assignment of the plan's work items to CTAs, so
// every role walks the same sequence of items and stages):
//   - eight producer warps in four pairs, each pair owning one of four stage
//     buffers: pair p takes the CTA's stages p, p + 4, ...  Owning its
//     buffer, a warp has itself filled the buffer's previous stage, so its
//     wait for that stage's MMAs can never be two mbarrier phases ahead (a
//     parity wait cannot tell those apart): the buffer's "empty" barrier
//     cannot complete this round before the warp's own half of the round's
//     stage has arrived.  A lane loads its record one stage ahead, then its
//     taps and value, waits for the buffer, writes its A column and B row,
//     and the warp arrives on the buffer's "full" mbarrier (two arrivals);
//   - one MMA thread: per stage it waits for "full", issues the MMAs (four of
//     K = 16 for the 16-bit forms) and commits them to the buffer's "empty"
//     mbarrier.  Per work item it accumulates into one of two tensor-memory
//     accumulators and commits "accf" after the item's last stage.  This
//     thread's per-stage chain (wait, issue, commit: about 550 cycles for
//     32-visibility stages, measured) is what stages of 64 halve;
//   - four epilogue warps (one per tensor-memory lane quarter): per item they
//     read the accumulator, release it ("accfree"), stage it in shared memory
//     and add the window to the HBM grid with float2 atomics (windows of
//     neighbouring tiles overlap).
// Every mbarrier wait is bounded; on expiry the kernel records SEPW_ETIMEOUT,
// every role leaves its loop, the MMA thread waits (bounded) for its own MMAs
// and the tensor memory is freed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "sepw_internal.cuh"
#include "sepw_tc_ptx.cuh"

namespace sepw {
namespace {

using namespace tcx;

constexpr int kProd = 8;                       // producer warps
constexpr int kWps = 2;                        // producer warps per stage
constexpr int kBufs = kProd / kWps;            // stage buffers, one per warp pair
static_assert((kBufs & (kBufs - 1)) == 0, "the issue loop takes t mod kBufs as a mask");
// Buffers may be released in groups of kGroup consecutive buffers (one
// tcgen05.commit per group); each group's "empty" barrier still completes
// once per round of kBufs stages.  Measured: groups gave nothing.
constexpr int kGroup = 1;
static_assert(kBufs % kGroup == 0, "groups tile the buffers");
constexpr int kWin = 32;                       // window edge, T + S - 1 <= 32
constexpr uint32_t kSboA = 128;                // M-adjacent core matrices
constexpr int kEpiWarps = 4;

// PREC: 0 = BF16, 1 = FP16 (scaled per item), 2 = FP16 hi + lo (scaled),
// 3 = BF16 hi + lo, 4 = TF32
template <int PREC>
struct Cfg {
    static constexpr int H = (PREC == 2 || PREC == 3) ? 2 : 1;  // split parts
    static constexpr bool SCALED = PREC == 1 || PREC == 2;
    static constexpr bool BF = PREC == 0 || PREC == 3;
    // TF32: K-major operands of 4-byte elements (MN-major TF32 operands gave
    // zeros on the GB300); K = 8 per MMA
    static constexpr bool TF32 = PREC == 4;
    // N: columns (g, d, x)
    static constexpr int N = 64 * H;
    // M = 64 H rows: (h, c, y).  An M = 64 accumulator puts row m in tensor-
    // memory lane 32 (m / 16) + m % 16 (measured), the first 16 lanes of each
    // warp quarter.
    static constexpr int M = 64 * H;
    static constexpr int SV = 32 * kWps;                   // visibilities per stage
    static constexpr int SLOTS = 1;                        // per lane
    // core matrices along K per stage: 8 visibilities each (16-bit forms), or
    // 4 (TF32)
    static constexpr int KG = TF32 ? SV / 4 : SV / 8;
    static constexpr int VPK = TF32 ? 8 : 16;              // visibilities per MMA
    // values and weights loaded one stage ahead (the one-part forms; the hi +
    // lo forms have no registers to spare: measured slower)
    static constexpr bool PRE = H == 1;
    // u-side table in the 16-bit format (the one-part forms: W V times the
    // rounded taps, rounded again); FP32 for the hi + lo forms
    static constexpr bool U16 = H == 1 && !TF32;
    // K-adjacent core matrices: 128-byte aligned for the 16-bit forms; TF32
    // pads by 16 bytes, so that 32 lanes storing 4 bytes of one row each
    // (four lanes a core-matrix row) hit eight different 16-byte bank groups
    static constexpr uint32_t kPad = TF32 ? 16 : 0;
    static constexpr uint32_t kLboA = (M / 8) * 128 + kPad;
    static constexpr int kABytes = KG * kLboA;
    // staged accumulator row: (d, x) summed over g; padded
    static constexpr int kStgStride = 65;
    static constexpr int kStgBytes = M * kStgStride * 4;
    static constexpr uint32_t kSboB = 128;
    static constexpr uint32_t kLboB = (N / 8) * 128 + kPad;
    static constexpr int kBBytes = KG * kLboB;
    static constexpr int kProdWarps = kProd;  // 13 warps: up to 128 registers each
    static constexpr int kMmaWarp = kProdWarps;
    static constexpr int kEpiWarp0 = kProdWarps + 1;
    static constexpr int kBlock = 32 * (kProdWarps + 1 + kEpiWarps);
    static constexpr uint32_t kTmemCols = 2 * N;  // two accumulators
    static constexpr size_t kSmem = (size_t)kBufs * (kABytes + kBBytes) + kStgBytes +
                                    sizeof(uint64_t) * (2 * kBufs + 5);
    static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
};

// (x, y) rounded to the 16-bit format, part h: 0 = hi = rn(v), 1 = lo = rn(v - hi)
template <bool BF>
__device__ __forceinline__ uint32_t pack_part(float x, float y, int h)
{
    if constexpr (BF) {
        __nv_bfloat162 hi = __floats2bfloat162_rn(x, y);
        if (h) {
            const float2 f = __bfloat1622float2(hi);
            hi = __floats2bfloat162_rn(x - f.x, y - f.y);
        }
        return *reinterpret_cast<uint32_t *>(&hi);
    } else {
        __half2 hi = __floats2half2_rn(x, y);
        if (h) {
            const float2 f = __half22float2(hi);
            hi = __floats2half2_rn(x - f.x, y - f.y);
        }
        return *reinterpret_cast<uint32_t *>(&hi);
    }
}

// (x, y) of a pair of 16-bit values (exact)
template <bool BF>
__device__ __forceinline__ float2 unpack_part(uint32_t w)
{
    if constexpr (BF) {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    } else {
        return __half22float2(*reinterpret_cast<const __half2 *>(&w));
    }
}

// Moves 16 packed 16-bit values v[0..15] (pairs in in[0..7], zero beyond) to
// positions s .. s + 15 of 24 (pairs in out[0..11]), s = 0..7: two
// conditional word shifts and one half-word step (__byte_perm takes the high
// half of the lower word and the low half of the higher).
__device__ __forceinline__ void shift16(const uint32_t (&in)[8], int s, uint32_t (&out)[12])
{
    uint32_t t[12];
#pragma unroll
    for (int w = 0; w < 12; ++w)
        t[w] = w < 8 ? in[w] : 0u;
    const int m = s >> 1;
#pragma unroll
    for (int w = 11; w >= 0; --w)
        t[w] = (m & 2) ? (w >= 2 ? t[w - 2] : 0u) : t[w];
#pragma unroll
    for (int w = 11; w >= 0; --w)
        t[w] = (m & 1) ? (w >= 1 ? t[w - 1] : 0u) : t[w];
#pragma unroll
    for (int w = 0; w < 12; ++w)
        out[w] = (s & 1) ? __byte_perm(w >= 1 ? t[w - 1] : 0u, t[w], 0x5432) : t[w];
}

__device__ __forceinline__ void st16(unsigned char *p, uint4 v)
{
    *reinterpret_cast<uint4 *>(p) = v;
}

// One 32-byte read-only global load (a and b: the two 16-byte halves); p is
// 32-byte aligned.  A lane's table rows take half as many gathered accesses
// as with 16-byte loads.
__device__ __forceinline__ void ldg32(const void *p, uint4 &a, uint4 &b)
{
    asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z),
                   "=r"(b.w)
                 : "l"(p));
}

// FP32 -> TF32, round to nearest (ties away), as a 32-bit pattern
__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void st4(unsigned char *p, uint32_t a)
{
    *reinterpret_cast<uint32_t *>(p) = a;
}

// byte offset of row m of a K-major core-matrix column (8 rows of 16 bytes,
// 8-row groups 128 bytes apart)
__device__ __forceinline__ uint32_t tf32_row_off(int m)
{
    return (uint32_t)((m & 7) * 16 + (m >> 3) * 128);
}

// v[k] <- v[k - s] (zero below s), s = 0..31: one conditional shift per bit
__device__ __forceinline__ void shift_right32(float (&v)[32], int s)
{
#pragma unroll
    for (int b = 4; b >= 0; --b) {
        const int sh = 1 << b;
        const bool on = (s >> b) & 1;
#pragma unroll
        for (int k = 31; k >= 0; --k)
            v[k] = on ? (k >= sh ? v[k - sh] : 0.f) : v[k];
    }
}

// Per-call tables (layouts in the file comment): unshifted rows per (plane,
// oversample).  v (from the v-direction taps at voff): KV = 4 H uint4 =
// [part h][component][8 words of tap pairs (2 w, 2 w + 1)], zero beyond S,
// or 16 complex64 taps (TF32); u: KU uint4 = 16 (re, im) 16-bit words
// (one-part 16-bit forms) or 16 complex64 taps (hi + lo forms, TF32).
template <int PREC>
__global__ void tables_kernel(DevParams p, const float2 *__restrict__ taps, uint4 *vtab,
                              uint4 *utab)
{
    constexpr int H = Cfg<PREC>::H;
    constexpr bool U16 = Cfg<PREC>::U16, TF32 = Cfg<PREC>::TF32;
    constexpr int KV = TF32 ? 8 : 4 * H, KU = U16 ? 4 : 8;
    const int64_t nrow = (int64_t)p.P * p.OS;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nrow * (KV + KU);
         e += stride) {
        const int64_t row = e / (KV + KU);
        const int q = (int)(e % (KV + KU));
        uint32_t w[4];
        if (TF32 && q < KV) {  // complex64 v taps 2 q, 2 q + 1
            const float2 *tv = taps + p.voff + row * p.S;
            const float2 t0 = 2 * q < p.S ? tv[2 * q] : make_float2(0.f, 0.f);
            const float2 t1 = 2 * q + 1 < p.S ? tv[2 * q + 1] : make_float2(0.f, 0.f);
            vtab[row * KV + q] = make_uint4(__float_as_uint(t0.x), __float_as_uint(t0.y),
                                            __float_as_uint(t1.x), __float_as_uint(t1.y));
        } else if (q < KV) {
            const int h = q >> 2, comp = (q >> 1) & 1, half = q & 1;
            const float2 *tv = taps + p.voff + row * p.S;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int t0 = 2 * (4 * half + k);
                const float a = t0 < p.S ? (comp ? tv[t0].y : tv[t0].x) : 0.f;
                const float b = t0 + 1 < p.S ? (comp ? tv[t0 + 1].y : tv[t0 + 1].x) : 0.f;
                w[k] = pack_part<Cfg<PREC>::BF>(a, b, h);
            }
            vtab[row * KV + q] = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
            const int qu = q - KV;
            const float2 *tu = taps + row * p.S;
            if constexpr (U16) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int t0 = 4 * qu + k;
                    const float2 t = t0 < p.S ? tu[t0] : make_float2(0.f, 0.f);
                    w[k] = pack_part<Cfg<PREC>::BF>(t.x, t.y, 0);
                }
            } else {
                const float2 t0 = 2 * qu < p.S ? tu[2 * qu] : make_float2(0.f, 0.f);
                const float2 t1 = 2 * qu + 1 < p.S ? tu[2 * qu + 1] : make_float2(0.f, 0.f);
                w[0] = __float_as_uint(t0.x);
                w[1] = __float_as_uint(t0.y);
                w[2] = __float_as_uint(t1.x);
                w[3] = __float_as_uint(t1.y);
            }
            utab[row * KU + qu] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Power-of-two exponent a per work item such that the item's largest |W V|
// component is below 2^a (FP16 forms scale their B operand by 2^-a).
__global__ void item_scale_kernel(const WorkItem *__restrict__ items,
                                  const int32_t *__restrict__ nitems,
                                  const int32_t *__restrict__ perm,
                                  const float2 *__restrict__ vis, const float *__restrict__ weight,
                                  int32_t *item_exp)
{
    __shared__ float s_red[8];
    const int n_items = *nitems;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const WorkItem it = items[item];
        float m = 0.f;
        for (int e = threadIdx.x; e < it.count; e += blockDim.x) {
            const int i = perm[it.start + e];
            const float2 x = __ldg(vis + i);
            const float wt = weight ? __ldg(weight + i) : 1.0f;
            m = fmaxf(m, fmaxf(fabsf(wt * x.x), fabsf(wt * x.y)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0)
            s_red[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                m = fmaxf(m, s_red[w]);
            int a = 0;
            if (m > 0.f && m <= 3.0e38f) {
                frexpf(m, &a);  // m = f 2^a, f in [0.5, 1)
                a = max(-126, min(126, a));
            }
            item_exp[item] = a;
        }
        __syncthreads();
    }
}

// The CTA's work items in order (static round robin) and the global index of
// each item's first stage.
struct Cursor {
    int n = -1;      // ordinal of the item in this CTA's sequence
    int item = 0;    // plan index of the item
    int nst = 0;     // its stages
    int tb = 0;      // CTA stage index of its first stage
    int start = 0, count = 0, tile = 0;
};

template <int SV>
__device__ __forceinline__ bool cursor_next(Cursor &c, const WorkItem *__restrict__ items,
                                            int n_items)
{
    c.tb += c.nst;
    ++c.n;
    c.item = blockIdx.x + c.n * gridDim.x;
    if (c.item >= n_items) {
        c.nst = 0;
        return false;
    }
    const WorkItem it = items[c.item];
    c.start = it.start;
    c.count = it.count;
    c.tile = it.tile;
    c.nst = (it.count + SV - 1) / SV;
    return true;
}

// advance c to the item holding CTA stage t (false: past the last item)
template <int SV>
__device__ __forceinline__ bool cursor_seek(Cursor &c, int t, const WorkItem *__restrict__ items,
                                            int n_items)
{
    while (t >= c.tb + c.nst)
        if (!cursor_next<SV>(c, items, n_items))
            return false;
    return true;
}

template <int PREC>
__global__ void __launch_bounds__(Cfg<PREC>::kBlock, 1) grid_tc2_kernel(
    DevParams p, const WorkItem *__restrict__ items, const int32_t *__restrict__ nitems,
    const uint64_t *__restrict__ rec, const int32_t *__restrict__ perm,
    const float2 *__restrict__ vis, const float *__restrict__ weight,
    const uint4 *__restrict__ vtab, const uint4 *__restrict__ utab,
    const float2 *__restrict__ taps, const int32_t *__restrict__ item_exp, float2 *grid,
    int32_t *status, TcControl ctl)
{
    using C = Cfg<PREC>;
    constexpr int H = C::H, N = C::N, SV = C::SV;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *const Abuf = smem;                          // [kBufs]
    unsigned char *const Bbuf = smem + kBufs * C::kABytes;     // [kBufs]
    float *const stg = reinterpret_cast<float *>(Bbuf + kBufs * C::kBBytes);
    uint64_t *const full =
        reinterpret_cast<uint64_t *>(Bbuf + kBufs * C::kBBytes + C::kStgBytes);
    uint64_t *const empty = full + kBufs;
    uint64_t *const accf = empty + kBufs;     // [2]
    uint64_t *const accfree = accf + 2;       // [2]
    uint64_t *const drain = accfree + 2;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ int s_epi_ok[kEpiWarps];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_items = *nitems;

    // operand bytes every stage overwrites; zeroed once for a clean start
    for (int e = tid; e < kBufs * C::kABytes / 16; e += C::kBlock)
        reinterpret_cast<uint4 *>(Abuf)[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int b = 0; b < kBufs; ++b) {
            mbar_init(full + b, kWps);
            mbar_init(empty + b, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf + b, 1);
            mbar_init(accfree + b, kEpiWarps);
        }
        mbar_init(drain, 1);
        s_abort = 0;
        mbar_init_fence();
    }
    if (warp == 0)
        tmem_alloc(&s_tmem, C::kTmemCols);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp < C::kProdWarps) {
        // ------------------------------------------------------------ producers
        Cursor cur;
        int t = warp / kWps;                // the pair's first stage
        const int slot0 = 32 * (warp % kWps);  // this warp's half of a stage
        bool ok = cursor_next<SV>(cur, items, n_items) && cursor_seek<SV>(cur, t, items, n_items);
        // records and visibility indices of the lane's slots one stage ahead,
        // and with C::PRE their values and weights (random gathers from HBM)
        uint64_t r[C::SLOTS];
        int vi[C::SLOTS];
        float2 xv[C::SLOTS];
        float wv[C::SLOTS];
        auto fetch = [&](const Cursor &c, int t_, uint64_t (&r_)[C::SLOTS],
                         int (&vi_)[C::SLOTS], float2 (&x_)[C::SLOTS], float (&w_)[C::SLOTS]) {
#pragma unroll
            for (int sl = 0; sl < C::SLOTS; ++sl) {
                const int e = (t_ - c.tb) * SV + slot0 + 32 * sl + lane;
                vi_[sl] = -1;
                if (e < c.count) {
                    r_[sl] = __ldg(reinterpret_cast<const unsigned long long *>(rec) + c.start +
                                   e);
                    vi_[sl] = __ldg(perm + c.start + e);
                }
            }
#pragma unroll
            for (int sl = 0; sl < C::SLOTS; ++sl) {
                x_[sl] = make_float2(0.f, 0.f);
                w_[sl] = 0.f;
                if (C::PRE && vi_[sl] >= 0) {
                    x_[sl] = __ldg(vis + vi_[sl]);
                    w_[sl] = weight ? __ldg(weight + vi_[sl]) : 1.0f;
                }
            }
        };
        if (ok)
            fetch(cur, t, r, vi, xv, wv);
        while (ok && !s_abort) {
            Cursor cn = cur;
            const int tn = t + kBufs;
            bool okn = false;
            uint64_t rn[C::SLOTS];
            int vin[C::SLOTS];
            float2 xn[C::SLOTS];
            float wn[C::SLOTS];
#pragma unroll
            for (int sl = 0; sl < C::SLOTS; ++sl) {
                vin[sl] = -1;
                xn[sl] = make_float2(0.f, 0.f);
                wn[sl] = 0.f;
            }
            float scale = 1.0f;
            if constexpr (C::SCALED)
                scale = ldexpf(1.0f, -__ldg(item_exp + cur.item));
            const int b = t % kBufs;
            unsigned char *const A = Abuf + b * C::kABytes;
            unsigned char *const B = Bbuf + b * C::kBBytes;
            const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int sl = 0; sl < C::SLOTS; ++sl) {
                const int i = slot0 + 32 * sl + lane;  // slot in the stage
                if constexpr (C::TF32) {
                    // K-major, 4-byte elements: slot i is K = i; its column of A
                    // (rows (c, y)) and row of B (columns (d, x)) are one 4-byte
                    // element in each of 64 rows, which all lanes store together
                    uint4 vq[8], uq[8];  // 16 complex64 v- and u-taps, unshifted
                    float2 x = make_float2(0.f, 0.f);
                    float wt = 0.f;
                    int lx = 0, ly = 0;
                    bool cj = false;
                    const bool valid = vi[sl] >= 0;
                    if (valid) {
                        x = xv[sl];
                        wt = wv[sl];
                        lx = rec_lx(r[sl]);
                        ly = rec_ly(r[sl]);
                        cj = rec_conj(r[sl]);
                        const int64_t row = (int64_t)rec_plane(r[sl]) * p.OS;
                        const uint4 *pv = vtab + (row + rec_ov(r[sl])) * 8;
                        const uint4 *pu = utab + (row + rec_ou(r[sl])) * 8;
#pragma unroll
                        for (int k = 0; k < 8; k += 2) {
                            ldg32(pv + k, vq[k], vq[k + 1]);
                            ldg32(pu + k, uq[k], uq[k + 1]);
                        }
                    }
                    if (sl == 0) {
                        okn = cursor_seek<SV>(cn, tn, items, n_items);
                        if (okn)
                            fetch(cn, tn, rn, vin, xn, wn);
                    }
                    if (sl == 0 && t >= kBufs) {
                        if (lane == 0 && !s_abort &&
                            !mbar_wait(empty + b / kGroup, ((t / kBufs) - 1) & 1, ctl.wait_ns))
                            s_abort = 1;
                        __syncwarp();
                        tc_fence_after();
                    }
                    // element (m, k) at (k % 4) 4 + (k / 4) LBO + (m % 8) 16 + (m / 8) 128
                    unsigned char *const Ak = A + (i & 3) * 4 + (i >> 2) * C::kLboA;
                    unsigned char *const Bk = B + (i & 3) * 4 + (i >> 2) * C::kLboB;
                    auto tap = [](const uint4 (&q)[8], int j) {  // complex tap j
                        const uint4 w = q[j >> 1];
                        return (j & 1) ? make_float2(__uint_as_float(w.z), __uint_as_float(w.w))
                                       : make_float2(__uint_as_float(w.x), __uint_as_float(w.y));
                    };
                    // A: component c of a (conj for w < 0) at rows ly .. ly + S - 1
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        float col[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float2 a = j < 16 ? tap(vq, j) : make_float2(0.f, 0.f);
                            col[j] = !valid ? 0.f : c ? (cj ? -a.y : a.y) : a.x;
                        }
                        shift_right32(col, ly);
#pragma unroll
                        for (int y = 0; y < 32; ++y)
                            st4(Ak + tf32_row_off(32 * c + y), to_tf32(col[y]));
                    }
                    // B: W V times the u-taps (conj for w < 0), component d at
                    // columns lx .. lx + S - 1
                    const float wr = wt * x.x, wi = wt * x.y;
                    float bre[16], bim[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float2 u = tap(uq, j);
                        const float ur = u.x, ui = cj ? -u.y : u.y;
                        bre[j] = wr * ur - wi * ui;
                        bim[j] = wr * ui + wi * ur;
                    }
#pragma unroll
                    for (int d = 0; d < 2; ++d) {
                        float col[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            col[j] = (!valid || j >= 16) ? 0.f : d ? bim[j] : bre[j];
                        shift_right32(col, lx);
#pragma unroll
                        for (int xx = 0; xx < 32; ++xx)
                            st4(Bk + tf32_row_off(32 * d + xx), to_tf32(col[xx]));
                    }
                } else {
                // this slot's taps and value: unshifted table rows (v: 16-bit
                // words [h][component][8]; u: 16 (re, im) 16-bit words for the
                // one-part forms, 16 complex64 taps for the hi + lo forms)
                uint4 vq[H][4];
                uint4 uq[C::U16 ? 4 : 8];
                float2 x = make_float2(0.f, 0.f);
                float wt = 0.f;
                int lx = 0, ly = 0;
                uint32_t cjm = 0;
                const bool valid = vi[sl] >= 0;
                if (valid) {
                    if constexpr (C::PRE) {
                        x = xv[sl];
                        wt = wv[sl];
                    } else {
                        x = __ldg(vis + vi[sl]);
                        wt = weight ? __ldg(weight + vi[sl]) : 1.0f;
                    }
                    lx = rec_lx(r[sl]);
                    ly = rec_ly(r[sl]);
                    cjm = rec_conj(r[sl]) ? 0x80008000u : 0u;
                    const int64_t row = (int64_t)rec_plane(r[sl]) * p.OS;
                    const uint4 *pv = vtab + (row + rec_ov(r[sl])) * (4 * H);
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        ldg32(pv + 4 * h, vq[h][0], vq[h][1]);
                        ldg32(pv + 4 * h + 2, vq[h][2], vq[h][3]);
                    }
                    constexpr int kU = C::U16 ? 4 : 8;  // uint4 per u row
                    const uint4 *pu = reinterpret_cast<const uint4 *>(utab) + (row + rec_ou(r[sl])) * kU;
#pragma unroll
                    for (int k = 0; k < kU; k += 2)
                        ldg32(pu + k, uq[k], uq[k + 1]);
                }
                if (sl == 0) {
                    // the pair's next stage: its records and indices now
                    okn = cursor_seek<SV>(cn, tn, items, n_items);
                    if (okn)
                        fetch(cn, tn, rn, vin, xn, wn);
                }
                if (sl == 0 && t >= kBufs) {
                    // buffer b held stage t - kBufs: wait (lane 0) for its MMAs
                    if (lane == 0 && !s_abort &&
                        !mbar_wait(empty + b / kGroup, ((t / kBufs) - 1) & 1, ctl.wait_ns))
                        s_abort = 1;
                    __syncwarp();
                    tc_fence_after();
                }
                // byte offsets of this slot's K row in A and B (chunk row 0)
                const uint32_t a_off = (i >> 3) * C::kLboA + (i & 7) * 16;
                const uint32_t b_off = (i >> 3) * C::kLboB + (i & 7) * 16;
                // A: the v words of part h, component c, shifted to the row
                // offset ly mod 8; chunk j goes to chunk row j + ly / 8 of the
                // (h, c) row block
                const int oy8 = valid ? (ly >> 3) : 8;
#pragma unroll
                for (int h = 0; h < H; ++h) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const uint32_t in[8] = {vq[h][2 * c].x,     vq[h][2 * c].y,
                                                vq[h][2 * c].z,     vq[h][2 * c].w,
                                                vq[h][2 * c + 1].x, vq[h][2 * c + 1].y,
                                                vq[h][2 * c + 1].z, vq[h][2 * c + 1].w};
                        uint32_t o[12];
                        shift16(in, ly & 7, o);
                        const uint32_t m = c ? cjm : 0u;  // conj(a) for w < 0
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            const int xq = j + oy8;
                            if (xq < 4)
                                st16(A + a_off + (h * 8 + 4 * c + xq) * kSboA,
                                     make_uint4(o[4 * j] ^ m, o[4 * j + 1] ^ m, o[4 * j + 2] ^ m,
                                                o[4 * j + 3] ^ m));
                        }
#pragma unroll
                        for (int xq = 0; xq < 4; ++xq)
                            if (xq < oy8 || xq > oy8 + 2)
                                st16(A + a_off + (h * 8 + 4 * c + xq) * kSboA, z);
                    }
                }
                // B: W V times the u-taps (FP32), each split part g rounded and
                // packed in pairs, shifted to the column offset lx mod 8; chunk j
                // to chunk row j + lx / 8 of the (g, re) and (g, im) blocks
                const int ox8 = valid ? (lx >> 3) : 8;
                const float wr = (wt * x.x) * scale;  // exact power-of-two scaling
                const float wi = (wt * x.y) * scale;
                const float wis = cjm ? -wi : wi;      // conj(u-taps) for w < 0
                const float wrs = cjm ? -wr : wr;
                float re[16], im[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    float2 u;
                    if constexpr (C::U16) {
                        const uint4 q = uq[e >> 2];
                        u = unpack_part<C::BF>((e & 3) == 0 ? q.x : (e & 3) == 1 ? q.y
                                                     : (e & 3) == 2 ? q.z : q.w);
                    } else {
                        const uint4 q = uq[e >> 1];
                        u = (e & 1) ? make_float2(__uint_as_float(q.z), __uint_as_float(q.w))
                                    : make_float2(__uint_as_float(q.x), __uint_as_float(q.y));
                    }
                    // (wr + i wi)(tr + i s ti), s = -1 for w < 0
                    re[e] = wr * u.x - wis * u.y;
                    im[e] = wrs * u.y + wi * u.x;
                }
#pragma unroll
                for (int g = 0; g < H; ++g) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const float *v = c ? im : re;
                        uint32_t pk[8], o[12];
#pragma unroll
                        for (int w = 0; w < 8; ++w)
                            pk[w] = pack_part<C::BF>(v[2 * w], v[2 * w + 1], g);
                        shift16(pk, lx & 7, o);
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            const int xq = j + ox8;
                            if (xq < 4)
                                st16(B + b_off + (g * 8 + 4 * c + xq) * C::kSboB,
                                     make_uint4(o[4 * j], o[4 * j + 1], o[4 * j + 2], o[4 * j + 3]));
                        }
#pragma unroll
                        for (int xq = 0; xq < 4; ++xq)
                            if (xq < ox8 || xq > ox8 + 2)
                                st16(B + b_off + (g * 8 + 4 * c + xq) * C::kSboB, z);
                    }
                }
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(full + b);
            cur = cn;
            t = tn;
            ok = okn;
#pragma unroll
            for (int sl = 0; sl < C::SLOTS; ++sl) {
                r[sl] = rn[sl];
                vi[sl] = vin[sl];
                xv[sl] = xn[sl];
                wv[sl] = wn[sl];
            }
        }
    } else if (warp == C::kMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            // The issue loop is one thread's dependent chain per stage, so it
            // is kept short: descriptors of buffer 0 computed once, a buffer
            // and a K step are integer offsets of the start-address field
            // (shared addresses stay below 2^18, so the 14-bit field never
            // carries), the K steps are unrolled, and a partner that stopped
            // is noticed through the bounded wait itself.
            constexpr uint32_t idesc = C::TF32 ? instr_desc(2u, false, false, C::M, N)
                                               : instr_desc(C::BF ? 1u : 0u, true, true, C::M, N);
            const uint64_t da0 = smem_desc(smem_u32(Abuf), C::kLboA, kSboA);
            const uint64_t db0 = smem_desc(smem_u32(Bbuf), C::kLboB, C::kSboB);
            constexpr uint64_t kStepA = (2 * C::kLboA) >> 4, kStepB = (2 * C::kLboB) >> 4;
            constexpr uint64_t kBufA = C::kABytes >> 4, kBufB = C::kBBytes >> 4;
            Cursor cur;
            int ne = 0;  // non-empty items so far (accumulator ne & 1)
            bool ok = true;
            while (ok && cursor_next<SV>(cur, items, n_items)) {
                if (cur.nst == 0)
                    continue;
                const int ab = ne & 1;
                if (ne >= 2 && !mbar_wait(accfree + ab, ((ne >> 1) - 1) & 1, ctl.wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(ab * N);
                int t = cur.tb;
                int left = cur.count;
                for (int st = 0; st < cur.nst; ++st, ++t, left -= SV) {
                    const int b = t & (kBufs - 1);
                    if (!mbar_wait(full + b, (t / kBufs) & 1, ctl.wait_ns)) {
                        ok = false;
                        break;
                    }
                    if (ctl.stall)
                        continue;  // test hook: issue and signal nothing
                    tc_fence_after();
                    // K steps in use (16 visibilities each, 4 for TF32)
                    const int nk = (min(SV, left) + C::VPK - 1) / C::VPK;
                    const uint64_t da = da0 + kBufA * b, db = db0 + kBufB * b;
#pragma unroll
                    for (int kq = 0; kq < SV / C::VPK; ++kq)
                        if (kq < nk) {
                            if constexpr (C::TF32)
                                mma_tf32(d, da + kStepA * kq, db + kStepB * kq, idesc,
                                         (st > 0 || kq > 0) ? 1u : 0u);
                            else
                                mma_f16(d, da + kStepA * kq, db + kStepB * kq, idesc,
                                        (st > 0 || kq > 0) ? 1u : 0u);
                        }
                    // release the group once its last buffer is issued (a group
                    // cut short by the end of the CTA's stages has no later
                    // user, and the item's "accf" commit covers its MMAs)
                    if ((b % kGroup) == kGroup - 1)
                        mma_commit(empty + b / kGroup);
                }
                if (!ok)
                    break;
                if (!ctl.stall)
                    mma_commit(accf + ab);
                ++ne;
            }
            if (!ok) {
                s_abort = 1;
                // bounded wait for every MMA this thread issued before the
                // tensor memory is released
                mma_commit(drain);
                mbar_wait(drain, 0, ctl.wait_ns);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int qq = warp & 3;  // tensor-memory lane quarter of this warp
        const int ew = warp - C::kEpiWarp0;
        const int et = tid - 32 * C::kEpiWarp0;  // 0 .. 127
        // accumulator row held by this lane: M = 128, row 32 qq + lane; M = 64,
        // row 16 qq + lane for lanes below 16 (the other lanes hold nothing)
        const bool holds = C::M == 128 || lane < 16;
        float *const row =
            stg + (C::M == 128 ? 32 * qq + lane : 16 * qq + (lane & 15)) * C::kStgStride;
        constexpr int NC = 64;  // staged columns (d, x)
        Cursor cur;
        int ne = 0;
        while (cursor_next<SV>(cur, items, n_items)) {
            if (cur.nst == 0)
                continue;
            const int ab = ne & 1;
            // every epilogue warp takes the same decision: wait, publish, agree
            int okw = 0;
            if (lane == 0)
                okw = !s_abort && mbar_wait(accf + ab, (ne >> 1) & 1, ctl.wait_ns);
            okw = __shfl_sync(0xffffffffu, okw, 0);
            if (lane == 0)
                s_epi_ok[ew] = okw;
            asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");
            const bool go = s_epi_ok[0] && s_epi_ok[1] && s_epi_ok[2] && s_epi_ok[3];
            asm volatile("bar.sync 2, %0;" ::"n"(32 * kEpiWarps) : "memory");
            if (!go) {
                if (lane == 0)
                    s_abort = 1;
                break;
            }
            tc_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(32 * qq) << 16) + (uint32_t)(ab * N);
            // this row's columns (d, x), summed over the split part g of b'
            float v[NC];
#pragma unroll
            for (int d = 0; d < NC / 32; ++d) {
                uint32_t rr[32];
                SEPW_TMEM_LD32(ta + 32 * d, rr);
                tmem_wait_ld();
#pragma unroll
                for (int xx = 0; xx < 32; ++xx)
                    v[32 * d + xx] = __uint_as_float(rr[xx]);
                if constexpr (H == 2) {
                    SEPW_TMEM_LD32(ta + 64 + 32 * d, rr);  // the b'_lo columns
                    tmem_wait_ld();
#pragma unroll
                    for (int xx = 0; xx < 32; ++xx)
                        v[32 * d + xx] += __uint_as_float(rr[xx]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(accfree + ab);
            float back = 1.0f;
            if constexpr (C::SCALED)
                back = ldexpf(1.0f, __ldg(item_exp + cur.item));
            if (holds) {
#pragma unroll
                for (int xx = 0; xx < NC; ++xx)
                    row[xx] = v[xx] * back;
            }
            asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");
            const int W = p.T + p.S - 1;
            const TileOrigin o = tile_origin(p, cur.tile);
            for (int e = et; e < kWin * kWin; e += 32 * kEpiWarps) {
                const int y = e >> 5, xx = e & 31;
                if (y >= W || xx >= W)
                    continue;
                // rows (h, c, y), columns (d, x): Re = rr - ii, Im = ri + ir
                float re = 0.f, im = 0.f;
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    const float *r0 = stg + (64 * h + y) * C::kStgStride;
                    const float *r1 = r0 + 32 * C::kStgStride;
                    re += r0[xx] - r1[32 + xx];
                    im += r0[32 + xx] + r1[xx];
                }
                if (re != 0.f || im != 0.f)
                    atomicAdd(grid + o.base + (o.gy0 + y) * p.N + o.gx0 + xx, make_float2(re, im));
            }
            asm volatile("bar.sync 2, %0;" ::"n"(32 * kEpiWarps) : "memory");
            ++ne;
        }
    }

    __syncthreads();
    if (s_abort && tid == 0)
        atomicExch(status, SEPW_ETIMEOUT);
    tc_fence_after();
    if (warp == 0)
        tmem_dealloc(tmem, C::kTmemCols);
}

template <int PREC>
cudaError_t launch_prec(const DevParams &p, const Plan &plan, const float2 *vis,
                        const float *weight, const float2 *taps, void *tables, float2 *grid,
                        int num_sms, int32_t *status, TcControl ctl, cudaStream_t s)
{
    using C = Cfg<PREC>;
    const int64_t nrow = (int64_t)p.P * p.OS;
    constexpr int KV = C::TF32 ? 8 : 4 * C::H, KU = C::U16 ? 4 : 8;  // uint4 per row
    uint4 *vtab = reinterpret_cast<uint4 *>(tables);
    uint4 *utab = vtab + nrow * KV;
    int32_t *item_exp = reinterpret_cast<int32_t *>(utab + nrow * KU);
    cudaError_t e;
    {
        const int64_t n = nrow * (KV + KU);
        const int nb = (int)std::min<int64_t>((n + 255) / 256, 4096);
        tables_kernel<PREC><<<nb, 256, 0, s>>>(p, taps, vtab, utab);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
    }
    if constexpr (C::SCALED) {
        item_scale_kernel<<<std::max(1, std::min(plan.items_capacity, 8 * num_sms)), 256, 0, s>>>(
            plan.d_items, plan.d_nitems, plan.d_perm, vis, weight, item_exp);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
    }
    e = cudaFuncSetAttribute(grid_tc2_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)C::kSmem);
    if (e != cudaSuccess)
        return e;
    grid_tc2_kernel<PREC><<<num_sms, C::kBlock, C::kSmem, s>>>(
        p, plan.d_items, plan.d_nitems, plan.d_rec, plan.d_perm, vis, weight, vtab, utab, taps,
        item_exp, grid, status, ctl);
    return cudaGetLastError();
}

}  // namespace

int tc2_tile_for_support(int S)
{
    return (kWin - S + 1) & ~1;
}

size_t tc2_tables_bytes(const DevParams &p, int64_t items_capacity)
{
    // v and u rows sized for the hi + lo forms (8 + 8 uint4 per (plane,
    // oversample)), then one exponent per work item
    return (size_t)p.P * p.OS * (8 + 8) * 16 +
           sizeof(int32_t) * (size_t)std::max<int64_t>(items_capacity, 1);
}

cudaError_t launch_grid_tc2(const DevParams &p, const Plan &plan, const float2 *vis,
                            const float *weight, const float2 *taps, void *tables, float2 *grid,
                            int num_sms, int prec, int32_t *status, TcControl ctl,
                            cudaStream_t s)
{
    if (p.T + p.S - 1 > kWin || p.S > 16)
        return cudaErrorInvalidValue;
    switch (prec) {
    case 0: return launch_prec<0>(p, plan, vis, weight, taps, tables, grid, num_sms, status, ctl, s);
    case 1: return launch_prec<1>(p, plan, vis, weight, taps, tables, grid, num_sms, status, ctl, s);
    case 2: return launch_prec<2>(p, plan, vis, weight, taps, tables, grid, num_sms, status, ctl, s);
    case 3: return launch_prec<3>(p, plan, vis, weight, taps, tables, grid, num_sms, status, ctl, s);
    case 4: return launch_prec<4>(p, plan, vis, weight, taps, tables, grid, num_sms, status, ctl, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace sepw
