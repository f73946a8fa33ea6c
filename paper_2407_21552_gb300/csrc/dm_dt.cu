// dm_dt.cu -- batched Chebyshev distance transform on the block grid, clamped to uint8.
//
// §3.1: each PDM holds the Chebyshev distance (block units) from a block to the nearest
// occupied block of its POM; §3.2: stored as uint8 with larger distances clamped.  The
// chessboard distance separates over the axes:
//     D(x,y,z) = min_z' max(|z-z'|, min_y' max(|y-y'|, min_x' {|x-x'| : occupied})),
// so the transform is one x pass (1D distance to the nearest occupied block of the line)
// and two passes of the 1D max-min transform h(i) = min_j max(|i-j|, g(j)).  Clamping
// commutes with every min and max here, so saturating uint8 arithmetic stays exact.
//
// x pass: a row's occupancy becomes one bit line per partition in shared memory (the
// K-map pass transposes each warp's 32 blocks x 32 partitions bit matrix with shuffles;
// the one-map pass takes one ballot per 32 blocks); for every 32-bit word the nearest set
// bit left of it and right of it are precomputed.  The K-map pass gives each thread 16
// consecutive blocks of one bit line: their left and right neighbours' nearest bits come
// from the rest of the word or those tables, two 16-step scans give the 16 distances, and
// one 16-byte store writes them.  Short rows share a CTA; rows of at most 96 blocks (with
// at most 64 maps) take one warp each instead, their bit lines built by ballots in
// registers.  The one-map pass (full recompute) takes one masked clz/ffs plus the two
// lookups per output, four outputs per 32-bit store.
//
// y / z passes: one thread per line, a CTA per tile of kLineTile neighbouring lines (along
// x) staged whole in shared memory.  The transform splits into the sweeps
// F(i) = min over j <= i of max(i - j, g(j)) and, run backwards over F, h itself (the
// backward sweep of F takes the j > i terms; j <= i ones are already folded into F).  A
// sweep keeps its level v = F(i - 1) and T, the last position j with g(j) <= v.  A new
// value g(i) <= v starts a new level at i; otherwise the level holds while a source of
// value v lies within distance v (i - T <= v), and else rises by one: F(i) is then v + 1
// and T the last position whose value is exactly v + 1, read from a per-line table of the
// last position of every value (0..255) that the sweep fills as it goes.  Each output
// costs O(1) work whatever the distances are.  Clamping at 255 needs no extra step: a
// value of 255 is a source of level 255 that never expires.
#include <algorithm>

#include "dm_build_batch.cuh"
#include "dm_internal.cuh"

namespace dmk {
namespace {

constexpr int kThreads = 256;
constexpr int kNone = -30000;          // "no set bit" sentinels for the nearest-bit tables
constexpr int kFar = 30000;

// ------------------------------------------------------------------------------ x pass
struct XGeom {
    int gx, rows;
    int nw;             // 32-bit words per bit line
    int64_t plane;
    int vec4;           // rows are 4-byte aligned: store 4 outputs as one word
    int vec16;          // rows are 16-byte aligned: store 16 outputs as one vector
    int rpc;            // block rows per CTA of the K-map pass (short rows share a CTA)
    int warp_rows;      // rows of at most 96 blocks, at most 64 maps: one warp per row
    // optional (one row per CTA): proj[row][w] = the row's mask words ORed along x, the
    // occupancy of each map in the row
    uint64_t* proj;
};

struct SrcMinMax8 {     // min/max occupancy: one visible intensity in [min, max]
    const uint16_t* mm;
    const int32_t* cnt;
};
struct SrcMinMax16 {
    const uint32_t* mm;
    const int32_t* cnt;
};
struct SrcOcc {         // occupancy bytes (0/1)
    const uint8_t* occ;
};

// Nearest set bit around x in a bit line: own word by clz/ffs, else the precomputed
// nearest set bit left (prev) / right (next) of the word; saturates at 255.
__device__ __forceinline__ unsigned nearest_bit(const uint32_t* __restrict__ bits,
                                                const int16_t* __restrict__ prev,
                                                const int16_t* __restrict__ next, int x)
{
    const int wi = x >> 5, bi = x & 31;
    const uint32_t cur = bits[wi];
    const uint32_t ml = cur & (0xFFFFFFFFu >> (31 - bi));   // bits 0..bi
    const uint32_t mr = cur & (0xFFFFFFFFu << bi);          // bits bi..31
    const int l = ml ? (wi * 32 + 31 - __clz(ml)) : int(prev[wi]);
    const int r = mr ? (wi * 32 + __ffs(mr) - 1) : int(next[wi]);
    const int d = min(x - l, r - x);
    return unsigned(d > 255 ? 255 : d);
}

// prev[w] / next[w]: nearest set bit strictly left / right of word w of a bit line.
__device__ __forceinline__ void nearest_tables(const uint32_t* bits, int nw, int16_t* prev,
                                               int16_t* next)
{
    int last = kNone;
    for (int w = 0; w < nw; ++w) {
        prev[w] = int16_t(last);
        const uint32_t b = bits[w];
        if (b) last = w * 32 + 31 - __clz(b);
    }
    int first = kFar;
    for (int w = nw - 1; w >= 0; --w) {
        next[w] = int16_t(first);
        const uint32_t b = bits[w];
        if (b) first = w * 32 + __ffs(b) - 1;
    }
}

// 32x32 bit-matrix transpose across a warp: lane i holds row i (bit j = element (i, j))
// and ends holding column i (bit j = element (j, i)).  Each stage swaps the off-diagonal
// s x s blocks of every 2s x 2s block with the partner lane i ^ s.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t r, int lane)
{
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int s = 16 >> k;
        const uint32_t m = masks[k];
        const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, r, s);
        r = (lane & s) ? ((r & ~m) | ((o & ~m) >> s)) : ((r & m) | ((o & m) << s));
    }
    return r;
}

// 16 outputs of a bit line: blocks xb = 32 wi + 16 half .. xb + 15 of the row at `row`.
// The nearest set bit left and right of the 16 blocks comes from the rest of their word or
// the prev / next tables, then two 16-step scans give every distance, stored as one
// 16-byte vector where the row allows.
__device__ __forceinline__ void emit16(const uint32_t* __restrict__ bits,
                                       const int16_t* __restrict__ prev,
                                       const int16_t* __restrict__ next, int wi, int half,
                                       const XGeom& xg, uint8_t* __restrict__ row)
{
    const int xb = wi * 32 + half * 16;                      // first block of the item
    const uint32_t b = bits[wi];
    const unsigned below = half ? (b & 0xFFFFu) : 0u;        // bits left of the 16 blocks
    const unsigned above = half ? 0u : (b >> 16);            // bits right of them
    int last = below ? (wi * 32 + 31 - __clz(below)) : int(prev[wi]);
    int nxt = above ? (wi * 32 + 16 + __ffs(above) - 1) : int(next[wi]);
    const unsigned hb = (b >> (16 * half)) & 0xFFFFu;
    int dl[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        if ((hb >> i) & 1u) last = xb + i;
        dl[i] = xb + i - last;
    }
    unsigned pk[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int i = 15; i >= 0; --i) {
        if ((hb >> i) & 1u) nxt = xb + i;
        const int d = min(min(dl[i], nxt - (xb + i)), 255);
        pk[i >> 2] |= unsigned(d) << (8 * (i & 3));
    }
    uint8_t* dst = row + xb;
    if (xg.vec16 && xb + 16 <= xg.gx) {
        *reinterpret_cast<uint4*>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    } else if (xg.vec4 && xb + 16 <= xg.gx) {
#pragma unroll
        for (int k = 0; k < 4; ++k) reinterpret_cast<uint32_t*>(dst)[k] = pk[k];
    } else {
        for (int i = 0; i < 16 && xb + i < xg.gx; ++i)
            dst[i] = uint8_t(pk[i >> 2] >> (8 * (i & 3)));
    }
}

// K planes from the POM masks; one CTA per block row, 64 partitions (one mask word) at a
// time.  Shared memory: bits [cap][nw] uint32, prev / next [cap][nw] int16, cap = min(64, K).
// Outputs: one thread per (partition, 16 consecutive blocks); the nearest set bit left and
// right of its 16 blocks comes from the rest of the word or the prev / next tables, then
// two 16-step scans give every distance, stored as one 16-byte vector.
template <int W>
__device__ __forceinline__ void xpass_mask_row(const uint64_t* __restrict__ mask, int K,
                                               const XGeom& xg, uint8_t* __restrict__ out,
                                               int row)
{
    extern __shared__ uint32_t s_mem[];
    const int nw = xg.nw;
    const int cap = min(64, K);                              // partitions per chunk
    uint32_t* s_bits = s_mem;
    int16_t* s_prev = reinterpret_cast<int16_t*>(s_mem + cap * nw);
    int16_t* s_next = s_prev + cap * nw;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ uint64_t s_por[kThreads / 32];                // the row's OR, per warp
    const int64_t rbase = int64_t(row) * xg.gx;
    const int nh = 2 * nw;                                   // 16-block items per bit line
#pragma unroll 1
    for (int w = 0; w < W; ++w) {
        const int np = min(64, K - w * 64);
        if (w) __syncthreads();                              // previous chunk consumed
        uint64_t por = 0;                                    // this thread's mask words ORed
        for (int x0 = 0; x0 < xg.gx; x0 += kThreads) {
            if (x0 + warp * 32 >= xg.gx) continue;           // warp-uniform: no blocks here
            const int x = x0 + tid;
            const uint64_t m = x < xg.gx ? mask[(rbase + x) * W + w] : 0;
            por |= m;
            const int wi = (x0 >> 5) + warp;
            // bit lines of 32 blocks: lane q receives partition q's word (and 32 + q's)
            const uint32_t lo = warp_transpose32(uint32_t(m), lane);
            if (lane < np) s_bits[lane * nw + wi] = lo;
            if (np > 32) {                                   // warp-uniform
                const uint32_t hi = warp_transpose32(uint32_t(m >> 32), lane);
                if (lane + 32 < np) s_bits[(lane + 32) * nw + wi] = hi;
            }
        }
        if (xg.proj) {                                       // uniform
            const unsigned lo = __reduce_or_sync(0xFFFFFFFFu, unsigned(por));
            const unsigned hi = __reduce_or_sync(0xFFFFFFFFu, unsigned(por >> 32));
            if (lane == 0) s_por[warp] = (uint64_t(hi) << 32) | lo;
        }
        __syncthreads();
        if (xg.proj && tid == 0) {
            uint64_t all = 0;
            for (int k = 0; k < kThreads / 32; ++k) all |= s_por[k];
            xg.proj[int64_t(row) * W + w] = all;
        }
        for (int q = tid; q < np; q += kThreads)
            nearest_tables(s_bits + q * nw, nw, s_prev + q * nw, s_next + q * nw);
        __syncthreads();
        for (int it = tid; it < np * nh; it += kThreads) {
            const int q = it / nh, hw = it - q * nh;
            const int wi = hw >> 1, half = hw & 1;
            if (wi * 32 + half * 16 >= xg.gx) continue;
            emit16(s_bits + q * nw, s_prev + q * nw, s_next + q * nw, wi, half, xg,
                   out + int64_t(w * 64 + q) * xg.plane + rbase);
        }
    }
}

// The same for rows of at most a few words: xg.rpc consecutive block rows per CTA (rows
// row0 .. row0 + rpc - 1), so that short rows still give every warp a word of blocks and
// every thread an item.  Shared memory: bits [rpc][cap][nw], prev / next likewise.
template <int W>
__device__ __forceinline__ void xpass_mask_rows(const uint64_t* __restrict__ mask, int K,
                                                const XGeom& xg, uint8_t* __restrict__ out,
                                                int row0)
{
    extern __shared__ uint32_t s_mem[];
    const int nw = xg.nw;
    const int cap = min(64, K);
    const int nrow = min(xg.rpc, xg.rows - row0);            // rows of this CTA
    const int line = cap * nw;                               // words of one row's lines
    uint32_t* s_bits = s_mem;
    int16_t* s_prev = reinterpret_cast<int16_t*>(s_mem + xg.rpc * line);
    int16_t* s_next = s_prev + xg.rpc * line;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nh = 2 * nw;
#pragma unroll 1
    for (int w = 0; w < W; ++w) {
        const int np = min(64, K - w * 64);
        if (w) __syncthreads();                              // previous chunk consumed
        for (int t = warp; t < nrow * nw; t += kThreads / 32) {   // warp-uniform
            const int r = t / nw, wi = t - r * nw;
            const int x = wi * 32 + lane;
            const int64_t rbase = int64_t(row0 + r) * xg.gx;
            const uint64_t m = x < xg.gx ? mask[(rbase + x) * W + w] : 0;
            uint32_t* bits = s_bits + r * line;
            const uint32_t lo = warp_transpose32(uint32_t(m), lane);
            if (lane < np) bits[lane * nw + wi] = lo;
            if (np > 32) {                                   // warp-uniform
                const uint32_t hi = warp_transpose32(uint32_t(m >> 32), lane);
                if (lane + 32 < np) bits[(lane + 32) * nw + wi] = hi;
            }
        }
        __syncthreads();
        for (int q = tid; q < nrow * np; q += kThreads) {
            const int r = q / np;
            const int o = r * line + (q - r * np) * nw;
            nearest_tables(s_bits + o, nw, s_prev + o, s_next + o);
        }
        __syncthreads();
        const int per_row = np * nh;
        for (int it = tid; it < nrow * per_row; it += kThreads) {
            const int r = it / per_row, rem = it - r * per_row;
            const int q = rem / nh, hw = rem - q * nh;
            const int wi = hw >> 1, half = hw & 1;
            if (wi * 32 + half * 16 >= xg.gx) continue;
            const int o = r * line + q * nw;
            emit16(s_bits + o, s_prev + o, s_next + o, wi, half, xg,
                   out + int64_t(w * 64 + q) * xg.plane + int64_t(row0 + r) * xg.gx);
        }
    }
}

// Rows of at most 32 NW blocks (NW <= 3) and at most 64 maps: one warp per block row, no
// shared memory and no barrier.  Lane l holds the mask words of blocks l, 32 + l, ...; for
// each map one ballot per word gives the row's bit line, and each lane takes the nearest
// set bit left and right of each of its blocks from its own word or, beyond it, from the
// nearest set bits of the other words (the same for the whole warp).
template <int NW>
__device__ __forceinline__ void xpass_warp_row(const uint64_t* __restrict__ mask, int K,
                                               const XGeom& xg, uint8_t* __restrict__ out,
                                               int row, int lane)
{
    const int64_t rbase = int64_t(row) * xg.gx;
    uint64_t m[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int x = 32 * w + lane;
        m[w] = x < xg.gx ? mask[rbase + x] : 0ull;
    }
    const unsigned lomask = 0xFFFFFFFFu >> (31 - lane);     // bits 0..lane
    const unsigned himask = 0xFFFFFFFFu << lane;            // bits lane..31
    uint8_t* plane = out + rbase;
    for (int p = 0; p < K; ++p, plane += xg.plane) {
        unsigned b[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) b[w] = __ballot_sync(0xFFFFFFFFu, unsigned(m[w] >> p) & 1u);
        int lft[NW], rgt[NW];                              // nearest set bit beyond word w
        int last = kNone;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            lft[w] = last;
            if (b[w]) last = 32 * w + 31 - __clz(b[w]);
        }
        int first = kFar;
#pragma unroll
        for (int w = NW - 1; w >= 0; --w) {
            rgt[w] = first;
            if (b[w]) first = 32 * w + __ffs(b[w]) - 1;
        }
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int x = 32 * w + lane;
            if (x >= xg.gx) continue;
            const unsigned lo = b[w] & lomask, hi = b[w] & himask;
            const int l = lo ? 32 * w + 31 - __clz(lo) : lft[w];
            const int r = hi ? 32 * w + __ffs(hi) - 1 : rgt[w];
            plane[x] = uint8_t(min(min(x - l, r - x), 255));
        }
    }
}

template <int NW>
__global__ void __launch_bounds__(kThreads)
k_xpass_warp_rows(const uint64_t* __restrict__ mask, int K, XGeom xg, uint8_t* __restrict__ out)
{
    pdl_wait();
    const int row = int(blockIdx.x) * (kThreads / 32) + int(threadIdx.x >> 5);
    if (row >= xg.rows) return;                             // warp-uniform; no barrier
    xpass_warp_row<NW>(mask, K, xg, out, row, int(threadIdx.x & 31));
}

template <int W>
__global__ void __launch_bounds__(kThreads)
k_xpass_mask(const uint64_t* __restrict__ mask, int K, XGeom xg, uint8_t* __restrict__ out)
{
    pdl_wait();
    xpass_mask_row<W>(mask, K, xg, out, blockIdx.x);         // row = z * gy + y
}

template <int W>
__global__ void __launch_bounds__(kThreads)
k_xpass_mask_packed(const uint64_t* __restrict__ mask, int K, XGeom xg, uint8_t* __restrict__ out)
{
    pdl_wait();
    xpass_mask_rows<W>(mask, K, xg, out, int(blockIdx.x) * xg.rpc);
}

// Several volumes' x passes in one grid: one CTA per xg.rpc block rows, volume after
// volume.
struct XBatch {
    int n;
    int start[kMaxBuildBatch + 1];             // first row (CTA) of each volume
    const uint64_t* mask[kMaxBuildBatch];
    uint8_t* out[kMaxBuildBatch];
    int K[kMaxBuildBatch];
    XGeom xg[kMaxBuildBatch];
};

template <int W>
__global__ void __launch_bounds__(kThreads)
k_xpass_mask_batch(const __grid_constant__ XBatch B)
{
    const int i = batch_item_of(B.start, B.n, int(blockIdx.x));
    const XGeom& xg = B.xg[i];
    pdl_wait();
    if (W == 1 && xg.warp_rows) {                           // one warp per row, 8 rows per CTA
        const int row = (int(blockIdx.x) - B.start[i]) * (kThreads / 32) + int(threadIdx.x >> 5);
        if (row >= xg.rows) return;                         // warp-uniform; no barrier
        const int lane = int(threadIdx.x & 31);
        if (xg.nw == 1) xpass_warp_row<1>(B.mask[i], B.K[i], xg, B.out[i], row, lane);
        else if (xg.nw == 2) xpass_warp_row<2>(B.mask[i], B.K[i], xg, B.out[i], row, lane);
        else xpass_warp_row<3>(B.mask[i], B.K[i], xg, B.out[i], row, lane);
        return;
    }
    if (xg.rpc > 1)
        xpass_mask_rows<W>(B.mask[i], B.K[i], xg, B.out[i], (int(blockIdx.x) - B.start[i]) * xg.rpc);
    else
        xpass_mask_row<W>(B.mask[i], B.K[i], xg, B.out[i], int(blockIdx.x) - B.start[i]);
}

template <typename Src>
__device__ __forceinline__ bool occ_of(const Src& s, int64_t blk);

template <>
__device__ __forceinline__ bool occ_of<SrcMinMax8>(const SrcMinMax8& s, int64_t blk)
{
    const uint32_t v = s.mm[blk];
    const uint32_t mn = v & 0xFF, mx = v >> 8;
    return __ldg(s.cnt + mx + 1) > __ldg(s.cnt + mn);
}
template <>
__device__ __forceinline__ bool occ_of<SrcMinMax16>(const SrcMinMax16& s, int64_t blk)
{
    const uint32_t v = s.mm[blk];
    const uint32_t mn = v & 0xFFFF, mx = v >> 16;
    return __ldg(s.cnt + mx + 1) > __ldg(s.cnt + mn);
}
template <>
__device__ __forceinline__ bool occ_of<SrcOcc>(const SrcOcc& s, int64_t blk)
{
    return s.occ[blk] != 0;
}

// Single-map x pass (full recompute): one warp per block row, 8 rows per CTA.  A warp
// reads its whole row's occupancy before writing it, so `out` may alias the source.
template <typename Src>
__global__ void __launch_bounds__(kThreads)
k_xpass_single(Src src, XGeom xg, uint8_t* out)
{
    extern __shared__ uint32_t s_mem[];                      // per warp: bits, prev, next
    pdl_wait();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = xg.nw;
    const int per_warp = nw * 2;                             // words: bits + 2 x int16
    uint32_t* bits = s_mem + warp * per_warp;
    int16_t* prev = reinterpret_cast<int16_t*>(bits + nw);
    int16_t* next = prev + nw;                               // nw int16 + nw int16 = nw words
    const int row = blockIdx.x * (kThreads / 32) + warp;
    if (row >= xg.rows) return;                              // warp-uniform
    const int64_t rbase = int64_t(row) * xg.gx;
    for (int x0 = 0; x0 < xg.gx; x0 += 32) {
        const int x = x0 + lane;
        const bool o = x < xg.gx ? occ_of(src, rbase + x) : false;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, o);
        if (lane == 0) bits[x0 >> 5] = bal;
    }
    __syncwarp();
    if (lane == 0) nearest_tables(bits, nw, prev, next);
    __syncwarp();
    uint8_t* dst = out + rbase;
    for (int x = lane * 4; x < xg.gx; x += 128) {
        if (xg.vec4 && x + 3 < xg.gx) {
            unsigned v = nearest_bit(bits, prev, next, x) |
                         (nearest_bit(bits, prev, next, x + 1) << 8) |
                         (nearest_bit(bits, prev, next, x + 2) << 16) |
                         (nearest_bit(bits, prev, next, x + 3) << 24);
            *reinterpret_cast<uint32_t*>(dst + x) = v;
        } else {
            for (int k = 0; k < 4 && x + k < xg.gx; ++k)
                dst[x + k] = uint8_t(nearest_bit(bits, prev, next, x + k));
        }
    }
}

XGeom xgeom(const Geometry& g, int64_t plane, const void* out)
{
    XGeom x;
    x.gx = g.gx;
    x.rows = g.gy * g.gz;
    x.nw = (g.gx + 31) / 32;
    x.plane = plane;
    x.vec4 = (g.gx % 4 == 0) && (plane % 4 == 0) &&
             ((reinterpret_cast<uintptr_t>(out) & 3) == 0);
    x.vec16 = (g.gx % 16 == 0) && (plane % 16 == 0) &&
              ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
    x.rpc = 1;
    x.warp_rows = 0;
    x.proj = nullptr;
    return x;
}

// The one-warp-per-row x pass takes rows of at most 3 words and at most 64 maps.
static bool xpass_warp_rows_ok(int nw, int K) { return nw <= 3 && K <= 64; }

// Block rows per CTA of the K-map x pass: enough rows that a chunk of up to 64 maps gives
// about one 16-block item per thread (at most 8 rows).
static int xpass_rows_per_cta(int nw, int K)
{
    const int per_row = (K < 64 ? K : 64) * 2 * nw;
    const int r = kThreads / per_row;
    return r < 1 ? 1 : (r > 8 ? 8 : r);
}

// ------------------------------------------------------------------------ y / z passes
struct LineGeom {
    int L;              // line length (blocks)
    int gx;             // columns along x (contiguous)
    int n_outer;        // lines per plane per x column
    int64_t s;          // element stride along the line
    int64_t os;         // stride of the outer index
    int64_t plane;      // stride between planes
    int vec_ok;         // rows of kLineTile columns are 16-byte aligned and full
};

// Bytes of shared memory of a tile's values [L][TC]; the table of last positions
// [257][TC] follows.
__host__ __device__ inline size_t sweep_tile_bytes(int L, int TC)
{
    return (size_t(L) * TC + 15) / 16 * 16;
}

// One sweep over a line of the tile, rows in the order FINAL gives (forward from row 0, or
// backward from row L-1).  Positions enter the table as `off` + the step count, so that a
// sweep never mistakes an entry of an earlier sweep (all below its own `off`) for one of
// its own.  TO_TILE: the values go back into the tile; otherwise to global memory (column
// `col` of the tile's rows).
//
// A step enters its own row in the table first and then reads the entry of the next level
// up, so that the read already sees the step's own value.  That read only feeds T, and T
// only decides the rise of the next step, so its latency spans two steps.  The level can
// rise by one a step at most (d = pos - T never exceeds lv + 1), so the new level is
// min(g, max(lv, d)): two min/max operations, with no select on a compare, on the chain
// from one step's level to the next.  The values of kRun rows are read before any of them
// is processed; whole runs of kRun rows carry no bound checks, the last partial run does.
constexpr int kRun = 8;

struct SweepState {
    int lv;                      // level of the previous row (255 before the first)
    int T;                       // last position holding a value <= lv
};

template <int TC, bool FINAL, bool TO_TILE, bool TAIL, typename P>
__device__ __forceinline__ void sweep_run(uint8_t* __restrict__ tile, P* __restrict__ tab,
                                          int L, int k0, int off, SweepState& st,
                                          uint8_t* __restrict__ col, int64_t gstride)
{
    const int r0 = FINAL ? L - 1 : 0;
    const int dir = FINAL ? -1 : 1;
    int gv[kRun];
#pragma unroll
    for (int i = 0; i < kRun; ++i)
        gv[i] = (!TAIL || k0 + i < L) ? tile[(r0 + dir * (k0 + i)) * TC] : 0;
    int lv = st.lv, T = st.T;
#pragma unroll
    for (int i = 0; i < kRun; ++i) {
        const int k = k0 + i;
        if (TAIL && k >= L) break;
        const int r = r0 + dir * k;
        const int g = gv[i];
        const int pos = off + k;
        tab[g * TC] = P(pos);
        const int x = tab[(lv + 1) * TC];                 // last position of level lv + 1
        const int d = pos - T;                             // at most lv + 1
        const bool drop = g <= lv;
        T = drop ? pos : (d > lv ? max(T, x) : T);         // d > lv: level lv ran out here
        lv = min(g, max(lv, d));                           // g, lv + 1 or lv
        if (TO_TILE) tile[r * TC] = uint8_t(lv);
        else col[int64_t(r) * gstride] = uint8_t(lv);
    }
    st.lv = lv;
    st.T = T;
}

template <int TC, bool FINAL, bool TO_TILE, typename P>
__device__ __forceinline__ void sweep_line(uint8_t* __restrict__ tile, P* __restrict__ tab,
                                           int L, int off, uint8_t* __restrict__ col,
                                           int64_t gstride)
{
    SweepState st{255, off};
    int k0 = 0;
    for (; k0 + kRun <= L; k0 += kRun)
        sweep_run<TC, FINAL, TO_TILE, false>(tile, tab, L, k0, off, st, col, gstride);
    if (k0 < L) sweep_run<TC, FINAL, TO_TILE, true>(tile, tab, L, k0, off, st, col, gstride);
}

// One tile = TC adjacent columns x one whole line of every column; thread c takes column c.
// The tile is staged before any output is written, so the pass works in place.  P, the
// type of the table's positions: uint8_t for lines of at most 256 blocks, else uint16_t.
// The backward sweep's positions follow the forward sweep's (L .. 2L-1), so one clearing
// serves both, except for 8-bit positions on lines of more than 128 blocks: there each
// sweep numbers its rows 0..L-1 and the table is cleared between them.
template <int TC, typename P, bool VEC>
__device__ __forceinline__ void line_sweep_tile(uint8_t* buf, const LineGeom& lg, int cx,
                                                int cy, int cz)
{
    extern __shared__ uint32_t s_mem[];
    constexpr int V = TC / 16;                               // 16-byte vectors per row
    constexpr bool kShort = sizeof(P) == 1;
    const int L = lg.L;
    uint8_t* s_tile = reinterpret_cast<uint8_t*>(s_mem);     // [L][TC]
    P* s_tab = reinterpret_cast<P*>(s_tile + sweep_tile_bytes(L, TC));   // [257][TC]
    const int tid = threadIdx.x;
    const int x0 = cx * TC;
    uint8_t* base = buf + int64_t(cz) * lg.plane + int64_t(cy) * lg.os + x0;
    const int ncols = min(TC, lg.gx - x0);

    // ---- stage the tile (asynchronous copies, all in flight at once); note whether it can
    //      change at all (some value >= 2 and not everything 255)
    int any_big = 0, any_not255 = 0;
    if (VEC) {                               // lg.vec_ok
        for (int i = tid; i < L * V; i += TC) {
            const int r = i / V, q = i - r * V;
            const unsigned sa = static_cast<unsigned>(
                __cvta_generic_to_shared(reinterpret_cast<uint4*>(s_tile) + i));
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa),
                         "l"(base + int64_t(r) * lg.s + 16 * q)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        for (int i = tid; i < L * V; i += TC) {
            const uint4 v = reinterpret_cast<const uint4*>(s_tile)[i];
            const unsigned w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                any_not255 |= (w4[k] != 0xFFFFFFFFu);
                any_big |= ((w4[k] & 0xFEFEFEFEu) != 0);     // a byte >= 2
            }
        }
    } else {                                 // thread c stages column c, 8 rows per round
        const bool col_ok = tid < ncols;
        for (int r0 = 0; r0 < L; r0 += 8) {
            unsigned v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                v[k] = col_ok && r0 + k < L ? base[int64_t(r0 + k) * lg.s + tid] : 255u;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (r0 + k >= L) break;
                s_tile[(r0 + k) * TC + tid] = uint8_t(v[k]);
                any_not255 |= v[k] != 255u;
                any_big |= col_ok && v[k] >= 2u;
            }
        }
    }
    // the table starts at position 0 everywhere: a sweep's T is >= 0 from its first row on,
    // so these entries are never taken for a source.  Entry 256 (level 255 + 1) is read but
    // never written.
    constexpr int kTabVec = 257 * TC * int(sizeof(P)) / 16;
    for (int i = tid; i < kTabVec; i += TC)
        reinterpret_cast<uint4*>(s_tab)[i] = make_uint4(0u, 0u, 0u, 0u);
    any_big = __syncthreads_or(any_big);
    any_not255 = __syncthreads_or(any_not255);
    if (!any_big || !any_not255) return;   // all values <= 1, or all 255: h == g
    if (!VEC && tid >= ncols) return;       // (whole-row tiles have every column)
    uint8_t* tile = s_tile + tid;
    P* tab = s_tab + tid;
    sweep_line<TC, false, true>(tile, tab, L, 0, nullptr, 0);
    // whole-row tiles keep the result in the tile and write it out as 16-byte rows
    const int off2 = kShort && 2 * L > 256 ? 0 : L;
    if (off2 == 0)                          // clear this column's table again
        for (int v = 0; v < 256; ++v) tab[v * TC] = P(0);
    sweep_line<TC, true, VEC>(tile, tab, L, off2, base + tid, lg.s);
    if (VEC) {
        __syncthreads();
        for (int i = tid; i < L * V; i += TC) {
            const int r = i / V, q = i - r * V;
            *reinterpret_cast<uint4*>(base + int64_t(r) * lg.s + 16 * q) =
                reinterpret_cast<const uint4*>(s_tile)[i];
        }
    }
}

template <int TC, typename P, bool VEC>
__global__ void __launch_bounds__(TC)
k_line_sweep(uint8_t* buf, LineGeom lg)
{
    pdl_wait();
    line_sweep_tile<TC, P, VEC>(buf, lg, blockIdx.x, blockIdx.y, blockIdx.z);
}


// Several volumes' y (or z) passes in one grid; each volume keeps its one-volume grid
// (tiles along x fastest, then the outer index, then the plane).
struct LineBatch {
    int n;
    int start[kMaxBuildBatch + 1];             // first CTA of each volume
    uint8_t* buf[kMaxBuildBatch];
    LineGeom lg[kMaxBuildBatch];
    int gdx[kMaxBuildBatch];                   // tiles along x
};

template <int TC, typename P, bool VEC>
__global__ void __launch_bounds__(TC)
k_line_sweep_batch(const __grid_constant__ LineBatch B)
{
    const int i = batch_item_of(B.start, B.n, int(blockIdx.x));
    const int local = int(blockIdx.x) - B.start[i];
    const int gdx = B.gdx[i], n_outer = B.lg[i].n_outer;
    const int cx = local % gdx, rest = local / gdx;
    pdl_wait();
    line_sweep_tile<TC, P, VEC>(B.buf[i], B.lg[i], cx, rest % n_outer, rest / n_outer);
}

}  // namespace

size_t line_pass_smem(int L)
{
    const size_t pos_bytes = L <= 256 ? 1 : 2;
    return sweep_tile_bytes(L, kLineTile) + size_t(257) * kLineTile * pos_bytes;
}


size_t xpass_smem(int gx, int K)
{
    const int nw = (gx + 31) / 32;
    const size_t mask_pass = size_t(xpass_rows_per_cta(nw, K)) * (K < 64 ? K : 64) * nw * 8;
    const size_t single = size_t(kThreads / 32) * nw * 8;
    return mask_pass > single ? mask_pass : single;
}

cudaError_t launch_xpass_mask(const uint64_t* mask, int K, const Geometry& g, uint8_t* pdm,
                              cudaStream_t s, uint64_t* proj, bool* projected)
{
    XGeom xg = xgeom(g, g.plane, pdm);
    if (projected) *projected = false;
    if (xpass_warp_rows_ok(xg.nw, K)) {
        xg.warp_rows = 1;
        const unsigned ctas = unsigned((xg.rows + kThreads / 32 - 1) / (kThreads / 32));
        if (xg.nw == 1)
            return launch_pdl(k_xpass_warp_rows<1>, dim3(ctas), dim3(kThreads), 0, s, mask, K, xg, pdm);
        if (xg.nw == 2)
            return launch_pdl(k_xpass_warp_rows<2>, dim3(ctas), dim3(kThreads), 0, s, mask, K, xg, pdm);
        return launch_pdl(k_xpass_warp_rows<3>, dim3(ctas), dim3(kThreads), 0, s, mask, K, xg, pdm);
    }
    xg.rpc = xpass_rows_per_cta(xg.nw, K);
    const size_t smem = size_t(xg.rpc) * (K < 64 ? K : 64) * xg.nw * 8;
    const int W = (K + 63) / 64;
    const unsigned ctas = unsigned((xg.rows + xg.rpc - 1) / xg.rpc);
    cudaError_t e = cudaSuccess;
    switch (W) {
#define DM_XPASS_CASE(WW)                                                                    \
    case WW:                                                                                 \
        if (xg.rpc > 1) {                                                                    \
            e = ensure_dynamic_smem<k_xpass_mask_packed<WW>>(int(smem));                     \
            if (e != cudaSuccess) return e;                                                  \
            return launch_pdl(k_xpass_mask_packed<WW>, dim3(ctas), dim3(kThreads), smem, s,  \
                              mask, K, xg, pdm);                                             \
        }                                                                                    \
        e = ensure_dynamic_smem<k_xpass_mask<WW>>(int(smem));                                \
        if (e != cudaSuccess) return e;                                                      \
        xg.proj = proj;                                                                      \
        if (projected) *projected = proj != nullptr;                                         \
        return launch_pdl(k_xpass_mask<WW>, dim3(xg.rows), dim3(kThreads), smem, s, mask, K, \
                          xg, pdm);
        DM_XPASS_CASE(1)
        DM_XPASS_CASE(2)
        DM_XPASS_CASE(3)
        DM_XPASS_CASE(4)
#undef DM_XPASS_CASE
    default: return cudaErrorInvalidValue;
    }
}

template <typename Src>
static cudaError_t launch_single(Src src, const Geometry& g, uint8_t* out, cudaStream_t s)
{
    XGeom xg = xgeom(g, 0, out);
    const size_t smem = size_t(kThreads / 32) * xg.nw * 8;
    cudaError_t e = ensure_dynamic_smem<k_xpass_single<Src>>(int(smem));
    if (e != cudaSuccess) return e;
    const int ctas = (xg.rows + kThreads / 32 - 1) / (kThreads / 32);
    return launch_pdl(k_xpass_single<Src>, dim3(ctas), dim3(kThreads), smem, s, src, xg, out);
}

cudaError_t launch_xpass_minmax(const void* minmax, const int32_t* cnt, const Geometry& g,
                                uint8_t* out, cudaStream_t s)
{
    if (g.bpv == 1)
        return launch_single(SrcMinMax8{static_cast<const uint16_t*>(minmax), cnt}, g, out, s);
    return launch_single(SrcMinMax16{static_cast<const uint32_t*>(minmax), cnt}, g, out, s);
}

cudaError_t launch_xpass_occ(uint8_t* occ_inout, const Geometry& g, cudaStream_t s)
{
    return launch_single(SrcOcc{occ_inout}, g, occ_inout, s);
}

static LineGeom line_geom(uint8_t* buf, int64_t plane, const Geometry& g, int axis)
{
    LineGeom lg;
    lg.gx = g.gx;
    lg.plane = plane;
    if (axis == 1) {                     // lines along y, outer index z
        lg.L = g.gy;
        lg.s = g.gx;
        lg.n_outer = g.gz;
        lg.os = int64_t(g.gx) * g.gy;
    } else {                             // lines along z, outer index y
        lg.L = g.gz;
        lg.s = int64_t(g.gx) * g.gy;
        lg.n_outer = g.gy;
        lg.os = g.gx;
    }
    lg.vec_ok = (g.gx % kLineTile == 0) && ((reinterpret_cast<uintptr_t>(buf) & 15) == 0) &&
                (plane % 16 == 0);
    return lg;
}

cudaError_t launch_line_pass(uint8_t* buf, int P, int64_t plane, const Geometry& g, int axis,
                             cudaStream_t s)
{
    const LineGeom lg = line_geom(buf, plane, g, axis);
    if (lg.L <= 1) return cudaSuccess;   // a single block per line: h == g
    constexpr int TC = kLineTile;
    const size_t smem = line_pass_smem(lg.L);
    if (smem > size_t(kLineSmemLimit)) return cudaErrorInvalidConfiguration;
    dim3 grid((g.gx + TC - 1) / TC, lg.n_outer, P);
    cudaError_t e;
#define DM_SWEEP_LAUNCH(PP, VV)                                                              \
    e = ensure_dynamic_smem<k_line_sweep<TC, PP, VV>>(int(smem));                            \
    if (e != cudaSuccess) return e;                                                          \
    return launch_pdl(k_line_sweep<TC, PP, VV>, grid, dim3(TC), smem, s, buf, lg);
    if (lg.L <= 256) {
        if (lg.vec_ok) { DM_SWEEP_LAUNCH(uint8_t, true) }
        DM_SWEEP_LAUNCH(uint8_t, false)
    }
    if (lg.vec_ok) { DM_SWEEP_LAUNCH(uint16_t, true) }
    DM_SWEEP_LAUNCH(uint16_t, false)
#undef DM_SWEEP_LAUNCH
}

template <int W>
static cudaError_t launch_xpass_group(const BuildItem* const* its, int m, cudaStream_t s)
{
    XBatch B;
    B.n = m;
    int64_t rows = 0;                                        // CTAs
    size_t smem = 0;
    for (int k = 0; k < m; ++k) {
        const BuildItem& b = *its[k];
        B.mask[k] = b.mask;
        B.out[k] = b.pdm;
        B.K[k] = b.K;
        B.xg[k] = xgeom(b.g, b.g.plane, b.pdm);
        B.start[k] = int(rows);
        if (W == 1 && xpass_warp_rows_ok(B.xg[k].nw, b.K)) {     // one warp per row
            B.xg[k].warp_rows = 1;
            rows += (B.xg[k].rows + kThreads / 32 - 1) / (kThreads / 32);
        } else {
            B.xg[k].rpc = xpass_rows_per_cta(B.xg[k].nw, b.K);
            rows += (B.xg[k].rows + B.xg[k].rpc - 1) / B.xg[k].rpc;
            smem = std::max(smem, size_t(B.xg[k].rpc) * (b.K < 64 ? b.K : 64) * B.xg[k].nw * 8);
        }
        if (rows > int64_t(0x7FFFFFFF)) return cudaErrorInvalidConfiguration;
    }
    B.start[m] = int(rows);
    cudaError_t e = ensure_dynamic_smem<k_xpass_mask_batch<W>>(int(smem));
    if (e != cudaSuccess) return e;
    return launch_pdl(k_xpass_mask_batch<W>, dim3(unsigned(rows)), dim3(kThreads), smem, s, B);
}

cudaError_t launch_xpass_mask_batch(const BuildItem* items, int n, cudaStream_t s)
{
    const BuildItem* by_w[4][kMaxBuildBatch];
    int count[4] = {0, 0, 0, 0};
    for (int i = 0; i < n && i < kMaxBuildBatch; ++i) {
        const int w = (items[i].K + 63) / 64 - 1;
        if (w < 0 || w > 3) return cudaErrorInvalidValue;
        by_w[w][count[w]++] = &items[i];
    }
    cudaError_t e = cudaSuccess;
    if (count[0]) e = launch_xpass_group<1>(by_w[0], count[0], s);
    if (e == cudaSuccess && count[1]) e = launch_xpass_group<2>(by_w[1], count[1], s);
    if (e == cudaSuccess && count[2]) e = launch_xpass_group<3>(by_w[2], count[2], s);
    if (e == cudaSuccess && count[3]) e = launch_xpass_group<4>(by_w[3], count[3], s);
    return e;
}

template <typename P, bool VEC>
static cudaError_t launch_line_group(const BuildItem* const* its, const LineGeom* lgs, int m,
                                     cudaStream_t s)
{
    constexpr int TC = kLineTile;
    LineBatch B;
    B.n = m;
    int64_t ctas = 0;
    size_t smem = 0;
    for (int k = 0; k < m; ++k) {
        B.buf[k] = its[k]->pdm;
        B.lg[k] = lgs[k];
        B.gdx[k] = (lgs[k].gx + TC - 1) / TC;
        B.start[k] = int(ctas);
        ctas += int64_t(B.gdx[k]) * lgs[k].n_outer * its[k]->K;
        if (ctas > int64_t(0x7FFFFFFF)) return cudaErrorInvalidConfiguration;
        smem = std::max(smem, line_pass_smem(lgs[k].L));
    }
    B.start[m] = int(ctas);
    if (smem > size_t(kLineSmemLimit)) return cudaErrorInvalidConfiguration;
    cudaError_t e = ensure_dynamic_smem<k_line_sweep_batch<TC, P, VEC>>(int(smem));
    if (e != cudaSuccess) return e;
    return launch_pdl(k_line_sweep_batch<TC, P, VEC>, dim3(unsigned(ctas)), dim3(TC), smem, s, B);
}

cudaError_t launch_line_pass_batch(const BuildItem* items, int n, int axis, cudaStream_t s)
{
    // lines of at most 256 blocks take 8-bit table positions, longer ones 16-bit; tiles of
    // whole 16-byte rows are staged as vectors
    const BuildItem* its[4][kMaxBuildBatch];
    LineGeom lgs[4][kMaxBuildBatch];
    int count[4] = {0, 0, 0, 0};
    for (int i = 0; i < n && i < kMaxBuildBatch; ++i) {
        const BuildItem& b = items[i];
        const LineGeom lg = line_geom(b.pdm, b.g.plane, b.g, axis);
        if (lg.L <= 1) continue;         // a single block per line: h == g
        const int c = (lg.L <= 256 ? 0 : 2) + (lg.vec_ok ? 1 : 0);
        its[c][count[c]] = &b;
        lgs[c][count[c]++] = lg;
    }
    cudaError_t e = cudaSuccess;
    if (count[0]) e = launch_line_group<uint8_t, false>(its[0], lgs[0], count[0], s);
    if (e == cudaSuccess && count[1])
        e = launch_line_group<uint8_t, true>(its[1], lgs[1], count[1], s);
    if (e == cudaSuccess && count[2])
        e = launch_line_group<uint16_t, false>(its[2], lgs[2], count[2], s);
    if (e == cudaSuccess && count[3])
        e = launch_line_group<uint16_t, true>(its[3], lgs[3], count[3], s);
    return e;
}

}  // namespace dmk
