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
// x pass: one CTA per block row; warp ballots turn each partition's occupancy along the
// row into a bit line in shared memory; each output is the distance to the nearest set
// bit, found with clz/ffs over at most 9 words on either side (>= 256 blocks = 255).
//
// y / z passes: a CTA stages a tile of 16 neighbouring lines (full line length) in shared
// memory and builds a doubling table of window minima (level j holds min over 2^j rows,
// 4 lines per 32-bit word with __vminu4).  h(i) <= t holds exactly when the window of
// radius t around i has a value <= t, which is monotone in t, so each output is a binary
// search over t in [1, g(i)] with two table reads per step.  Lines are rewritten in place.
#include "dm_internal.cuh"

namespace dmk {
namespace {

constexpr int kThreads = 256;

// ------------------------------------------------------------------------------ x pass
struct XGeom {
    int gx, gy, gz;
    int nw;             // 32-bit words per bit line
    int64_t G, plane;
};

struct SrcMask {        // POM bits: partition p is bit p%64 of word p/64
    const uint64_t* mask;
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

__device__ __forceinline__ uint8_t nearest_bit(const uint32_t* __restrict__ bits, int nw, int x)
{
    const int wi = x >> 5, bi = x & 31;
    const uint32_t cur = bits[wi];
    int dl = 256, dr = 256;
    uint32_t m = cur & (0xFFFFFFFFu >> (31 - bi));          // bits 0..bi
    if (m) {
        dl = bi - (31 - __clz(m));
    } else {
        for (int k = wi - 1, s = 0; k >= 0 && s < 9; --k, ++s) {
            uint32_t w = bits[k];
            if (w) { dl = x - (k * 32 + 31 - __clz(w)); break; }
        }
    }
    m = cur & (0xFFFFFFFFu << bi);                          // bits bi..31
    if (m) {
        dr = __ffs(m) - 1 - bi;
    } else {
        for (int k = wi + 1, s = 0; k < nw && s < 9; ++k, ++s) {
            uint32_t w = bits[k];
            if (w) { dr = k * 32 + __ffs(w) - 1 - x; break; }
        }
    }
    int d = min(dl, dr);
    return uint8_t(d > 255 ? 255 : d);
}

// Occupancy of (row, x) for plane p; templated sources.
template <int W>
__device__ __forceinline__ void load_src(const SrcMask& s, int64_t blk, uint64_t (&m)[4])
{
#pragma unroll
    for (int w = 0; w < W; ++w) m[w] = s.mask[blk * W + w];
}

template <int W>
__global__ void __launch_bounds__(kThreads)
k_xpass_mask(SrcMask src, int K, XGeom xg, uint8_t* __restrict__ out)
{
    extern __shared__ uint32_t s_bits[];                     // [K][nw]
    const int row = blockIdx.x;                              // z * gy + y
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t rbase = int64_t(row) * xg.gx;
    for (int x0 = 0; x0 < xg.gx; x0 += kThreads) {
        int x = x0 + tid;
        uint64_t m[4] = {0, 0, 0, 0};
        if (x < xg.gx) load_src<W>(src, rbase + x, m);
        const int wi = (x0 >> 5) + warp;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const int pmax = min(64, K - w * 64);
            for (int q = 0; q < pmax; ++q) {
                unsigned bal = __ballot_sync(0xFFFFFFFFu, (m[w] >> q) & 1);
                if (lane == 0 && wi < xg.nw) s_bits[(w * 64 + q) * xg.nw + wi] = bal;
            }
        }
    }
    __syncthreads();
    const int total = K * xg.gx;
    for (int it = tid; it < total; it += kThreads) {
        int p = it / xg.gx, x = it - p * xg.gx;
        out[int64_t(p) * xg.plane + rbase + x] = nearest_bit(s_bits + p * xg.nw, xg.nw, x);
    }
}

template <typename Src>
__device__ __forceinline__ bool occ_of(const Src& s, int64_t blk);

template <>
__device__ __forceinline__ bool occ_of<SrcMinMax8>(const SrcMinMax8& s, int64_t blk)
{
    uint32_t v = s.mm[blk];
    uint32_t mn = v & 0xFF, mx = v >> 8;
    return __ldg(s.cnt + mx + 1) > __ldg(s.cnt + mn);
}
template <>
__device__ __forceinline__ bool occ_of<SrcMinMax16>(const SrcMinMax16& s, int64_t blk)
{
    uint32_t v = s.mm[blk];
    uint32_t mn = v & 0xFFFF, mx = v >> 16;
    return __ldg(s.cnt + mx + 1) > __ldg(s.cnt + mn);
}
template <>
__device__ __forceinline__ bool occ_of<SrcOcc>(const SrcOcc& s, int64_t blk)
{
    return s.occ[blk] != 0;
}

// Single-map x pass (full recompute).  Reads the whole row's occupancy before writing,
// so `out` may alias the occupancy source.
template <typename Src>
__global__ void __launch_bounds__(kThreads)
k_xpass_single(Src src, XGeom xg, uint8_t* out)
{
    extern __shared__ uint32_t s_bits[];                     // [nw]
    const int row = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t rbase = int64_t(row) * xg.gx;
    for (int x0 = 0; x0 < xg.gx; x0 += kThreads) {
        int x = x0 + tid;
        bool o = x < xg.gx ? occ_of(src, rbase + x) : false;
        unsigned bal = __ballot_sync(0xFFFFFFFFu, o);
        const int wi = (x0 >> 5) + warp;
        if (lane == 0 && wi < xg.nw) s_bits[wi] = bal;
    }
    __syncthreads();
    for (int x = tid; x < xg.gx; x += kThreads)
        out[rbase + x] = nearest_bit(s_bits, xg.nw, x);
}

XGeom xgeom(const Geometry& g, int64_t plane)
{
    XGeom x;
    x.gx = g.gx;
    x.gy = g.gy;
    x.gz = g.gz;
    x.nw = (g.gx + 31) / 32;
    x.G = g.G;
    x.plane = plane;
    return x;
}

// ------------------------------------------------------------------------ y / z passes
struct LineGeom {
    int L;              // line length (blocks)
    int gx;             // columns along x (contiguous)
    int n_outer;        // lines per plane per x column
    int64_t s;          // element stride along the line
    int64_t os;         // stride of the outer index
    int64_t plane;      // stride between planes
    int J;              // highest sparse-table level
    int vec_ok;         // rows of 16 columns are 16-byte aligned and full
};

__global__ void __launch_bounds__(kThreads)
k_line_pass(uint8_t* buf, LineGeom lg)
{
    extern __shared__ __align__(16) uint8_t s_lvl[];        // [J+1][L][16]
    constexpr int TC = kLineTile;
    const int tid = threadIdx.x;
    const int L = lg.L;
    const int x0 = blockIdx.x * TC;
    uint8_t* base = buf + int64_t(blockIdx.z) * lg.plane + int64_t(blockIdx.y) * lg.os + x0;
    const int ncols = min(TC, lg.gx - x0);

    // ---- stage level 0 and note whether the tile can change at all (values >= 2 that
    //      are not all 255)
    int any_big = 0, any_not255 = 0;
    if (lg.vec_ok) {
        for (int r = tid; r < L; r += kThreads) {
            uint4 v = *reinterpret_cast<const uint4*>(base + int64_t(r) * lg.s);
            reinterpret_cast<uint4*>(s_lvl)[r] = v;
            unsigned w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                any_not255 |= (w4[k] != 0xFFFFFFFFu);
                // a byte >= 2 exists iff some byte has a bit above bit 0 set
                any_big |= ((w4[k] & 0xFEFEFEFEu) != 0);
            }
        }
    } else {
        for (int i = tid; i < L * TC; i += kThreads) {
            int r = i / TC, c = i - r * TC;
            uint8_t v = 255;
            if (c < ncols) v = base[int64_t(r) * lg.s + c];
            s_lvl[r * TC + c] = v;
            any_not255 |= (c < ncols) && (v != 255);
            any_big |= (c < ncols) && (v >= 2);
        }
    }
    any_big = __syncthreads_or(any_big);
    any_not255 = __syncthreads_or(any_not255);
    if (!any_big || !any_not255) return;   // all values <= 1 or all 255: h == g

    // ---- doubling table of window minima, 4 columns per word
    uint32_t* lv = reinterpret_cast<uint32_t*>(s_lvl);
    const int wpr = TC / 4;                                   // words per row
    for (int j = 1; j <= lg.J; ++j) {
        const uint32_t* prev = lv + (j - 1) * L * wpr;
        uint32_t* cur = lv + j * L * wpr;
        const int half = 1 << (j - 1);
        for (int i = tid; i < L * wpr; i += kThreads) {
            int r = i / wpr, q = i - r * wpr;
            int r2 = min(r + half, L - 1);
            cur[i] = __vminu4(prev[i], prev[r2 * wpr + q]);
        }
        __syncthreads();
    }

    // ---- outputs: binary search for the least t with min(window radius t) <= t
    for (int i = tid; i < L * TC; i += kThreads) {
        int r = i / TC, c = i - r * TC;
        if (c >= ncols) continue;
        int gv = s_lvl[r * TC + c];
        int h = gv;
        if (gv >= 2) {
            int lo = 1, hi = gv;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                int wl = max(0, r - mid), wh = min(L - 1, r + mid);
                int j = 31 - __clz(wh - wl + 1);
                const uint8_t* Lj = s_lvl + j * L * TC;
                int m = min(int(Lj[wl * TC + c]), int(Lj[(wh - (1 << j) + 1) * TC + c]));
                if (m <= mid) hi = mid; else lo = mid + 1;
            }
            h = lo;
        }
        if (h != gv) base[int64_t(r) * lg.s + c] = uint8_t(h);
    }
}

}  // namespace

size_t line_pass_smem(int L)
{
    int J = 0;
    while (J < kMaxLevels - 1 && (2 << J) <= L) ++J;
    return size_t(J + 1) * size_t(L) * kLineTile;
}

cudaError_t launch_xpass_mask(const uint64_t* mask, int K, const Geometry& g, uint8_t* pdm,
                              cudaStream_t s)
{
    XGeom xg = xgeom(g, g.plane);
    size_t smem = size_t(K) * xg.nw * 4;
    int W = (K + 63) / 64;
    SrcMask src{mask};
    const int rows = g.gy * g.gz;
    cudaError_t e = cudaSuccess;
#define DM_XPASS_CASE(WW)                                                                   \
    case WW:                                                                                \
        e = cudaFuncSetAttribute(k_xpass_mask<WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 int(smem));                                                \
        if (e != cudaSuccess) return e;                                                     \
        k_xpass_mask<WW><<<rows, kThreads, smem, s>>>(src, K, xg, pdm);                     \
        break;
    switch (W) {
        DM_XPASS_CASE(1)
        DM_XPASS_CASE(2)
        DM_XPASS_CASE(3)
        DM_XPASS_CASE(4)
    default: return cudaErrorInvalidValue;
    }
#undef DM_XPASS_CASE
    return cudaGetLastError();
}

cudaError_t launch_xpass_minmax(const void* minmax, const int32_t* cnt, const Geometry& g,
                                uint8_t* out, cudaStream_t s)
{
    XGeom xg = xgeom(g, g.G);
    size_t smem = size_t(xg.nw) * 4;
    const int rows = g.gy * g.gz;
    if (g.bpv == 1) {
        SrcMinMax8 src{static_cast<const uint16_t*>(minmax), cnt};
        k_xpass_single<SrcMinMax8><<<rows, kThreads, smem, s>>>(src, xg, out);
    } else {
        SrcMinMax16 src{static_cast<const uint32_t*>(minmax), cnt};
        k_xpass_single<SrcMinMax16><<<rows, kThreads, smem, s>>>(src, xg, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_xpass_occ(uint8_t* occ_inout, const Geometry& g, cudaStream_t s)
{
    XGeom xg = xgeom(g, g.G);
    size_t smem = size_t(xg.nw) * 4;
    SrcOcc src{occ_inout};
    k_xpass_single<SrcOcc><<<g.gy * g.gz, kThreads, smem, s>>>(src, xg, occ_inout);
    return cudaGetLastError();
}

cudaError_t launch_line_pass(uint8_t* buf, int P, int64_t plane, const Geometry& g, int axis,
                             cudaStream_t s)
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
    if (lg.L <= 1) return cudaSuccess;   // a single block per line: h == g
    int J = 0;
    while (J < kMaxLevels - 1 && (2 << J) <= lg.L) ++J;
    lg.J = J;
    lg.vec_ok = (g.gx % kLineTile == 0) && ((reinterpret_cast<uintptr_t>(buf) & 15) == 0) &&
                (plane % 16 == 0);
    size_t smem = line_pass_smem(lg.L);
    if (smem > size_t(kLineSmemLimit)) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_line_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    dim3 grid((g.gx + kLineTile - 1) / kLineTile, lg.n_outer, P);
    k_line_pass<<<grid, kThreads, smem, s>>>(buf, lg);
    return cudaGetLastError();
}

}  // namespace dmk
