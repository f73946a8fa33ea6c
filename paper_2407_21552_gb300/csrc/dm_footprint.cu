// dm_footprint.cu -- streaming the volume into per-block footprint reductions.
//
// §3.1: a block of the POM of partition p is occupied when one voxel of the block holds an
// intensity in [rho_min^p, rho_max^p]; blocks are non-overlapping b^3 cubes, and the
// footprint adds `a` voxels of interpolation apron per side (clipped at the volume).  One
// pass over the volume yields all K POMs at once as a per-block K-bit mask, and the block
// min/max of the intensity that the plain min/max full recompute needs.  The same kernel,
// with a per-intensity visibility bit instead of a partition bit, gives the exact TF
// occupancy of the plain recompute in its exact mode.
//
// Tiling: one warp per block row and one lane per block column (32 x 8 blocks per CTA),
// the CTA streaming a chunk of 4 block-slices along z.  The general kernel reads a voxel
// once per footprint row it lies in; the b = 4 / apron-1 kernels classify each voxel row
// about once and trade apron rows between warps in shared memory.  The x apron reaches
// the neighbouring block through a warp shuffle.  The vector kernel (k_pom_vec) gives a
// lane 16 bytes of a row (2 or 4 blocks); rows that are not whole 16-byte vectors, or a
// volume off a 16-byte boundary, take its ragged-row form.  The batched forms
// (k_pom_vec_batch, k_footprint_batch, k_partition_lut_batch) run the same per-CTA work
// over the concatenated grids of several volumes.
#include <algorithm>

#include "dm_build_batch.cuh"
#include "dm_internal.cuh"

namespace dmk {
namespace {

__global__ void k_partition_lut(uint8_t* __restrict__ lut, int N, int K, Borders bd)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    // largest p with v[p] <= i (borders strictly increase, v[0] = 0)
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (bd.v[mid] <= i) lo = mid; else hi = mid - 1;
    }
    lut[i] = static_cast<uint8_t>(lo);
}

// Several partition tables in one grid, 256 entries a CTA; the borders of all tables are
// packed into the parameters (K + 1 each).
constexpr int kLutBorderCap = 4096;
struct LutBatch {
    int n;
    int start[kMaxBuildBatch + 1];             // first CTA of each table
    uint8_t* lut[kMaxBuildBatch];
    int N[kMaxBuildBatch], K[kMaxBuildBatch], boff[kMaxBuildBatch];
    int32_t bv[kLutBorderCap];
};

__global__ void k_partition_lut_batch(const __grid_constant__ LutBatch B)
{
    const int t = batch_item_of(B.start, B.n, int(blockIdx.x));
    const int i = (int(blockIdx.x) - B.start[t]) * int(blockDim.x) + int(threadIdx.x);
    if (i >= B.N[t]) return;
    const int32_t* v = B.bv + B.boff[t];
    int lo = 0, hi = B.K[t] - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (v[mid] <= i) lo = mid; else hi = mid - 1;
    }
    B.lut[t][i] = static_cast<uint8_t>(lo);
}

template <typename T>
struct Quad;                                   // four consecutive voxels in one load
template <>
struct Quad<uint8_t> {
    using V = uint32_t;
    __device__ static unsigned get(V v, int k) { return (v >> (8 * k)) & 0xFFu; }
};
template <>
struct Quad<uint16_t> {
    using V = uint2;
    __device__ static unsigned get(V v, int k)
    {
        return ((k < 2 ? v.x : v.y) >> (16 * (k & 1))) & 0xFFFFu;
    }
};

struct FpParams {
    int X, Y, Z;
    int gx, gy, gz;
    int b, a, N, W64;
    int zchunk;                                // block-slices per CTA
    int sh;                                    // uniform partitions of 2^sh intensities (else -1)
};

enum { kModePom = 0, kModeVis = 1 };
constexpr int kWarps = 8;
constexpr int kMaxRows = 12;                   // b + 2a rows of a footprint when b = 4
constexpr size_t kFpTabLimit = 64 * 1024;     // one-hot mask table in shared memory

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// Accumulates one voxel into a mask (NW 32-bit words) and a min / max.
template <int NW, int MODE>
__device__ __forceinline__ void classify(unsigned v, int N, const uint8_t* s_cls, uint32_t (&m)[NW],
                                         unsigned& mn, unsigned& mx)
{
    if (v > unsigned(N - 1)) v = unsigned(N - 1);
    const unsigned c = s_cls[v];
    if (MODE == kModePom) {
#pragma unroll
        for (int w = 0; w < NW; ++w) m[w] |= ((c >> 5) == unsigned(w)) ? (1u << (c & 31)) : 0u;
        mn = min(mn, v);
        mx = max(mx, v);
    } else {
        m[0] |= c;
    }
}

// One warp per block row, one lane per block column; the CTA streams its chunk of
// block-slices along z.  Per voxel slice: every footprint row of the warp's block row is
// loaded once (FAST: the lane's 4 core voxels in one load), the lane's core mask and the
// masks of its first / last `a` voxels are formed, the x apron comes from the neighbour
// lanes by shuffle (lanes 0 and 31 read theirs), and the rows are ORed into the slice
// mask.  The slice mask goes to every block whose z footprint holds the slice (at most 3
// when a <= b: a ring of per-thread accumulators in shared memory); a block is written
// when its last slice has been added.
template <typename T, int NW, int MODE, bool FAST>
__device__ __forceinline__ void
footprint_cta(const T* __restrict__ vol, const FpParams& p, const uint8_t* __restrict__ lut,
              const int32_t* __restrict__ cnt, uint64_t* __restrict__ mask, void* minmax,
              uint8_t* __restrict__ occ, int cx, int cy, int cz)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint8_t* s_cls = smem;
    uint32_t* s_ring = reinterpret_cast<uint32_t*>(smem + align16(size_t(p.N)));  // [3][NW][256]
    uint32_t* s_rmm = s_ring + 3 * NW * kWarps * 32;                                // [3][256]
    for (int i = tid; i < p.N; i += kWarps * 32)
        s_cls[i] = MODE == kModePom ? lut[i] : uint8_t(cnt[i + 1] > cnt[i]);
    __syncthreads();
    const int bx = cx * 32 + lane, by = cy * kWarps + warp;
    if (by >= p.gy) return;                                   // warp-uniform; no CTA barrier follows
    const int b = p.b, a = p.a, X = p.X, N = p.N;
    const bool col_ok = bx < p.gx;
    const int zb0 = cz * p.zchunk, zb1 = min(p.gz, zb0 + p.zchunk);
    const int zs = max(0, zb0 * b - a), ze = min(p.Z - 1, (zb1 - 1) * b + b - 1 + a);
    const int y0 = max(0, by * b - a), y1 = min(p.Y - 1, by * b + b - 1 + a);
    const int nrows = y1 - y0 + 1;
    const int xc0 = bx * b;
    const int64_t rowX = X;
    for (int z = zs; z <= ze; ++z) {
        uint32_t S[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) S[w] = 0;
        unsigned smn = 0xFFFFu, smx = 0;
        const T* slice = vol + int64_t(z) * p.Y * rowX;
        typename Quad<T>::V q[FAST ? kMaxRows : 1];
        if (FAST) {                                           // issue all row loads first
#pragma unroll
            for (int r = 0; r < kMaxRows; ++r)
                if (r < nrows && col_ok)
                    q[r] = *reinterpret_cast<const typename Quad<T>::V*>(
                        slice + int64_t(y0 + r) * rowX + xc0);
        }
#pragma unroll 1
        for (int r = 0; r < nrows; ++r) {
            const T* row = slice + int64_t(y0 + r) * rowX;
            uint32_t core[NW], head[NW], tail[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) core[w] = head[w] = tail[w] = 0;
            unsigned cmn = 0xFFFFu, cmx = 0, hmn = 0xFFFFu, hmx = 0, tmn = 0xFFFFu, tmx = 0;
            if (col_ok) {
                if (FAST) {
                    typename Quad<T>::V v4 = q[0];
#pragma unroll
                    for (int rr = 1; rr < kMaxRows; ++rr)
                        if (rr == r) v4 = q[rr];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        uint32_t m1[NW];
#pragma unroll
                        for (int w = 0; w < NW; ++w) m1[w] = 0;
                        unsigned mn1 = 0xFFFFu, mx1 = 0;
                        classify<NW, MODE>(Quad<T>::get(v4, k), N, s_cls, m1, mn1, mx1);
#pragma unroll
                        for (int w = 0; w < NW; ++w) core[w] |= m1[w];
                        cmn = min(cmn, mn1);
                        cmx = max(cmx, mx1);
                        if (k < a) {
#pragma unroll
                            for (int w = 0; w < NW; ++w) head[w] |= m1[w];
                            hmn = min(hmn, mn1);
                            hmx = max(hmx, mx1);
                        }
                        if (k >= 4 - a) {
#pragma unroll
                            for (int w = 0; w < NW; ++w) tail[w] |= m1[w];
                            tmn = min(tmn, mn1);
                            tmx = max(tmx, mx1);
                        }
                    }
                } else {
                    for (int k = 0; k < b && xc0 + k < X; ++k) {
                        uint32_t m1[NW];
#pragma unroll
                        for (int w = 0; w < NW; ++w) m1[w] = 0;
                        unsigned mn1 = 0xFFFFu, mx1 = 0;
                        classify<NW, MODE>(row[xc0 + k], N, s_cls, m1, mn1, mx1);
#pragma unroll
                        for (int w = 0; w < NW; ++w) core[w] |= m1[w];
                        cmn = min(cmn, mn1);
                        cmx = max(cmx, mx1);
                        if (k < a) {
#pragma unroll
                            for (int w = 0; w < NW; ++w) head[w] |= m1[w];
                            hmn = min(hmn, mn1);
                            hmx = max(hmx, mx1);
                        }
                        if (k >= b - a) {
#pragma unroll
                            for (int w = 0; w < NW; ++w) tail[w] |= m1[w];
                            tmn = min(tmn, mn1);
                            tmx = max(tmx, mx1);
                        }
                    }
                }
            }
            // x apron: the last `a` voxels of the block to the left, the first `a` of the
            // block to the right (neighbour lanes; lanes 0 / 31 read them from memory)
            uint32_t left[NW], right[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                left[w] = __shfl_up_sync(0xFFFFFFFFu, tail[w], 1);
                right[w] = __shfl_down_sync(0xFFFFFFFFu, head[w], 1);
            }
            unsigned lmm = __shfl_up_sync(0xFFFFFFFFu, tmn | (tmx << 16), 1);
            unsigned rmm = __shfl_down_sync(0xFFFFFFFFu, hmn | (hmx << 16), 1);
            if (lane == 0 || lane == 31) {
                const bool lft = lane == 0;
#pragma unroll
                for (int w = 0; w < NW; ++w) (lft ? left[w] : right[w]) = 0;
                unsigned mn2 = 0xFFFFu, mx2 = 0;
                uint32_t m2[NW];
#pragma unroll
                for (int w = 0; w < NW; ++w) m2[w] = 0;
                if (col_ok) {
                    for (int k = 0; k < a; ++k) {
                        const int x = lft ? xc0 - 1 - k : xc0 + b + k;
                        if (x >= 0 && x < X) classify<NW, MODE>(row[x], N, s_cls, m2, mn2, mx2);
                    }
                }
#pragma unroll
                for (int w = 0; w < NW; ++w) (lft ? left[w] : right[w]) = m2[w];
                (lft ? lmm : rmm) = mn2 | (mx2 << 16);
            }
#pragma unroll
            for (int w = 0; w < NW; ++w) S[w] |= core[w] | left[w] | right[w];
            smn = min(smn, min(cmn, min(lmm & 0xFFFFu, rmm & 0xFFFFu)));
            smx = max(smx, max(cmx, max(lmm >> 16, rmm >> 16)));
        }
        // hand the slice to the blocks whose z footprint holds it
        const int bzc = z / b;
        for (int bz = max(zb0, bzc - 1); bz <= min(zb1 - 1, bzc + 1); ++bz) {
            const int f0 = max(0, bz * b - a), f1 = min(p.Z - 1, bz * b + b - 1 + a);
            if (z < f0 || z > f1) continue;
            const int slot = bz % 3;
            uint32_t* rg = s_ring + slot * NW * (kWarps * 32) + tid;
            uint32_t* rm = s_rmm + slot * (kWarps * 32) + tid;
            unsigned mn = smn, mx = smx;
            if (z == f0) {
#pragma unroll
                for (int w = 0; w < NW; ++w) rg[w * kWarps * 32] = S[w];
            } else {
#pragma unroll
                for (int w = 0; w < NW; ++w) rg[w * kWarps * 32] |= S[w];
                mn = min(mn, *rm & 0xFFFFu);
                mx = max(mx, *rm >> 16);
            }
            *rm = mn | (mx << 16);
            if (z == f1 && col_ok) {
                const int64_t blk = (int64_t(bz) * p.gy + by) * p.gx + bx;
                if (MODE == kModePom) {
                    for (int w64 = 0; w64 < p.W64; ++w64) {
                        const uint32_t lo = (2 * w64 < NW) ? rg[(2 * w64) * kWarps * 32] : 0u;
                        const uint32_t hi = (2 * w64 + 1 < NW) ? rg[(2 * w64 + 1) * kWarps * 32] : 0u;
                        mask[blk * p.W64 + w64] = uint64_t(lo) | (uint64_t(hi) << 32);
                    }
                    if (minmax) {
                        if (sizeof(T) == 1)
                            reinterpret_cast<uint16_t*>(minmax)[blk] = uint16_t(mn | (mx << 8));
                        else
                            reinterpret_cast<uint32_t*>(minmax)[blk] = mn | (mx << 16);
                    }
                } else {
                    occ[blk] = uint8_t(rg[0] != 0);
                }
            }
        }
    }
}

template <typename T, int NW, int MODE, bool FAST>
__global__ void __launch_bounds__(kWarps * 32)
k_footprint(const T* __restrict__ vol, FpParams p, const uint8_t* __restrict__ lut,
            const int32_t* __restrict__ cnt, uint64_t* __restrict__ mask, void* minmax,
            uint8_t* __restrict__ occ)
{
    pdl_wait();
    footprint_cta<T, NW, MODE, FAST>(vol, p, lut, cnt, mask, minmax, occ, blockIdx.x, blockIdx.y,
                                     blockIdx.z);
}

// Several volumes' POM builds with the general kernel (any b and apron) in one grid, laid
// out as for the vector kernel's batch.
struct FpBatchItem {
    const void* vol;
    FpParams p;
    const uint8_t* lut;
    uint64_t* mask;
    void* minmax;
    int gdx, gdy;                              // the volume's grid in x and y
};
struct FpBatch {
    int n;
    int start[kMaxBuildBatch + 1];             // first CTA of each volume
    FpBatchItem it[kMaxBuildBatch];
};

template <typename T, int NW>
__global__ void __launch_bounds__(kWarps * 32)
k_footprint_batch(const __grid_constant__ FpBatch B)
{
    const int i = batch_item_of(B.start, B.n, int(blockIdx.x));
    const FpBatchItem& it = B.it[i];
    const int local = int(blockIdx.x) - B.start[i];
    const int cx = local % it.gdx, rest = local / it.gdx;
    pdl_wait();
    footprint_cta<T, NW, kModePom, false>(static_cast<const T*>(it.vol), it.p, it.lut, nullptr,
                                          it.mask, it.minmax, nullptr, cx, rest % it.gdy,
                                          rest / it.gdy);
}

// Onehot partition / visibility bit of one (already clamped) intensity.
template <int NW, int MODE>
__device__ __forceinline__ void onehot(unsigned c, uint32_t (&m)[NW])
{
    if (MODE == kModePom) {
#pragma unroll
        for (int w = 0; w < NW; ++w) m[w] = ((c >> 5) == unsigned(w)) ? (1u << (c & 31)) : 0u;
    } else {
        m[0] = c;
    }
}

// One-hot partition mask of an intensity: from the mask table (TAB) or the class table.
template <int NW, int MODE, bool TAB>
__device__ __forceinline__ void lookup_mask(const unsigned char* s_tab, unsigned v, uint32_t (&m)[NW])
{
    if (TAB) {
        const uint32_t* t = reinterpret_cast<const uint32_t*>(s_tab) + size_t(v) * NW;
#pragma unroll
        for (int w = 0; w < NW; ++w) m[w] = t[w];
    } else {
        onehot<NW, MODE>(s_tab[v], m);
    }
}

// Footprint mask and min / max of one voxel row for the b = 4, apron-1 kernel: the lane's
// 4 voxels, the last voxel of the left block and the first of the right one (shuffles;
// lanes 0 / 31 take the edge voxel they loaded).  `ok` (the row lies in the volume) is
// warp-uniform.  An empty row gives mask 0 and (min, max) = (FFFF, 0).
template <typename T, int NW, int MODE, bool TAB>
__device__ __forceinline__ void row_footprint(const typename Quad<T>::V& q, unsigned ev, bool ok,
                                              bool col_ok, int lane, unsigned nmax,
                                              const unsigned char* s_tab, uint32_t (&R)[NW],
                                              unsigned& rmn, unsigned& rmx)
{
#pragma unroll
    for (int w = 0; w < NW; ++w) R[w] = 0;
    rmn = 0xFFFFu;
    rmx = 0;
    if (!ok) return;
    uint32_t core[NW], head[NW], tail[NW], edge[NW];
    unsigned cmn = 0xFFFFu, cmx = 0, hv = 0, tv = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) core[w] = head[w] = tail[w] = edge[w] = 0;
    if (col_ok) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned v = min(Quad<T>::get(q, k), nmax);
            uint32_t m1[NW];
            lookup_mask<NW, MODE, TAB>(s_tab, v, m1);
#pragma unroll
            for (int w = 0; w < NW; ++w) core[w] |= m1[w];
            if (k == 0) {
#pragma unroll
                for (int w = 0; w < NW; ++w) head[w] = m1[w];
                hv = v;
            }
            if (k == 3) {
#pragma unroll
                for (int w = 0; w < NW; ++w) tail[w] = m1[w];
                tv = v;
            }
            cmn = min(cmn, v);
            cmx = max(cmx, v);
        }
    }
    const bool has_e = ev != 0xFFFFFFFFu;
    if (has_e) {
        ev = min(ev, nmax);
        lookup_mask<NW, MODE, TAB>(s_tab, ev, edge);
    }
    uint32_t left[NW], right[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        left[w] = __shfl_up_sync(0xFFFFFFFFu, tail[w], 1);
        right[w] = __shfl_down_sync(0xFFFFFFFFu, head[w], 1);
    }
    const unsigned tpack = col_ok ? (tv | (tv << 16)) : 0xFFFFu;
    const unsigned hpack = col_ok ? (hv | (hv << 16)) : 0xFFFFu;
    unsigned lmm = __shfl_up_sync(0xFFFFFFFFu, tpack, 1);
    unsigned rmm = __shfl_down_sync(0xFFFFFFFFu, hpack, 1);
    if (lane == 0) {
#pragma unroll
        for (int w = 0; w < NW; ++w) left[w] = edge[w];
        lmm = has_e ? (ev | (ev << 16)) : 0xFFFFu;
    }
    if (lane == 31) {
#pragma unroll
        for (int w = 0; w < NW; ++w) right[w] = edge[w];
        rmm = has_e ? (ev | (ev << 16)) : 0xFFFFu;
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) R[w] = core[w] | left[w] | right[w];
    rmn = min(cmn, min(lmm & 0xFFFFu, rmm & 0xFFFFu));
    rmx = max(cmx, max(lmm >> 16, rmm >> 16));
}

// The footprint kernel for b = 4 and apron 1, with X % 4 == 0 and an aligned volume.  A
// lane's block covers 4 voxels of a row (one vector load) and its x apron comes from the
// neighbouring lanes (row_footprint).  Every voxel row is classified about once: a warp
// classifies the 4 core rows of its block row and takes its two apron rows from the
// neighbouring warps' first and last core rows through shared memory (one CTA barrier per
// voxel slice, double-buffered); the CTA's first and last warps classify the CTA's outer
// apron rows themselves.  Min / max are taken on clamped intensities.  TAB: one-hot masks
// read from a shared-memory table (K <= 64).  Same outputs as k_footprint.
template <typename T, int NW, int MODE, bool TAB>
__global__ void __launch_bounds__(kWarps * 32)
k_footprint41(const T* __restrict__ vol, FpParams p, const uint8_t* __restrict__ lut,
               const int32_t* __restrict__ cnt, uint64_t* __restrict__ mask, void* minmax,
               uint8_t* __restrict__ occ)
{
    constexpr int TW = kWarps * 32;
    extern __shared__ __align__(16) unsigned char smem[];
    pdl_wait();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned char* s_tab = smem;
    const size_t tab_bytes = TAB ? size_t(p.N) * NW * 4 : size_t(p.N);
    uint32_t* s_ring = reinterpret_cast<uint32_t*>(smem + align16(tab_bytes));
    uint32_t* s_rmm = s_ring + 3 * NW * TW;
    uint32_t* s_xr = s_rmm + 3 * TW;                        // [2][2][kWarps][NW][32]
    uint32_t* s_xmm = s_xr + 2 * 2 * kWarps * NW * 32;      // [2][2][kWarps][32]
    for (int i = tid; i < p.N; i += TW) {
        if (TAB) {
            const unsigned c = lut[i];
            uint32_t* t = reinterpret_cast<uint32_t*>(s_tab) + size_t(i) * NW;
#pragma unroll
            for (int w = 0; w < NW; ++w) t[w] = ((c >> 5) == unsigned(w)) ? (1u << (c & 31)) : 0u;
        } else {
            s_tab[i] = MODE == kModePom ? lut[i] : uint8_t(cnt[i + 1] > cnt[i]);
        }
    }
    __syncthreads();
    const int bx = blockIdx.x * 32 + lane, by = blockIdx.y * kWarps + warp;
    const bool by_ok = by < p.gy;           // warp-uniform; every warp joins the barriers
    const int X = p.X, Y = p.Y;
    const unsigned nmax = unsigned(p.N - 1);
    const bool col_ok = bx < p.gx;
    const int xc0 = bx * 4;
    const int xe = lane == 0 ? xc0 - 1 : xc0 + 4;
    const bool edge_ok = col_ok && (lane == 0 || lane == 31) && xe >= 0 && xe < X;
    const int zb0 = blockIdx.z * p.zchunk, zb1 = min(p.gz, zb0 + p.zchunk);
    const int zs = max(0, zb0 * 4 - 1), ze = min(p.Z - 1, (zb1 - 1) * 4 + 4);
    const int y0 = by * 4;                                  // first core row
    // the extra row: the CTA's top apron row (warp 0) or bottom apron row (last warp)
    const bool has_x = warp == 0 || warp == kWarps - 1;
    const int yx = warp == 0 ? y0 - 1 : y0 + 4;
    const int64_t rowX = X;
    for (int z = zs; z <= ze; ++z) {
        const T* slice = vol + int64_t(z) * Y * rowX;
        typename Quad<T>::V q[5];
        unsigned e[5];
        bool okr[5];
#pragma unroll
        for (int t = 0; t < 5; ++t) {                         // issue every load first
            const int y = t < 4 ? y0 + t : yx;
            okr[t] = (t < 4 || has_x) && y >= 0 && y < Y;     // warp-uniform
            q[t] = typename Quad<T>::V{};
            if (okr[t] && col_ok)
                q[t] = *reinterpret_cast<const typename Quad<T>::V*>(slice + int64_t(y) * rowX + xc0);
            e[t] = (okr[t] && edge_ok) ? unsigned(slice[int64_t(y) * rowX + xe]) : 0xFFFFFFFFu;
        }
        uint32_t R[5][NW];
        unsigned rmn[5], rmx[5];
#pragma unroll
        for (int t = 0; t < 5; ++t)
            row_footprint<T, NW, MODE, TAB>(q[t], e[t], okr[t], col_ok, lane, nmax, s_tab, R[t],
                                            rmn[t], rmx[t]);
        // publish the first and last core rows for the neighbouring warps
        const int buf = z & 1;
        uint32_t* xf = s_xr + ((buf * 2 + 0) * kWarps + warp) * NW * 32 + lane;
        uint32_t* xl = s_xr + ((buf * 2 + 1) * kWarps + warp) * NW * 32 + lane;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            xf[w * 32] = R[0][w];
            xl[w * 32] = R[3][w];
        }
        s_xmm[((buf * 2 + 0) * kWarps + warp) * 32 + lane] = rmn[0] | (rmx[0] << 16);
        s_xmm[((buf * 2 + 1) * kWarps + warp) * 32 + lane] = rmn[3] | (rmx[3] << 16);
        __syncthreads();
        uint32_t S[NW];
        unsigned smn = min(min(rmn[0], rmn[1]), min(rmn[2], rmn[3]));
        unsigned smx = max(max(rmx[0], rmx[1]), max(rmx[2], rmx[3]));
#pragma unroll
        for (int w = 0; w < NW; ++w) S[w] = R[0][w] | R[1][w] | R[2][w] | R[3][w];
        if (warp > 0) {                                       // row y0 - 1: warp above's last
            const uint32_t* nl = s_xr + ((buf * 2 + 1) * kWarps + warp - 1) * NW * 32 + lane;
#pragma unroll
            for (int w = 0; w < NW; ++w) S[w] |= nl[w * 32];
            const unsigned mm = s_xmm[((buf * 2 + 1) * kWarps + warp - 1) * 32 + lane];
            smn = min(smn, mm & 0xFFFFu);
            smx = max(smx, mm >> 16);
        }
        if (warp < kWarps - 1) {                              // row y0 + 4: warp below's first
            const uint32_t* nf = s_xr + ((buf * 2 + 0) * kWarps + warp + 1) * NW * 32 + lane;
#pragma unroll
            for (int w = 0; w < NW; ++w) S[w] |= nf[w * 32];
            const unsigned mm = s_xmm[((buf * 2 + 0) * kWarps + warp + 1) * 32 + lane];
            smn = min(smn, mm & 0xFFFFu);
            smx = max(smx, mm >> 16);
        }
        if (has_x) {
#pragma unroll
            for (int w = 0; w < NW; ++w) S[w] |= R[4][w];
            smn = min(smn, rmn[4]);
            smx = max(smx, rmx[4]);
        }
        if (!by_ok) continue;
        // hand the slice to the blocks whose z footprint holds it
        const int bzc = z >> 2;
        for (int bz = max(zb0, bzc - 1); bz <= min(zb1 - 1, bzc + 1); ++bz) {
            const int f0 = max(0, bz * 4 - 1), f1 = min(p.Z - 1, bz * 4 + 4);
            if (z < f0 || z > f1) continue;
            const int slot = bz % 3;
            uint32_t* rg = s_ring + slot * NW * TW + tid;
            uint32_t* rm = s_rmm + slot * TW + tid;
            unsigned mn = smn, mx = smx;
            if (z == f0) {
#pragma unroll
                for (int w = 0; w < NW; ++w) rg[w * TW] = S[w];
            } else {
#pragma unroll
                for (int w = 0; w < NW; ++w) rg[w * TW] |= S[w];
                mn = min(mn, *rm & 0xFFFFu);
                mx = max(mx, *rm >> 16);
            }
            *rm = mn | (mx << 16);
            if (z == f1 && col_ok) {
                const int64_t blk = (int64_t(bz) * p.gy + by) * p.gx + bx;
                if (MODE == kModePom) {
                    for (int w64 = 0; w64 < p.W64; ++w64) {
                        const uint32_t lo = (2 * w64 < NW) ? rg[(2 * w64) * TW] : 0u;
                        const uint32_t hi = (2 * w64 + 1 < NW) ? rg[(2 * w64 + 1) * TW] : 0u;
                        mask[blk * p.W64 + w64] = uint64_t(lo) | (uint64_t(hi) << 32);
                    }
                    if (minmax) {
                        if (sizeof(T) == 1)
                            reinterpret_cast<uint16_t*>(minmax)[blk] = uint16_t(mn | (mx << 8));
                        else
                            reinterpret_cast<uint32_t*>(minmax)[blk] = mn | (mx << 16);
                    }
                } else {
                    occ[blk] = uint8_t(rg[0] != 0);
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// The b = 4, apron-1 footprint kernel with 16-byte voxel loads (X a multiple of 16 / sizeof(T)
// and a 16-byte aligned volume).  A lane loads 16 bytes of a voxel row, VL = 16 / sizeof(T)
// voxels, i.e. BL = VL / 4 whole blocks; the 32 lanes of a warp cover 32 * VL voxels of one
// block row, the CTA's 8 warps 8 block rows, and the CTA streams a chunk of block-slices
// along z.  Per voxel slice and warp:
//  - each voxel's one-hot partition mask (or visibility bit) comes from a shared-memory
//    table indexed by the clamped intensity; min / max are taken on whole 32-bit words
//    (two 16-bit or four 8-bit voxels per operation);
//  - the x footprint of a block is its 4 voxels plus the last voxel of the block to the left
//    and the first of the block to the right: inside the lane directly, across lanes by a
//    shuffle (the CTA's outermost lanes load the edge voxel themselves);
//  - rows: a warp handles the 4 core rows of its block row.  The footprints of its first
//    and last row go through shared memory to the warps above and below, which hold them as
//    apron rows; warp 0 and warp 7 load the CTA's outer apron rows themselves.  One CTA
//    barrier per slice (double-buffered);
//  - z: a slice belongs to one or two block-slices; their running masks and min / max stay
//    in registers, and a block is written once its last slice is in (16-byte mask stores);
//  - the next slice's rows are copied into shared memory (cp.async) while the current one
//    is reduced, so that the voxel reads stay in flight.
// OR distributes over the footprint's parts and min / max likewise, so the result is the
// footprint reduction of §3.1 whatever order the parts are combined in.
constexpr int kVZChunk = 8;                    // block-slices per CTA

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src)
{
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem_src) : "memory");
}

template <typename T>
struct VTraits;
template <>
struct VTraits<uint16_t> {
    static constexpr int VL = 8;
    __device__ static uint32_t vmin(uint32_t a, uint32_t b) { return min_u16x2(a, b); }
    __device__ static uint32_t vmax(uint32_t a, uint32_t b)
    {
        uint32_t d;
        asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
        return d;
    }
    __device__ static unsigned get(uint32_t w, int k) { return (w >> (16 * k)) & 0xFFFFu; }
    static constexpr int PER_WORD = 2;
    static constexpr uint32_t NEUTRAL_MIN = 0xFFFFFFFFu;
};
template <>
struct VTraits<uint8_t> {
    static constexpr int VL = 16;
    __device__ static uint32_t vmin(uint32_t a, uint32_t b) { return __vminu4(a, b); }
    __device__ static uint32_t vmax(uint32_t a, uint32_t b) { return __vmaxu4(a, b); }
    __device__ static unsigned get(uint32_t w, int k) { return (w >> (8 * k)) & 0xFFu; }
    static constexpr int PER_WORD = 4;
    static constexpr uint32_t NEUTRAL_MIN = 0xFFFFFFFFu;
};

// Footprint masks and min / max of the BL blocks of a lane from per-voxel-position parts
// (one row, or several rows already combined position by position): `core` = OR of each
// block's 4 voxels, `first` / `last` = its first / last voxel, `em`, `emn`, `emx` = the edge
// voxel of lanes 0 and 31; `wmn` / `wmx` = the 4 words of voxel minima / maxima.
template <typename T, int NW>
__device__ __forceinline__ void lane_footprint(const uint32_t (&core)[16 / sizeof(T) / 4][NW],
                                               const uint32_t (&first)[16 / sizeof(T) / 4][NW],
                                               const uint32_t (&last)[16 / sizeof(T) / 4][NW],
                                               const uint32_t (&em)[NW], unsigned emn, unsigned emx,
                                               const uint32_t (&wmn)[4], const uint32_t (&wmx)[4],
                                               int lane, bool want_mm,
                                               uint32_t (&fp)[16 / sizeof(T) / 4][NW],
                                               unsigned (&fmn)[16 / sizeof(T) / 4],
                                               unsigned (&fmx)[16 / sizeof(T) / 4])
{
    using Tr = VTraits<T>;
    constexpr int BL = Tr::VL / 4;
    uint32_t lft[NW], rgt[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        lft[w] = __shfl_up_sync(0xFFFFFFFFu, last[BL - 1][w], 1);
        rgt[w] = __shfl_down_sync(0xFFFFFFFFu, first[0][w], 1);
        if (lane == 0) lft[w] = em[w];
        if (lane == 31) rgt[w] = em[w];
    }
#pragma unroll
    for (int j = 0; j < BL; ++j)
#pragma unroll
        for (int w = 0; w < NW; ++w)
            fp[j][w] = core[j][w] | (j == 0 ? lft[w] : last[j - 1][w]) |
                       (j == BL - 1 ? rgt[w] : first[j + 1][w]);
#pragma unroll
    for (int j = 0; j < BL; ++j) {
        fmn[j] = 0xFFFFu;
        fmx[j] = 0;
    }
    if (!want_mm) return;
    // voxel minima / maxima of the positions next to the lane (packed min | max << 16)
    constexpr int VB = 32 / Tr::PER_WORD;                     // bits per voxel in a word
    const unsigned lastv = (wmn[3] >> (32 - VB)) | ((wmx[3] >> (32 - VB)) << 16);
    const unsigned firstv = Tr::get(wmn[0], 0) | (Tr::get(wmx[0], 0) << 16);
    unsigned lp = __shfl_up_sync(0xFFFFFFFFu, lastv, 1);
    unsigned rp = __shfl_down_sync(0xFFFFFFFFu, firstv, 1);
    if (lane == 0) lp = emn | (emx << 16);
    if (lane == 31) rp = emn | (emx << 16);
#pragma unroll
    for (int j = 0; j < BL; ++j) {
        unsigned mn, mx;
        if constexpr (sizeof(T) == 2) {                       // block j: words 2j, 2j+1
            const uint32_t a = Tr::vmin(wmn[2 * j], wmn[2 * j + 1]);
            const uint32_t b = Tr::vmax(wmx[2 * j], wmx[2 * j + 1]);
            mn = min(a & 0xFFFFu, a >> 16);
            mx = max(b & 0xFFFFu, b >> 16);
            const unsigned bef = j == 0 ? lp : (Tr::get(wmn[2 * j - 1], 1) | (Tr::get(wmx[2 * j - 1], 1) << 16));
            const unsigned aft = j == BL - 1 ? rp : (Tr::get(wmn[2 * j + 2], 0) | (Tr::get(wmx[2 * j + 2], 0) << 16));
            mn = min(mn, min(bef & 0xFFFFu, aft & 0xFFFFu));
            mx = max(mx, max(bef >> 16, aft >> 16));
        } else {                                              // block j: word j
            const uint32_t a = min_u16x2(wmn[j] & 0x00FF00FFu, (wmn[j] >> 8) & 0x00FF00FFu);
            const uint32_t b = VTraits<uint16_t>::vmax(wmx[j] & 0x00FF00FFu, (wmx[j] >> 8) & 0x00FF00FFu);
            mn = min(a & 0xFFFFu, a >> 16);
            mx = max(b & 0xFFFFu, b >> 16);
            const unsigned bef = j == 0 ? lp : (Tr::get(wmn[j - 1], 3) | (Tr::get(wmx[j - 1], 3) << 16));
            const unsigned aft = j == BL - 1 ? rp : (Tr::get(wmn[j + 1], 0) | (Tr::get(wmx[j + 1], 0) << 16));
            mn = min(mn, min(bef & 0xFFFFu, aft & 0xFFFFu));
            mx = max(mx, max(bef >> 16, aft >> 16));
        }
        fmn[j] = mn;
        fmx[j] = mx;
    }
}

// Shift by a register amount; amounts above 31 give 0 (PTX shl clamps the amount).
__device__ __forceinline__ uint32_t shl_clamped(uint32_t v, uint32_t n)
{
    uint32_t d;
    asm("shl.b32 %0, %1, %2;" : "=r"(d) : "r"(v), "r"(n));
    return d;
}

// One voxel row of a lane: per-position parts from one 16-byte vector `q` (meaningful
// when `ok`) and the edge voxel `ev` (lanes 0 / 31; 0xFFFFFFFF = none).  SHIFT: uniform
// partitions of 2^sh intensities, the partition is the clamped intensity >> sh; otherwise
// the one-hot mask (or visibility bit) comes from the shared-memory table.
template <typename T, int NW, bool SHIFT>
__device__ __forceinline__ void onehot_of(unsigned x, unsigned sh, const uint32_t* __restrict__ s_tab,
                                          uint32_t (&m)[NW])
{
    if (SHIFT) {
        const unsigned c = x >> sh;
        m[0] = shl_clamped(1u, c);
        if (NW > 1) m[NW - 1] = shl_clamped(1u, c - 32u);
    } else if (NW == 2) {
        const uint2 t2 = reinterpret_cast<const uint2*>(s_tab)[x];
        m[0] = t2.x;
        m[NW - 1] = t2.y;
    } else {
        m[0] = s_tab[x];
    }
}

template <typename T, int NW, bool SHIFT>
__device__ __forceinline__ void lane_row(const uint4& q, unsigned ev, bool ok, uint32_t nmax2,
                                         unsigned nmax, unsigned sh,
                                         const uint32_t* __restrict__ s_tab,
                                         uint32_t (&core)[16 / sizeof(T) / 4][NW],
                                         uint32_t (&first)[16 / sizeof(T) / 4][NW],
                                         uint32_t (&last)[16 / sizeof(T) / 4][NW],
                                         uint32_t (&em)[NW], unsigned& emn, unsigned& emx,
                                         uint32_t (&wv)[4])
{
    using Tr = VTraits<T>;
    constexpr int BL = Tr::VL / 4;
    constexpr int PW = Tr::PER_WORD;
    wv[0] = q.x; wv[1] = q.y; wv[2] = q.z; wv[3] = q.w;
#pragma unroll
    for (int j = 0; j < BL; ++j)
#pragma unroll
        for (int w = 0; w < NW; ++w) core[j][w] = first[j][w] = last[j][w] = 0;
    if (ok) {
#pragma unroll
        for (int k = 0; k < 4; ++k) wv[k] = Tr::vmin(wv[k], nmax2);
#pragma unroll
        for (int j = 0; j < BL; ++j) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int v = 4 * j + i;                       // voxel position in the lane
                uint32_t m[NW];
                onehot_of<T, NW, SHIFT>(Tr::get(wv[v / PW], v % PW), sh, s_tab, m);
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    core[j][w] |= m[w];
                    if (i == 0) first[j][w] = m[w];
                    if (i == 3) last[j][w] = m[w];
                }
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) wv[k] = Tr::NEUTRAL_MIN;
    }
    if (ev != 0xFFFFFFFFu) {
        const unsigned x = min(ev, nmax);
        onehot_of<T, NW, SHIFT>(x, sh, s_tab, em);
        emn = x;
        emx = x;
    } else {
#pragma unroll
        for (int w = 0; w < NW; ++w) em[w] = 0;
        emn = 0xFFFFu;
        emx = 0;
    }
}

// The CTA (cx, cy, cz) of the vector kernel's grid over one volume; the caller has waited
// for the previous kernel (pdl_wait).
template <typename T, int NW, int MODE, bool SHIFT, bool RAG>
__device__ __forceinline__ void
pom_vec_cta(const T* __restrict__ vol, const FpParams& p, const uint8_t* __restrict__ lut,
            const int32_t* __restrict__ cnt, uint64_t* __restrict__ mask, void* minmax,
            uint8_t* __restrict__ occ, int tab_n, int sh, int cx, int cy, int cz)
{
    using Tr = VTraits<T>;
    constexpr int VL = Tr::VL, BL = VL / 4;
    constexpr int XW = BL * (NW + 1);                          // words a lane publishes per row
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem);       // [tab_n][NW] (not SHIFT)
    uint32_t* s_x = reinterpret_cast<uint32_t*>(smem + align16(size_t(tab_n) * NW * 4));
    // s_x: [2 buffers][2 rows (first, last)][kWarps][XW][32 lanes]
    uint4* s_rows = reinterpret_cast<uint4*>(s_x + 2 * 2 * kWarps * XW * 32);
    // s_rows: [2 slices][kWarps][5 rows][32 lanes]: the voxel rows, copied one slice ahead
    uint4* s_edge = s_rows + 2 * kWarps * 5 * 32;
    // s_edge: [2 slices][kWarps][5 rows][2]: the 16-byte vectors holding the CTA's edge
    // voxels (left of lane 0, right of lane 31), copied with the rows.  RAG (rows of any
    // length and alignment): the same space is [2 slices][kWarps][5 rows][34], the aligned
    // 16-byte vectors under the warp's row segment: slot 0 the one before lane 0's, slot
    // 1 + l lane l's, slot 33 the one after lane 31's
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (!SHIFT) {
        for (int i = tid; i < tab_n; i += kWarps * 32) {
            if (MODE == kModePom) {
                const unsigned c = lut[i];
#pragma unroll
                for (int w = 0; w < NW; ++w) s_tab[i * NW + w] = ((c >> 5) == unsigned(w)) ? (1u << (c & 31)) : 0u;
            } else {
                s_tab[i] = cnt[i + 1] > cnt[i] ? 1u : 0u;
            }
        }
        __syncthreads();
    }
    const bool want_mm = MODE == kModePom && minmax != nullptr;
    const int X = p.X, Y = p.Y;
    const unsigned nmax = unsigned(p.N - 1);
    const uint32_t nmax2 = sizeof(T) == 2 ? (min(nmax, 0xFFFFu) * 0x10001u)
                                          : (min(nmax, 0xFFu) * 0x01010101u);
    const int by = cy * kWarps + warp;
    const int xv0 = (cx * 32 + lane) * VL;                     // first voxel of the lane
    const bool lane_ok = xv0 < X;
    const int xe = lane == 0 ? cx * 32 * VL - 1 : (cx + 1) * 32 * VL;
    const bool edge_ok = (lane == 0 || lane == 31) && xe >= 0 && xe < X;
    // RAG: a lane's 16 bytes start `ra` bytes into its aligned vector (ra = the row's
    // address mod 16) and reach into the next one; voxels past the row end are replaced by
    // the row's last voxel, which changes no footprint it shares a block with
    constexpr int S = int(sizeof(T));
    constexpr int PW = Tr::PER_WORD;
    const bool tail = RAG && lane_ok && X - xv0 < VL;
    uint32_t keep[4];
    int lw = 0, lsub = 0;
    if (RAG) {
        const int nv = X - xv0;                                // valid voxels, if < VL
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            keep[k] = 0;
#pragma unroll
            for (int i = 0; i < PW; ++i)
                if (k * PW + i < nv) keep[k] |= (S == 1 ? 0xFFu : 0xFFFFu) << (8 * S * i);
        }
        lw = (nv - 1) / PW;
        lsub = (nv - 1) % PW;
    }
    const uintptr_t vaddr = reinterpret_cast<uintptr_t>(vol);
    const int zb0 = cz * p.zchunk, zb1 = min(p.gz, zb0 + p.zchunk);
    const int zs = max(0, 4 * zb0 - 1), ze = min(p.Z - 1, 4 * zb1);
    const int y0 = by * 4;
    const int yx = warp == 0 ? y0 - 1 : y0 + 4;                 // warps 0 / 7: outer apron row
    const bool has_x = warp == 0 || warp == kWarps - 1;
    const int64_t rowX = X;
    // running footprint of two block-slices: A = z >> 2, B = the next one (started at its
    // first apron slice)
    uint32_t aM[BL][NW], bM[BL][NW];
    unsigned aMn[BL], aMx[BL], bMn[BL], bMx[BL];
#pragma unroll
    for (int j = 0; j < BL; ++j) {
#pragma unroll
        for (int w = 0; w < NW; ++w) aM[j][w] = bM[j][w] = 0;
        aMn[j] = bMn[j] = 0xFFFFu;
        aMx[j] = bMx[j] = 0;
    }
    auto store_block = [&](int bz, const uint32_t (&M)[BL][NW], const unsigned (&Mn)[BL],
                           const unsigned (&Mx)[BL]) {
        if (bz < zb0 || bz >= zb1 || by >= p.gy || !lane_ok) return;
        const int64_t blk0 = (int64_t(bz) * p.gy + by) * p.gx + xv0 / 4;
        if (RAG) {                                             // blocks inside the row only
#pragma unroll
            for (int j = 0; j < BL; ++j) {
                if (xv0 / 4 + j >= p.gx) break;
                if (MODE == kModePom) {
                    mask[blk0 + j] = uint64_t(M[j][0]) |
                                     (NW > 1 ? (uint64_t(M[j][NW > 1 ? 1 : 0]) << 32) : 0ull);
                    if (want_mm) {
                        if (sizeof(T) == 1)
                            reinterpret_cast<uint16_t*>(minmax)[blk0 + j] =
                                uint16_t(Mn[j] | (Mx[j] << 8));
                        else
                            reinterpret_cast<uint32_t*>(minmax)[blk0 + j] = Mn[j] | (Mx[j] << 16);
                    }
                } else {
                    occ[blk0 + j] = uint8_t(M[j][0] != 0);
                }
            }
            return;
        }
        if (MODE == kModePom) {
            uint64_t m64[BL];
#pragma unroll
            for (int j = 0; j < BL; ++j)
                m64[j] = uint64_t(M[j][0]) | (NW > 1 ? (uint64_t(M[j][NW > 1 ? 1 : 0]) << 32) : 0ull);
            uint64_t* dst = mask + blk0;                       // one mask word per block
#pragma unroll
            for (int j = 0; j < BL; j += 2)
                *reinterpret_cast<uint4*>(dst + j) =
                    make_uint4(uint32_t(m64[j]), uint32_t(m64[j] >> 32), uint32_t(m64[j + 1]),
                               uint32_t(m64[j + 1] >> 32));
            if (want_mm) {
                if (sizeof(T) == 1) {
                    uint32_t pk[BL / 2];
#pragma unroll
                    for (int j = 0; j < BL; j += 2)
                        pk[j / 2] = (Mn[j] | (Mx[j] << 8)) | ((Mn[j + 1] | (Mx[j + 1] << 8)) << 16);
                    uint16_t* mm = reinterpret_cast<uint16_t*>(minmax) + blk0;
                    *reinterpret_cast<uint2*>(mm) = make_uint2(pk[0], pk[BL / 2 - 1]);
                } else {
                    uint32_t* mm = reinterpret_cast<uint32_t*>(minmax) + blk0;
                    *reinterpret_cast<uint2*>(mm) = make_uint2(Mn[0] | (Mx[0] << 16),
                                                               Mn[BL - 1] | (Mx[BL - 1] << 16));
                }
            }
        } else {                                               // any alignment
#pragma unroll
            for (int j = 0; j < BL; ++j) occ[blk0 + j] = uint8_t(M[j][0] != 0);
        }
    };
    // the rows of a slice: the 4 core rows and, for warps 0 / 7, the outer apron row
    auto row_y = [&](int t) { return t < 4 ? y0 + t : yx; };
    auto row_ok = [&](int t) {                                 // warp-uniform
        const int y = row_y(t);
        return (t < 4 || has_x) && y >= 0 && y < Y;
    };
    // the 16-byte vector that holds the edge voxel of lane 0 (its last voxel) or lane 31
    // (its first voxel): aligned, since rows are whole vectors
    const int xev = lane == 0 ? xe - (VL - 1) : xe;
    const int eslot = lane == 0 ? 0 : 1;
    // copies of slice z's rows (and edge vectors) into buffer `bsel`, asynchronous, one group
    auto fetch = [&](int z, int bsel) {
        const T* slice = vol + int64_t(z) * Y * rowX;
        if constexpr (RAG) {
#pragma unroll
            for (int t = 0; t < 5; ++t) {
                if (!row_ok(t)) continue;                      // warp-uniform
                const T* row = slice + int64_t(row_y(t)) * rowX;
                const int ra = int(reinterpret_cast<uintptr_t>(row) & 15);
                const unsigned char* a = reinterpret_cast<const unsigned char*>(row) + xv0 * S - ra;
                uint4* dst = s_rows + ((bsel * kWarps + warp) * 5 + t) * 34;
                // every copied vector holds a byte of the row
                if (xv0 * S - ra < X * S) cp_async16(dst + lane + 1, a);
                if (lane == 0 && cx > 0) cp_async16(dst, a - 16);
                if (lane == 31 && (xv0 + VL) * S - ra < X * S) cp_async16(dst + 33, a + 16);
            }
        } else {
#pragma unroll
            for (int t = 0; t < 5; ++t) {
                const bool ok = row_ok(t);
                const T* row = slice + int64_t(ok ? row_y(t) : 0) * rowX;
                if (ok && lane_ok) {
                    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(
                        s_rows + ((bsel * kWarps + warp) * 5 + t) * 32 + lane));
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa),
                                 "l"(row + xv0)
                                 : "memory");
                }
                if (ok && edge_ok) {
                    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(
                        s_edge + ((bsel * kWarps + warp) * 5 + t) * 2 + eslot));
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa),
                                 "l"(row + xev)
                                 : "memory");
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    fetch(zs, 0);
    for (int z = zs; z <= ze; ++z) {
        const int bsel = (z - zs) & 1;
        if (z < ze) fetch(z + 1, bsel ^ 1);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");     // this lane's copies of z
        if (RAG) __syncwarp();                                // and the neighbours' (RAG)
        const uint4* rows = s_rows + (bsel * kWarps + warp) * 5 * 32 + lane;
        const uint4* edges = s_edge + (bsel * kWarps + warp) * 5 * 2 + eslot;
        const uint4* rrow = s_rows + (bsel * kWarps + warp) * 5 * 34;      // RAG
        // RAG: the offset of row t's first byte within its aligned vector
        auto ra_of = [&](int t) {
            return int((vaddr + uint64_t((int64_t(z) * Y + row_y(t)) * rowX) * S) & 15);
        };
        // the lane's 16 bytes of row t
        auto vec_of = [&](int t) -> uint4 {
            if (!RAG) return rows[t * 32];
            const uint4 va = rrow[t * 34 + lane + 1], vb = rrow[t * 34 + lane + 2];
            const uint32_t v[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
            const int ra = ra_of(t);
            uint32_t w[5];
            switch (ra >> 2) {                                // warp-uniform
            case 0: w[0] = v[0]; w[1] = v[1]; w[2] = v[2]; w[3] = v[3]; w[4] = v[4]; break;
            case 1: w[0] = v[1]; w[1] = v[2]; w[2] = v[3]; w[3] = v[4]; w[4] = v[5]; break;
            case 2: w[0] = v[2]; w[1] = v[3]; w[2] = v[4]; w[3] = v[5]; w[4] = v[6]; break;
            default: w[0] = v[3]; w[1] = v[4]; w[2] = v[5]; w[3] = v[6]; w[4] = v[7]; break;
            }
            const unsigned sh8 = unsigned(ra & 3) * 8;
            uint32_t q[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = __funnelshift_r(w[k], w[k + 1], sh8);
            if (tail) {                                       // past the row end: the last voxel
                const uint32_t lwv = lw == 0 ? q[0] : (lw == 1 ? q[1] : (lw == 2 ? q[2] : q[3]));
                const uint32_t last = Tr::get(lwv, lsub);
                const uint32_t rep = S == 1 ? last * 0x01010101u : last * 0x00010001u;
#pragma unroll
                for (int k = 0; k < 4; ++k) q[k] = (q[k] & keep[k]) | (rep & ~keep[k]);
            }
            return make_uint4(q[0], q[1], q[2], q[3]);
        };
        // the edge voxel of row t (lanes 0 / 31), else none
        auto edge_of = [&](int t) -> unsigned {
            if (!(row_ok(t) && edge_ok)) return 0xFFFFFFFFu;
            if (RAG) {
                const uint32_t* rb = reinterpret_cast<const uint32_t*>(rrow + t * 34);
                const int ra = ra_of(t);
                const int off = lane == 0 ? 16 + ra - S : 33 * 16 + ra;
                return (rb[off >> 2] >> (8 * (off & 3))) & (S == 1 ? 0xFFu : 0xFFFFu);
            }
            const uint4 q = edges[t * 2];
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
            return lane == 0 ? VTraits<T>::get(w[3], VTraits<T>::PER_WORD - 1)
                             : VTraits<T>::get(w[0], 0);
        };
        // ---- the slice's footprint of every block of the lane, S: rows 0 and 3 (published
        //      for the warps above and below), rows 1 and 2 combined position by position
        //      first, the warp's own outer apron row, then the neighbours' rows
        uint32_t S[BL][NW];
        unsigned Smn[BL], Smx[BL];
#pragma unroll
        for (int j = 0; j < BL; ++j) {
#pragma unroll
            for (int w = 0; w < NW; ++w) S[j][w] = 0;
            Smn[j] = 0xFFFFu;
            Smx[j] = 0;
        }
        const int buf = z & 1;
        uint32_t* xf = s_x + ((buf * 2 + 0) * kWarps + warp) * XW * 32 + lane;
        uint32_t* xl = s_x + ((buf * 2 + 1) * kWarps + warp) * XW * 32 + lane;
        auto fold = [&](const uint32_t (&fp)[BL][NW], const unsigned (&fmn)[BL],
                        const unsigned (&fmx)[BL]) {
#pragma unroll
            for (int j = 0; j < BL; ++j) {
#pragma unroll
                for (int w = 0; w < NW; ++w) S[j][w] |= fp[j][w];
                Smn[j] = min(Smn[j], fmn[j]);
                Smx[j] = max(Smx[j], fmx[j]);
            }
        };
        auto publish = [&](uint32_t* dst, const uint32_t (&fp)[BL][NW], const unsigned (&fmn)[BL],
                           const unsigned (&fmx)[BL]) {
#pragma unroll
            for (int j = 0; j < BL; ++j) {
#pragma unroll
                for (int w = 0; w < NW; ++w) dst[(j * NW + w) * 32] = fp[j][w];
                dst[(BL * NW + j) * 32] = fmn[j] | (fmx[j] << 16);
            }
        };
        {
            uint32_t core[BL][NW], first[BL][NW], last[BL][NW], em[NW], wv[4], wmx[4];
            uint32_t fp[BL][NW];
            unsigned emn, emx, fmn[BL], fmx[BL];
            const unsigned sh = unsigned(p.sh);
            // one row on its own: rows 0, 3 and the apron row
            auto single = [&](int t) {
                const bool ok = row_ok(t) && lane_ok;
                lane_row<T, NW, SHIFT>(ok ? vec_of(t) : make_uint4(0u, 0u, 0u, 0u), edge_of(t), ok,
                                       nmax2, nmax, sh, s_tab, core, first, last, em, emn, emx, wv);
#pragma unroll
                for (int k = 0; k < 4; ++k) wmx[k] = ok ? wv[k] : 0u;
                lane_footprint<T, NW>(core, first, last, em, emn, emx, wv, wmx, lane, want_mm, fp,
                                      fmn, fmx);
            };
            single(0);
            publish(xf, fp, fmn, fmx);
            fold(fp, fmn, fmx);
            single(3);
            publish(xl, fp, fmn, fmx);
            fold(fp, fmn, fmx);
            if (has_x) {                                        // warp-uniform
                single(4);
                fold(fp, fmn, fmx);
            }
            // rows 1 and 2, combined position by position before the footprint
            uint32_t c12[BL][NW], f12[BL][NW], l12[BL][NW], e12[NW], mn12[4], mx12[4];
            unsigned en12, ex12;
            {
                const bool ok = row_ok(1) && lane_ok;
                lane_row<T, NW, SHIFT>(ok ? vec_of(1) : make_uint4(0u, 0u, 0u, 0u), edge_of(1), ok,
                                       nmax2, nmax, sh, s_tab, c12, f12, l12, e12, en12, ex12, mn12);
#pragma unroll
                for (int k = 0; k < 4; ++k) mx12[k] = ok ? mn12[k] : 0u;
            }
            {
                const bool ok = row_ok(2) && lane_ok;
                lane_row<T, NW, SHIFT>(ok ? vec_of(2) : make_uint4(0u, 0u, 0u, 0u), edge_of(2), ok,
                                       nmax2, nmax, sh, s_tab, core, first, last, em, emn, emx, wv);
#pragma unroll
                for (int j = 0; j < BL; ++j)
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        c12[j][w] |= core[j][w];
                        f12[j][w] |= first[j][w];
                        l12[j][w] |= last[j][w];
                    }
#pragma unroll
                for (int w = 0; w < NW; ++w) e12[w] |= em[w];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    mn12[k] = Tr::vmin(mn12[k], wv[k]);
                    mx12[k] = Tr::vmax(mx12[k], ok ? wv[k] : 0u);
                }
                en12 = min(en12, emn);
                ex12 = max(ex12, emx);
            }
            lane_footprint<T, NW>(c12, f12, l12, e12, en12, ex12, mn12, mx12, lane, want_mm, fp,
                                  fmn, fmx);
            fold(fp, fmn, fmx);
        }
        __syncthreads();
        // ---- the neighbours' rows: the last row of the warp above, the first of the one below
        if (warp > 0) {
            const uint32_t* up = s_x + ((buf * 2 + 1) * kWarps + warp - 1) * XW * 32 + lane;
#pragma unroll
            for (int j = 0; j < BL; ++j) {
#pragma unroll
                for (int w = 0; w < NW; ++w) S[j][w] |= up[(j * NW + w) * 32];
                const unsigned pa = up[(BL * NW + j) * 32];
                Smn[j] = min(Smn[j], pa & 0xFFFFu);
                Smx[j] = max(Smx[j], pa >> 16);
            }
        }
        if (warp < kWarps - 1) {
            const uint32_t* dn = s_x + ((buf * 2 + 0) * kWarps + warp + 1) * XW * 32 + lane;
#pragma unroll
            for (int j = 0; j < BL; ++j) {
#pragma unroll
                for (int w = 0; w < NW; ++w) S[j][w] |= dn[(j * NW + w) * 32];
                const unsigned pb = dn[(BL * NW + j) * 32];
                Smn[j] = min(Smn[j], pb & 0xFFFFu);
                Smx[j] = max(Smx[j], pb >> 16);
            }
        }
        // ---- z: slice z = 4 q + t belongs to block-slice q, to q - 1 when t == 0 and to
        //      q + 1 when t == 3
        const int t = z & 3, qz = z >> 2;
        if (t == 0) {
#pragma unroll
            for (int j = 0; j < BL; ++j) {
#pragma unroll
                for (int w = 0; w < NW; ++w) aM[j][w] |= S[j][w];
                aMn[j] = min(aMn[j], Smn[j]);
                aMx[j] = max(aMx[j], Smx[j]);
            }
            store_block(qz - 1, aM, aMn, aMx);
#pragma unroll
            for (int j = 0; j < BL; ++j) {
#pragma unroll
                for (int w = 0; w < NW; ++w) { aM[j][w] = bM[j][w] | S[j][w]; bM[j][w] = 0; }
                aMn[j] = min(bMn[j], Smn[j]);
                aMx[j] = max(bMx[j], Smx[j]);
                bMn[j] = 0xFFFFu;
                bMx[j] = 0;
            }
        } else {
#pragma unroll
            for (int j = 0; j < BL; ++j) {
#pragma unroll
                for (int w = 0; w < NW; ++w) aM[j][w] |= S[j][w];
                aMn[j] = min(aMn[j], Smn[j]);
                aMx[j] = max(aMx[j], Smx[j]);
                if (t == 3) {
#pragma unroll
                    for (int w = 0; w < NW; ++w) bM[j][w] = S[j][w];
                    bMn[j] = Smn[j];
                    bMx[j] = Smx[j];
                }
            }
        }
    }
    // the volume ends inside block-slice ze >> 2 (when it ends before the chunk's last apron
    // slice): that block is complete now
    if (ze < 4 * zb1) store_block(ze >> 2, aM, aMn, aMx);
}

template <typename T, int NW, int MODE, bool SHIFT, bool RAG>
__global__ void __launch_bounds__(kWarps * 32, (SHIFT && sizeof(T) == 2) ? 3 : 2)
k_pom_vec(const T* __restrict__ vol, FpParams p, const uint8_t* __restrict__ lut,
          const int32_t* __restrict__ cnt, uint64_t* __restrict__ mask, void* minmax,
          uint8_t* __restrict__ occ, int tab_n, int sh)
{
    pdl_wait();
    pom_vec_cta<T, NW, MODE, SHIFT, RAG>(vol, p, lut, cnt, mask, minmax, occ, tab_n, sh,
                                         blockIdx.x, blockIdx.y, blockIdx.z);
}

// Several volumes' POM builds in one grid: the CTAs of volume i follow those of volume
// i - 1, each volume keeping its own one-volume grid (cx fastest, then cy, cz).
struct PomBatchItem {
    const void* vol;
    FpParams p;
    const uint8_t* lut;
    uint64_t* mask;
    void* minmax;
    int tab_n;
    int gdx, gdy;                              // the volume's grid in x and y
};
struct PomBatch {
    int n;
    int start[kMaxBuildBatch + 1];             // first CTA of each volume
    PomBatchItem it[kMaxBuildBatch];
};

template <typename T, int NW, bool SHIFT, bool RAG>
__global__ void __launch_bounds__(kWarps * 32, (SHIFT && sizeof(T) == 2) ? 3 : 2)
k_pom_vec_batch(const __grid_constant__ PomBatch B)
{
    const int i = batch_item_of(B.start, B.n, int(blockIdx.x));
    const PomBatchItem& it = B.it[i];
    const int local = int(blockIdx.x) - B.start[i];
    const int cx = local % it.gdx, rest = local / it.gdx;
    pdl_wait();
    pom_vec_cta<T, NW, kModePom, SHIFT, RAG>(static_cast<const T*>(it.vol), it.p, it.lut,
                                             nullptr, it.mask, it.minmax, nullptr, it.tab_n,
                                             it.p.sh, cx, rest % it.gdy, rest / it.gdy);
}

size_t fp_smem(int N, int NW) { return align16(size_t(N)) + size_t(3) * (NW + 1) * kWarps * 32 * 4; }

template <typename T, int NW, int MODE, bool SHIFT, bool RAG>
cudaError_t launch_pom_vec(const T* v, const FpParams& p, int tab_n, const uint8_t* lut,
                           const int32_t* cnt, uint64_t* mask, void* minmax, uint8_t* occ,
                           cudaStream_t s)
{
    constexpr int VL = 16 / int(sizeof(T));
    const size_t tab_bytes = SHIFT ? 0 : align16(size_t(tab_n) * NW * 4);
    const size_t xb = size_t(2) * 2 * kWarps * (VL / 4) * (NW + 1) * 32 * 4;
    const size_t rows = size_t(2) * kWarps * 5 * (32 + 2) * 16;
    const size_t sm = tab_bytes + xb + rows;
    dim3 gv(((p.X + VL - 1) / VL + 31) / 32, (p.gy + kWarps - 1) / kWarps,
            (p.gz + p.zchunk - 1) / p.zchunk);
    cudaError_t e = ensure_dynamic_smem<k_pom_vec<T, NW, MODE, SHIFT, RAG>>(int(sm));
    if (e != cudaSuccess) return e;
    return launch_pdl(k_pom_vec<T, NW, MODE, SHIFT, RAG>, gv, dim3(kWarps * 32), sm, s, v, p, lut,
                      cnt, mask, minmax, occ, SHIFT ? 0 : tab_n, p.sh);
}

// Whether the 16-byte vector kernel takes the volume: b = 4, apron 1, at most 4 mask words
// per lane (so that the per-lane state stays in registers), and partitions by shift or a
// mask table that fits shared memory.  0: no; 1: rows of whole 16-byte vectors and an
// aligned volume; 2: other rows (the ragged-row form, RAG).
template <typename T, int NW>
int pom_vec_kind(const void* vol, const Geometry& g, int N, bool shift_ok)
{
    constexpr int VL = 16 / int(sizeof(T));
    constexpr bool kVecOk = sizeof(T) == 2 ? NW <= 2 : NW == 1;
    if (!kVecOk) return 0;
    const int tab_n = sizeof(T) == 1 ? (N < 256 ? N : 256) : N;
    const size_t tab_bytes = align16(size_t(tab_n) * NW * 4);
    if (g.b != 4 || g.a != 1 || !(shift_ok || tab_bytes <= kFpTabLimit)) return 0;
    return g.X % VL == 0 && (reinterpret_cast<uintptr_t>(vol) & 15) == 0 ? 1 : 2;
}

template <typename T, int NW, int MODE>
cudaError_t launch_fp_t(const void* vol, const Geometry& g, int N, int K, const uint8_t* lut,
                        const int32_t* cnt, uint64_t* mask, void* minmax, uint8_t* occ,
                        int shift, cudaStream_t s)
{
    FpParams p;
    p.X = g.X; p.Y = g.Y; p.Z = g.Z;
    p.gx = g.gx; p.gy = g.gy; p.gz = g.gz;
    p.b = g.b; p.a = g.a; p.N = N;
    p.W64 = (K + 63) / 64;
    p.zchunk = 4;
    p.sh = shift;
    const size_t smem = fp_smem(N, NW);
    const bool fast = g.b == 4 && ((reinterpret_cast<uintptr_t>(vol) & (4 * sizeof(T) - 1)) == 0) &&
                      ((int64_t(g.X) * sizeof(T)) % (4 * sizeof(T)) == 0) && (g.X % 4 == 0);
    dim3 grid((g.gx + 31) / 32, (g.gy + kWarps - 1) / kWarps, (g.gz + p.zchunk - 1) / p.zchunk);
    const T* v = static_cast<const T*>(vol);
    cudaError_t e;
    constexpr bool kVecOk = sizeof(T) == 2 ? NW <= 2 : NW == 1;
    if constexpr (kVecOk) {
        const int tab_n = sizeof(T) == 1 ? (N < 256 ? N : 256) : N;
        const bool shift_ok = MODE == kModePom && shift >= 0;
        const int kind = pom_vec_kind<T, NW>(vol, g, N, shift_ok);
        if (kind > 0) {
            FpParams pv = p;
            pv.zchunk = kVZChunk;
            if constexpr (MODE == kModePom) {
                if (shift_ok)
                    return kind == 1 ? launch_pom_vec<T, NW, MODE, true, false>(
                                           v, pv, tab_n, lut, cnt, mask, minmax, occ, s)
                                     : launch_pom_vec<T, NW, MODE, true, true>(
                                           v, pv, tab_n, lut, cnt, mask, minmax, occ, s);
            }
            return kind == 1 ? launch_pom_vec<T, NW, MODE, false, false>(v, pv, tab_n, lut, cnt,
                                                                          mask, minmax, occ, s)
                             : launch_pom_vec<T, NW, MODE, false, true>(v, pv, tab_n, lut, cnt,
                                                                         mask, minmax, occ, s);
        }
    }
    if (fast && g.a == 1) {
        const size_t xsm = size_t(2) * 2 * kWarps * (NW + 1) * 32 * 4;   // row exchange
        if constexpr (MODE == kModePom && NW <= 2) {
            if (size_t(N) * NW * 4 <= kFpTabLimit) {
                const size_t sm = align16(size_t(N) * NW * 4) + size_t(3) * (NW + 1) * kWarps * 32 * 4 + xsm;
                e = ensure_dynamic_smem<k_footprint41<T, NW, MODE, true>>(int(sm));
                if (e != cudaSuccess) return e;
                return launch_pdl(k_footprint41<T, NW, MODE, true>, grid, dim3(kWarps * 32), sm, s,
                                  v, p, lut, cnt, mask, minmax, occ);
            }
        }
        const size_t sm = smem + xsm;
        e = ensure_dynamic_smem<k_footprint41<T, NW, MODE, false>>(int(sm));
        if (e != cudaSuccess) return e;
        return launch_pdl(k_footprint41<T, NW, MODE, false>, grid, dim3(kWarps * 32), sm, s, v, p,
                          lut, cnt, mask, minmax, occ);
    }
    if (fast) {
        e = ensure_dynamic_smem<k_footprint<T, NW, MODE, true>>(int(smem));
        if (e != cudaSuccess) return e;
        return launch_pdl(k_footprint<T, NW, MODE, true>, grid, dim3(kWarps * 32), smem, s, v, p,
                          lut, cnt, mask, minmax, occ);
    }
    e = ensure_dynamic_smem<k_footprint<T, NW, MODE, false>>(int(smem));
    if (e != cudaSuccess) return e;
    return launch_pdl(k_footprint<T, NW, MODE, false>, grid, dim3(kWarps * 32), smem, s, v, p,
                      lut, cnt, mask, minmax, occ);
}

template <typename T>
cudaError_t launch_pom_t(const void* vol, const Geometry& g, int N, int K, const uint8_t* lut,
                         uint64_t* mask, void* minmax, int shift, cudaStream_t s)
{
    if (K <= 32)
        return launch_fp_t<T, 1, kModePom>(vol, g, N, K, lut, nullptr, mask, minmax, nullptr, shift, s);
    if (K <= 64)
        return launch_fp_t<T, 2, kModePom>(vol, g, N, K, lut, nullptr, mask, minmax, nullptr, shift, s);
    if (K <= 128)
        return launch_fp_t<T, 4, kModePom>(vol, g, N, K, lut, nullptr, mask, minmax, nullptr, shift, s);
    return launch_fp_t<T, 8, kModePom>(vol, g, N, K, lut, nullptr, mask, minmax, nullptr, shift, s);
}

}  // namespace

cudaError_t launch_partition_lut(uint8_t* lut, int N, int K, const Borders& bd, cudaStream_t s)
{
    k_partition_lut<<<(N + 255) / 256, 256, 0, s>>>(lut, N, K, bd);
    return cudaGetLastError();
}

cudaError_t launch_pom_build(const void* vol, const Geometry& g, int N, int K,
                             const uint8_t* lut, uint64_t* mask, void* minmax, int shift,
                             cudaStream_t s)
{
    if (g.bpv == 1) return launch_pom_t<uint8_t>(vol, g, N, K, lut, mask, minmax, shift, s);
    return launch_pom_t<uint16_t>(vol, g, N, K, lut, mask, minmax, shift, s);
}

namespace {

template <typename T, int NW, bool SHIFT, bool RAG>
cudaError_t launch_pom_vec_batch(const BuildItem* const* its, int m, cudaStream_t s)
{
    constexpr int VL = 16 / int(sizeof(T));
    PomBatch B;
    B.n = m;
    int64_t total = 0;
    size_t tab_bytes = 0;
    for (int k = 0; k < m; ++k) {
        const BuildItem& b = *its[k];
        PomBatchItem& it = B.it[k];
        FpParams& p = it.p;
        p.X = b.g.X; p.Y = b.g.Y; p.Z = b.g.Z;
        p.gx = b.g.gx; p.gy = b.g.gy; p.gz = b.g.gz;
        p.b = b.g.b; p.a = b.g.a; p.N = b.N;
        p.W64 = (b.K + 63) / 64;
        p.zchunk = kVZChunk;
        p.sh = b.shift;
        it.vol = b.vol;
        it.lut = b.lut;
        it.mask = b.mask;
        it.minmax = b.minmax;
        it.tab_n = SHIFT ? 0 : (sizeof(T) == 1 ? (b.N < 256 ? b.N : 256) : b.N);
        if (!SHIFT) tab_bytes = std::max(tab_bytes, align16(size_t(it.tab_n) * NW * 4));
        it.gdx = ((p.X + VL - 1) / VL + 31) / 32;
        it.gdy = (p.gy + kWarps - 1) / kWarps;
        B.start[k] = int(total);
        total += int64_t(it.gdx) * it.gdy * ((p.gz + p.zchunk - 1) / p.zchunk);
        if (total > int64_t(0x7FFFFFFF)) return cudaErrorInvalidConfiguration;
    }
    B.start[m] = int(total);
    const size_t xb = size_t(2) * 2 * kWarps * (VL / 4) * (NW + 1) * 32 * 4;
    const size_t rows = size_t(2) * kWarps * 5 * (32 + 2) * 16;
    const size_t sm = tab_bytes + xb + rows;
    cudaError_t e = ensure_dynamic_smem<k_pom_vec_batch<T, NW, SHIFT, RAG>>(int(sm));
    if (e != cudaSuccess) return e;
    return launch_pdl(k_pom_vec_batch<T, NW, SHIFT, RAG>, dim3(unsigned(total)), dim3(kWarps * 32),
                      sm, s, B);
}

// The four vector-kernel variants of one (T, mask words) slot: shift or table, whole or
// ragged rows (variant index 2 * shift + ragged).
template <typename T, int NW>
cudaError_t launch_vec_slot(const BuildItem* const (*by)[kMaxBuildBatch], const int* count,
                            cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (count[0]) e = launch_pom_vec_batch<T, NW, false, false>(by[0], count[0], s);
    if (e == cudaSuccess && count[1]) e = launch_pom_vec_batch<T, NW, false, true>(by[1], count[1], s);
    if (e == cudaSuccess && count[2]) e = launch_pom_vec_batch<T, NW, true, false>(by[2], count[2], s);
    if (e == cudaSuccess && count[3]) e = launch_pom_vec_batch<T, NW, true, true>(by[3], count[3], s);
    return e;
}

template <typename T, int NW>
cudaError_t launch_fp_batch(const BuildItem* const* its, int m, cudaStream_t s)
{
    FpBatch B;
    B.n = m;
    int64_t total = 0;
    size_t sm = 0;
    for (int k = 0; k < m; ++k) {
        const BuildItem& b = *its[k];
        FpBatchItem& it = B.it[k];
        FpParams& p = it.p;
        p.X = b.g.X; p.Y = b.g.Y; p.Z = b.g.Z;
        p.gx = b.g.gx; p.gy = b.g.gy; p.gz = b.g.gz;
        p.b = b.g.b; p.a = b.g.a; p.N = b.N;
        p.W64 = (b.K + 63) / 64;
        p.zchunk = 4;
        p.sh = b.shift;
        it.vol = b.vol;
        it.lut = b.lut;
        it.mask = b.mask;
        it.minmax = b.minmax;
        it.gdx = (p.gx + 31) / 32;
        it.gdy = (p.gy + kWarps - 1) / kWarps;
        B.start[k] = int(total);
        total += int64_t(it.gdx) * it.gdy * ((p.gz + p.zchunk - 1) / p.zchunk);
        if (total > int64_t(0x7FFFFFFF)) return cudaErrorInvalidConfiguration;
        sm = std::max(sm, fp_smem(b.N, NW));
    }
    B.start[m] = int(total);
    cudaError_t e = ensure_dynamic_smem<k_footprint_batch<T, NW>>(int(sm));
    if (e != cudaSuccess) return e;
    return launch_pdl(k_footprint_batch<T, NW>, dim3(unsigned(total)), dim3(kWarps * 32), sm, s,
                      B);
}

// The batched POM kernel of a volume.  Variants 0..11: the vector kernel, slot (uint8, 1
// mask word), (uint16, 1), (uint16, 2) times 4 + 2 * shift + ragged; 12..15: the general
// kernel (any b and apron, K <= 64) for (uint8, 1), (uint8, 2), (uint16, 1), (uint16, 2);
// -1 when neither takes the volume (K > 64), which then runs its one-volume kernel.
constexpr int kPomVariants = 16;
int pom_batch_variant(const BuildItem& b)
{
    const bool sh = b.shift >= 0;
    int slot = -1, kind = 0;
    if (b.g.bpv == 1) {
        if (b.K <= 32) { slot = 0; kind = pom_vec_kind<uint8_t, 1>(b.vol, b.g, b.N, sh); }
    } else if (b.K <= 32) {
        slot = 1; kind = pom_vec_kind<uint16_t, 1>(b.vol, b.g, b.N, sh);
    } else if (b.K <= 64) {
        slot = 2; kind = pom_vec_kind<uint16_t, 2>(b.vol, b.g, b.N, sh);
    }
    if (slot >= 0 && kind > 0) return 4 * slot + (sh ? 2 : 0) + (kind == 2 ? 1 : 0);
    if (b.K > 64) return -1;
    return 12 + (b.g.bpv == 1 ? 0 : 2) + (b.K <= 32 ? 0 : 1);
}

}  // namespace

cudaError_t launch_partition_lut_batch(const BuildItem* items, int n, cudaStream_t s)
{
    LutBatch B;
    int m = 0, used = 0, ctas = 0;
    auto flush = [&]() -> cudaError_t {
        if (m == 0) return cudaSuccess;
        B.n = m;
        B.start[m] = ctas;
        k_partition_lut_batch<<<ctas, 256, 0, s>>>(B);
        m = used = ctas = 0;
        return cudaGetLastError();
    };
    for (int i = 0; i < n; ++i) {
        const BuildItem& b = items[i];
        if (m == kMaxBuildBatch || used + b.K + 1 > kLutBorderCap) {
            cudaError_t e = flush();
            if (e != cudaSuccess) return e;
        }
        B.lut[m] = b.lut;
        B.N[m] = b.N;
        B.K[m] = b.K;
        B.boff[m] = used;
        for (int p = 0; p <= b.K; ++p) B.bv[used + p] = b.borders->v[p];
        used += b.K + 1;
        B.start[m] = ctas;
        ctas += (b.N + 255) / 256;
        ++m;
    }
    return flush();
}

cudaError_t launch_pom_build_batch(const BuildItem* items, int n, cudaStream_t s)
{
    const BuildItem* by_variant[kPomVariants][kMaxBuildBatch];
    int count[kPomVariants] = {};
    for (int i = 0; i < n && i < kMaxBuildBatch; ++i) {
        const BuildItem& b = items[i];
        const int v = pom_batch_variant(b);
        if (v < 0) {                                   // a one-volume kernel
            cudaError_t e = launch_pom_build(b.vol, b.g, b.N, b.K, b.lut, b.mask, b.minmax,
                                             b.shift, s);
            if (e != cudaSuccess) return e;
            continue;
        }
        by_variant[v][count[v]++] = &b;
    }
    cudaError_t e = launch_vec_slot<uint8_t, 1>(by_variant + 0, count + 0, s);
    if (e == cudaSuccess) e = launch_vec_slot<uint16_t, 1>(by_variant + 4, count + 4, s);
    if (e == cudaSuccess) e = launch_vec_slot<uint16_t, 2>(by_variant + 8, count + 8, s);
    if (e == cudaSuccess && count[12]) e = launch_fp_batch<uint8_t, 1>(by_variant[12], count[12], s);
    if (e == cudaSuccess && count[13]) e = launch_fp_batch<uint8_t, 2>(by_variant[13], count[13], s);
    if (e == cudaSuccess && count[14]) e = launch_fp_batch<uint16_t, 1>(by_variant[14], count[14], s);
    if (e == cudaSuccess && count[15]) e = launch_fp_batch<uint16_t, 2>(by_variant[15], count[15], s);
    return e;
}

cudaError_t launch_occ_exact(const void* vol, const Geometry& g, int N, const int32_t* cnt,
                             uint8_t* occ, cudaStream_t s)
{
    if (g.bpv == 1)
        return launch_fp_t<uint8_t, 1, kModeVis>(vol, g, N, 1, nullptr, cnt, nullptr, nullptr, occ,
                                                 -1, s);
    return launch_fp_t<uint16_t, 1, kModeVis>(vol, g, N, 1, nullptr, cnt, nullptr, nullptr, occ,
                                              -1, s);
}

}  // namespace dmk
