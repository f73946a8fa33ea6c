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
// Tiling: a CTA owns tbx x tby blocks of one block-slice bz and walks the b + 2a voxel
// slices of their z-footprint.  Each slice's voxel tile (with its x/y apron) is staged in
// shared memory with 16-byte vector loads where rows are aligned; a row pass ORs the
// classes over each block's x-footprint, then a column pass ORs those over the block's
// y-footprint into per-block accumulators that live in shared memory across slices.
#include "dm_internal.cuh"

namespace dmk {
namespace {

constexpr int kThreads = 256;

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

struct FpParams {
    Geometry g;
    int N;
    int tbx, tby;          // blocks per tile in x / y
    int ap;                // tile columns left of the core (>= a, 16-byte aligned)
    int tile_w, tile_h;    // voxel tile extent
    int vec_ok;            // core rows can use 16-byte loads
};

enum { kModePom = 0, kModeVis = 1 };

template <typename T>
struct MinMaxPack;
template <>
struct MinMaxPack<uint8_t> {
    using P = uint16_t;
    __device__ static P pack(unsigned mn, unsigned mx) { return P(mn | (mx << 8)); }
};
template <>
struct MinMaxPack<uint16_t> {
    using P = uint32_t;
    __device__ static P pack(unsigned mn, unsigned mx) { return P(mn | (mx << 16)); }
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

struct FpSmem {
    size_t cls, tile, rowacc, rowmm, blkacc, blkmm, total;
};

__host__ __device__ inline FpSmem fp_smem_layout(int N, int W, int bpv, int tile_w, int tile_h,
                                                 int tbx, int tby)
{
    FpSmem s;
    size_t o = 0;
    s.cls = o;    o = align16(o + size_t(N));
    s.tile = o;   o = align16(o + size_t(tile_w) * tile_h * bpv);
    s.rowacc = o; o = align16(o + size_t(tile_h) * tbx * W * 8);
    s.rowmm = o;  o = align16(o + size_t(tile_h) * tbx * 4);
    s.blkacc = o; o = align16(o + size_t(tby) * tbx * W * 8);
    s.blkmm = o;  o = align16(o + size_t(tby) * tbx * 4);
    s.total = o;
    return s;
}

template <typename T, int W, int MODE>
__global__ void __launch_bounds__(kThreads)
k_footprint(const T* __restrict__ vol, FpParams prm, const uint8_t* __restrict__ lut,
            const int32_t* __restrict__ cnt, uint64_t* __restrict__ mask, void* minmax,
            uint8_t* __restrict__ occ)
{
    extern __shared__ __align__(16) unsigned char smem[];
    pdl_wait();
    const Geometry& g = prm.g;
    const int tid = threadIdx.x;
    const int tbx = prm.tbx, tby = prm.tby, tw = prm.tile_w, th = prm.tile_h;
    const FpSmem L = fp_smem_layout(prm.N, W, int(sizeof(T)), tw, th, tbx, tby);
    uint8_t* s_cls = smem + L.cls;
    T* s_tile = reinterpret_cast<T*>(smem + L.tile);
    uint64_t* s_row = reinterpret_cast<uint64_t*>(smem + L.rowacc);
    uint16_t* s_rowmm = reinterpret_cast<uint16_t*>(smem + L.rowmm);   // [th*tbx][2]
    uint64_t* s_blk = reinterpret_cast<uint64_t*>(smem + L.blkacc);
    uint16_t* s_blkmm = reinterpret_cast<uint16_t*>(smem + L.blkmm);   // [tby*tbx][2]

    const int bx0 = blockIdx.x * tbx, by0 = blockIdx.y * tby, bz = blockIdx.z;
    const int b = g.b, a = g.a, N = prm.N;

    // class table: partition index (POM) or visibility bit (exact occupancy)
    for (int i = tid; i < N; i += kThreads) {
        if (MODE == kModePom) s_cls[i] = lut[i];
        else s_cls[i] = uint8_t(cnt[i + 1] > cnt[i]);
    }
    for (int i = tid; i < tby * tbx; i += kThreads) {
        for (int w = 0; w < W; ++w) s_blk[i * W + w] = 0;
        s_blkmm[2 * i] = 0xFFFF;
        s_blkmm[2 * i + 1] = 0;
    }

    // voxel tile origin: column c <-> x = bx0*b - ap + c, row r <-> y = by0*b - a + r
    const int xo = bx0 * b - prm.ap;
    const int yo = by0 * b - a;
    const int xlo = max(0, bx0 * b - a), xhi = min(g.X - 1, (bx0 + tbx) * b - 1 + a);
    const int ylo = max(0, yo), yhi = min(g.Y - 1, (by0 + tby) * b - 1 + a);
    const int zlo = max(0, bz * b - a), zhi = min(g.Z - 1, bz * b + b - 1 + a);
    const int nrows = yhi - ylo + 1;
    const int64_t rowstride = g.X;
    const int64_t slicestride = int64_t(g.X) * g.Y;

    for (int z = zlo; z <= zhi; ++z) {
        __syncthreads();   // the previous slice's tile and row accumulators are consumed
        const T* sl = vol + int64_t(z) * slicestride;
        // ---- stage the slice tile
        if (prm.vec_ok) {
            // core columns [bx0*b, (bx0+tbx)*b) with 16-byte loads, apron columns scalar
            const int per_row = (tbx * b * int(sizeof(T))) / 16;
            const int nvec = nrows * per_row;
            for (int i = tid; i < nvec; i += kThreads) {
                int r = i / per_row, q = i - r * per_row;
                int y = ylo + r;
                const uint4* src = reinterpret_cast<const uint4*>(sl + int64_t(y) * rowstride
                                                                  + int64_t(bx0) * b) + q;
                uint4 v = __ldg(src);
                T* dst = s_tile + (y - yo) * tw + prm.ap;
                reinterpret_cast<uint4*>(dst)[q] = v;
            }
            const int na = 2 * a;
            for (int i = tid; i < nrows * na; i += kThreads) {
                int r = i / na, k = i - r * na;
                int y = ylo + r;
                int x = k < a ? bx0 * b - a + k : (bx0 + tbx) * b + (k - a);
                if (x >= 0 && x < g.X)
                    s_tile[(y - yo) * tw + (x - xo)] = sl[int64_t(y) * rowstride + x];
            }
        } else {
            const int ncols = xhi - xlo + 1;
            for (int i = tid; i < nrows * ncols; i += kThreads) {
                int r = i / ncols, c = i - r * ncols;
                int y = ylo + r, x = xlo + c;
                s_tile[(y - yo) * tw + (x - xo)] = sl[int64_t(y) * rowstride + x];
            }
        }
        __syncthreads();
        // ---- row pass: per (tile row, block column) OR over the block's x-footprint
        for (int i = tid; i < nrows * tbx; i += kThreads) {
            int r = i / tbx, bxl = i - r * tbx;
            int y = ylo + r;
            int bx = bx0 + bxl;
            uint64_t acc[W];
#pragma unroll
            for (int w = 0; w < W; ++w) acc[w] = 0;
            unsigned mn = 0xFFFF, mx = 0;
            if (bx < g.gx) {
                int x0 = max(0, bx * b - a), x1 = min(g.X - 1, bx * b + b - 1 + a);
                const T* row = s_tile + (y - yo) * tw - xo;
                for (int x = x0; x <= x1; ++x) {
                    unsigned v = row[x];
                    if (v > unsigned(N - 1)) v = unsigned(N - 1);
                    unsigned c = s_cls[v];
                    if (MODE == kModePom) {
#pragma unroll
                        for (int w = 0; w < W; ++w)
                            acc[w] |= ((c >> 6) == unsigned(w)) ? (uint64_t(1) << (c & 63)) : 0;
                        mn = min(mn, v);
                        mx = max(mx, v);
                    } else {
                        acc[0] |= c;
                    }
                }
            }
            int ri = (y - yo) * tbx + bxl;
#pragma unroll
            for (int w = 0; w < W; ++w) s_row[ri * W + w] = acc[w];
            s_rowmm[2 * ri] = uint16_t(mn);
            s_rowmm[2 * ri + 1] = uint16_t(mx);
        }
        __syncthreads();
        // ---- column pass: per block OR over its y-footprint rows of this slice
        for (int i = tid; i < tby * tbx; i += kThreads) {
            int byl = i / tbx, bxl = i - byl * tbx;
            int by = by0 + byl, bx = bx0 + bxl;
            if (by >= g.gy || bx >= g.gx) continue;
            int y0 = max(0, by * b - a), y1 = min(g.Y - 1, by * b + b - 1 + a);
            uint64_t acc[W];
#pragma unroll
            for (int w = 0; w < W; ++w) acc[w] = s_blk[i * W + w];
            unsigned mn = s_blkmm[2 * i], mx = s_blkmm[2 * i + 1];
            for (int y = y0; y <= y1; ++y) {
                int ri = (y - yo) * tbx + bxl;
#pragma unroll
                for (int w = 0; w < W; ++w) acc[w] |= s_row[ri * W + w];
                mn = min(mn, unsigned(s_rowmm[2 * ri]));
                mx = max(mx, unsigned(s_rowmm[2 * ri + 1]));
            }
#pragma unroll
            for (int w = 0; w < W; ++w) s_blk[i * W + w] = acc[w];
            s_blkmm[2 * i] = uint16_t(mn);
            s_blkmm[2 * i + 1] = uint16_t(mx);
        }
    }
    __syncthreads();
    // ---- write the tile's blocks
    for (int i = tid; i < tby * tbx; i += kThreads) {
        int byl = i / tbx, bxl = i - byl * tbx;
        int by = by0 + byl, bx = bx0 + bxl;
        if (by >= g.gy || bx >= g.gx) continue;
        int64_t blk = (int64_t(bz) * g.gy + by) * g.gx + bx;
        if (MODE == kModePom) {
#pragma unroll
            for (int w = 0; w < W; ++w) mask[blk * W + w] = s_blk[i * W + w];
            if (minmax) {
                using P = typename MinMaxPack<T>::P;
                reinterpret_cast<P*>(minmax)[blk] =
                    MinMaxPack<T>::pack(s_blkmm[2 * i], s_blkmm[2 * i + 1]);
            }
        } else {
            occ[blk] = uint8_t(s_blk[i * W] != 0);
        }
    }
}

// Pick the tile so that shared memory stays under `limit`; voxel extent starts at 128 x 32.
bool plan_tiles(const Geometry& g, int N, int W, size_t limit, FpParams* p, size_t* smem)
{
    int b = g.b, a = g.a, s = g.bpv;
    int vx = 128, vy = 32;
    for (int attempt = 0; attempt < 8; ++attempt) {
        int tbx = max(1, vx / b), tby = max(1, vy / b);
        int ap = max(16 / s, ((a + 16 / s - 1) / (16 / s)) * (16 / s));
        int tw = ap + tbx * b + ap;
        int th = tby * b + 2 * a;
        FpSmem L = fp_smem_layout(N, W, s, tw, th, tbx, tby);
        if (L.total <= limit) {
            p->g = g;
            p->N = N;
            p->tbx = tbx;
            p->tby = tby;
            p->ap = ap;
            p->tile_w = tw;
            p->tile_h = th;
            *smem = L.total;
            return true;
        }
        if (vx > 16) vx /= 2; else if (vy > 4) vy /= 2; else break;
    }
    return false;
}

template <typename T, int W, int MODE>
cudaError_t launch_fp_t(const void* vol, const Geometry& g, int N, const uint8_t* lut,
                        const int32_t* cnt, uint64_t* mask, void* minmax, uint8_t* occ,
                        size_t limit, cudaStream_t s)
{
    FpParams p;
    size_t smem = 0;
    if (!plan_tiles(g, N, W, limit, &p, &smem)) return cudaErrorInvalidConfiguration;
    const int sz = int(sizeof(T));
    p.vec_ok = ((reinterpret_cast<uintptr_t>(vol) & 15) == 0) &&
               ((int64_t(g.X) * sz) % 16 == 0) && ((p.tbx * g.b * sz) % 16 == 0) &&
               (int64_t(g.gx) % p.tbx == 0) && (int64_t(g.gx) * g.b == g.X);
    cudaError_t e = ensure_dynamic_smem<k_footprint<T, W, MODE>>(int(smem));
    if (e != cudaSuccess) return e;
    dim3 grid((g.gx + p.tbx - 1) / p.tbx, (g.gy + p.tby - 1) / p.tby, g.gz);
    return launch_pdl(k_footprint<T, W, MODE>, grid, dim3(kThreads), smem, s,
                      static_cast<const T*>(vol), p, lut, cnt, mask, minmax, occ);
}

template <typename T>
cudaError_t launch_pom_t(const void* vol, const Geometry& g, int N, int K, const uint8_t* lut,
                         uint64_t* mask, void* minmax, size_t limit, cudaStream_t s)
{
    int W = (K + 63) / 64;
    switch (W) {
    case 1: return launch_fp_t<T, 1, kModePom>(vol, g, N, lut, nullptr, mask, minmax, nullptr, limit, s);
    case 2: return launch_fp_t<T, 2, kModePom>(vol, g, N, lut, nullptr, mask, minmax, nullptr, limit, s);
    case 3: return launch_fp_t<T, 3, kModePom>(vol, g, N, lut, nullptr, mask, minmax, nullptr, limit, s);
    case 4: return launch_fp_t<T, 4, kModePom>(vol, g, N, lut, nullptr, mask, minmax, nullptr, limit, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_partition_lut(uint8_t* lut, int N, int K, const Borders& bd, cudaStream_t s)
{
    k_partition_lut<<<(N + 255) / 256, 256, 0, s>>>(lut, N, K, bd);
    return cudaGetLastError();
}

cudaError_t launch_pom_build(const void* vol, const Geometry& g, int N, int K,
                             const uint8_t* lut, uint64_t* mask, void* minmax,
                             size_t smem_limit, cudaStream_t s)
{
    if (g.bpv == 1) return launch_pom_t<uint8_t>(vol, g, N, K, lut, mask, minmax, smem_limit, s);
    return launch_pom_t<uint16_t>(vol, g, N, K, lut, mask, minmax, smem_limit, s);
}

cudaError_t launch_occ_exact(const void* vol, const Geometry& g, int N, const int32_t* cnt,
                             uint8_t* occ, size_t smem_limit, cudaStream_t s)
{
    if (g.bpv == 1)
        return launch_fp_t<uint8_t, 1, kModeVis>(vol, g, N, nullptr, cnt, nullptr, nullptr, occ,
                                                 smem_limit, s);
    return launch_fp_t<uint16_t, 1, kModeVis>(vol, g, N, nullptr, cnt, nullptr, nullptr, occ,
                                              smem_limit, s);
}

}  // namespace dmk
