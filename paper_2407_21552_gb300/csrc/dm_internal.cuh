// dm_internal.cuh -- launchers shared between the C-ABI layer and the kernel files.
// Internal to libdm: nothing here is part of the public ABI in include/dm.h.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace dmk {

constexpr int kMaxPartitions = 256;
constexpr int kLineTile = 32;         // lines per y / z pass tile (one thread each)
constexpr int kLineSmemLimit = 200 * 1024;
constexpr int kXpassSmemLimit = 160 * 1024;

// Partition borders as a by-value kernel parameter: v[p] is the lowest intensity of
// partition p, v[K] = N (§3.1: integer borders rho_min^p .. rho_max^p = v[p+1]-1).
struct Borders {
    int32_t v[kMaxPartitions + 1];
};

// Volume and block-grid geometry (§3.1: non-overlapping b^3 blocks; footprint adds an
// apron of `a` voxels per side, clipped at the volume).
struct Geometry {
    int32_t X, Y, Z;        // voxels
    int32_t gx, gy, gz;     // blocks: ceil(dim / b)
    int32_t b, a;           // block edge, apron
    int32_t bpv;            // bytes per voxel: 1 or 2
    int64_t G;              // gx * gy * gz
    int64_t plane;          // bytes between PDM planes (G rounded up to 64)
};

// Programmatic dependent launch (PDL).  A kernel launched with the programmatic stream
// serialization attribute may start while the previous kernel in the stream still runs;
// pdl_wait() blocks until that kernel has finished and its writes are visible, and must
// precede every access to memory the previous kernel touches.  pdl_trigger() lets the
// next kernel's CTAs launch early.  Both are no-ops for a kernel launched normally.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch `kern` on `s` with the PDL attribute set.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the current device,
// calling cudaFuncSetAttribute only when the limit set so far is lower.
template <auto Kern>
cudaError_t ensure_dynamic_smem(int bytes)
{
    static std::atomic<int> set_to[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && set_to[dev].load(std::memory_order_relaxed) >= bytes)
        return cudaSuccess;
    e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && dev >= 0 && dev < 64) {
        int cur = set_to[dev].load(std::memory_order_relaxed);
        while (cur < bytes && !set_to[dev].compare_exchange_weak(cur, bytes)) {
        }
    }
    return e;
}

// ---------------------------------------------------------------- byte-wise minimum
// The PDM combine folds bytes with min.u16x2: every 32-bit word of a running minimum is
// kept as its even bytes (w & 0x00FF00FF) and its odd bytes (w & 0xFF00FF00) in two
// registers.  A byte in one half of a 16-bit lane whose other half is zero orders like the
// byte itself, so one 16x2 min folds two bytes; splitting a loaded word costs two logic
// operations, and the halves are OR-ed back together once per output word.
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ uint32_t max_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// Byte minimum of 16 bytes.
__device__ __forceinline__ unsigned bytemin16(const uint4& v)
{
    const unsigned w = __vminu4(__vminu4(v.x, v.y), __vminu4(v.z, v.w));
    return min(min(w & 0xFFu, (w >> 8) & 0xFFu), min((w >> 16) & 0xFFu, w >> 24));
}

struct ByteMin16 {                                   // running byte minimum of 16 bytes
    uint32_t e[4], o[4];
    __device__ __forceinline__ void reset()
    {
#pragma unroll
        for (int k = 0; k < 4; ++k) { e[k] = 0x00FF00FFu; o[k] = 0xFF00FF00u; }
    }
    __device__ __forceinline__ void fold(const uint4& v)
    {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            e[k] = min_u16x2(e[k], w[k] & 0x00FF00FFu);
            o[k] = min_u16x2(o[k], w[k] & 0xFF00FF00u);
        }
    }
    __device__ __forceinline__ uint4 value() const
    {
        return make_uint4(e[0] | o[0], e[1] | o[1], e[2] | o[2], e[3] | o[3]);
    }
    // some byte above 0: a minimum that reached 0 everywhere no plane can lower
    __device__ __forceinline__ bool nonzero() const
    {
        return ((e[0] | e[1] | e[2] | e[3]) | (o[0] | o[1] | o[2] | o[3])) != 0u;
    }
    // the largest of the 16 minima
    __device__ __forceinline__ uint32_t max_byte() const
    {
        const uint32_t a = max_u16x2(max_u16x2(e[0], e[1]), max_u16x2(e[2], e[3]));
        const uint32_t b = max_u16x2(max_u16x2(o[0], o[1]), max_u16x2(o[2], o[3])) >> 8;
        const uint32_t c = max_u16x2(a, b & 0x00FF00FFu);
        return max(c & 0xFFFFu, c >> 16);
    }
};

// Regions of the combine's bound (Eq. 1 read region by region): kRegionBlocks consecutive
// blocks of a map, 256 chunks of 16 bytes, one warp's 8 chunks per lane.
constexpr int64_t kRegionBlocks = 4096;
constexpr int kRegionChunks = 256;
__host__ __device__ inline int64_t num_regions(int64_t G)
{
    return (G + kRegionBlocks - 1) / kRegionBlocks;
}

// Adds a warp's sum of v to *count (one atomic, lane 0).  Every lane of the warp must call
// it at the same point (the update kernels do so at their end).
__device__ __forceinline__ void add_warp_count(unsigned long long* count, unsigned long long v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
    if ((threadIdx.x & 31) == 0) atomicAdd(count, v);
}

// ---------------------------------------------------------------- partition-range index
// Optional sparse index over the K PDMs: plane (k, i) = min of PDM_i .. PDM_{i + 2^k - 1}
// for k = 0..J (level 0 = the PDMs), J = floor(log2 K).  Level k starts at plane
// index_level_base(K, k).  A run of consecutive active partitions [i, e] is covered by the
// two planes (k, i) and (k, e - 2^k + 1) with k = floor(log2(e - i + 1)).
__host__ __device__ inline int index_level_base(int K, int k)
{
    int b = 0;
    for (int l = 0; l < k; ++l) b += K - (1 << l) + 1;
    return b;
}
__host__ __device__ inline int index_levels(int K)
{
    int J = 0;
    while ((2 << J) <= K) ++J;
    return J;
}

// From the active-partition bit set `bits` (shared memory, 8 words, bit p = partition p),
// write the plane indices to combine to `list` and return their number (to every thread).
// Without the index (J < 0) the planes are the active partitions, listed in the order in
// which thread t < K passes them as `mine` (a permutation of 0..K-1: the context's plane
// order, or t itself); with it, one or two planes per maximal run of active partitions,
// threads 0..255 handling partition threadIdx.x.  Every thread of the CTA must call it (it
// synchronises the CTA); `s_scan` is 9 ints of shared scratch.
__device__ inline int plan_maps(const uint32_t* bits, int K, int J, uint16_t* list, int* s_scan,
                                int mine)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto on = [&](int p) { return (bits[p >> 5] >> (p & 31)) & 1u; };
    int c = 0;
    int m0 = 0, m1 = 0;
    if (J < 0) {                                          // the planes, in the given order
        if (tid < K && on(mine)) {
            c = 1;
            m0 = mine;
        }
    } else if (tid < K && on(tid)) {
        if (tid == 0 || !on(tid - 1)) {                   // run start: find the run's end
            int e = tid;
            while (e + 1 < K && on(e + 1)) ++e;
            const int k = 31 - __clz(e - tid + 1);
            const int base = index_level_base(K, k);
            m0 = base + tid;
            m1 = base + e - (1 << k) + 1;
            c = m1 == m0 ? 1 : 2;
        }
    }
    int incl = c;                                         // scan over threads 0..255
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31 && warp < 8) s_scan[warp] = incl;
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int w = 0; w < 8; ++w) {
            const int t = s_scan[w];
            s_scan[w] = run;
            run += t;
        }
        s_scan[8] = run;
    }
    __syncthreads();
    if (tid < 256 && c) {
        const int pos = s_scan[warp] + incl - c;
        list[pos] = uint16_t(m0);
        if (c == 2) list[pos + 1] = uint16_t(m1);
    }
    __syncthreads();
    return s_scan[8];
}

// ---------------------------------------------------------------- one-time precompute
cudaError_t launch_partition_lut(uint8_t* lut, int N, int K, const Borders& bd,
                                 cudaStream_t s);

// POM bit masks [G][W] (+ block footprint min/max pairs when minmax != nullptr).
// shift >= 0: the partitions are uniform with 2^shift intensities each (partition of
// intensity i = i >> shift), which the kernels may use instead of the table; else -1.
cudaError_t launch_pom_build(const void* vol, const Geometry& g, int N, int K,
                             const uint8_t* lut, uint64_t* mask, void* minmax, int shift,
                             cudaStream_t s);

// Exact TF occupancy per block (1 byte, 0/1) from a per-voxel visibility test over the
// footprint; visibility of intensity i is cnt[i+1] > cnt[i].
cudaError_t launch_occ_exact(const void* vol, const Geometry& g, int N, const int32_t* cnt,
                             uint8_t* occ, cudaStream_t s);

// ---------------------------------------------------------------- distance transform
// x pass: 1D distance along x to the nearest occupied block, saturating at 255.
// proj (optional): where the one-row-per-CTA form runs, it also writes each row's mask words
// ORed along x to proj[row][W] and sets *projected.
cudaError_t launch_xpass_mask(const uint64_t* mask, int K, const Geometry& g, uint8_t* pdm,
                              cudaStream_t s, uint64_t* proj = nullptr,
                              bool* projected = nullptr);
cudaError_t launch_xpass_minmax(const void* minmax, const int32_t* cnt, const Geometry& g,
                                uint8_t* out, cudaStream_t s);
cudaError_t launch_xpass_occ(uint8_t* occ_inout, const Geometry& g, cudaStream_t s);

// y (axis 1) or z (axis 2) pass in place over P maps at `plane` bytes apart:
// h(i) = min over j of max(|i - j|, g(j)), saturating at 255.
cudaError_t launch_line_pass(uint8_t* buf, int P, int64_t plane, const Geometry& g, int axis,
                             cudaStream_t s);
size_t line_pass_smem(int L);

// Index levels 1..J over the K PDM planes (level 0), each level one streaming min pass.
cudaError_t launch_build_index(uint8_t* pdm, int64_t plane, int64_t G, int K, cudaStream_t s);
size_t xpass_smem(int gx, int K);

// ---------------------------------------------------------------- per-TF update
// Visibility prefix count cnt[0..N] (cnt[i] = #{j < i : alpha_j > 0}), active set S as a
// bit set smask[4] and as an ascending list act[0..*nact).  smask_out may be null.
cudaError_t launch_tf_active(const float* tf, int N, int K, const Borders& bd, int32_t* cnt,
                             uint16_t* act, int32_t* nact, uint64_t* smask,
                             uint64_t* smask_out, cudaStream_t s);

// The active set alone (no prefix count), for the update path; without the index (J < 0)
// act lists the active planes in the plane order `order` (null: ascending).
cudaError_t launch_active_set(const float* tf, int N, int K, int J, const Borders& bd,
                              const uint16_t* order, uint16_t* act, int32_t* nact,
                              uint64_t* smask, uint64_t* smask_out, cudaStream_t s);

// Step 1 and Eq. 1 in one launch: each CTA derives S from the TF itself (N <= 8192).
bool update_fused_ok(int N);
// `uniform`: the borders are the default floor(p N / K), which the kernel computes instead of
// indexing the parameter array per thread.  `order` as in launch_active_set; `rmin`: the
// context's region bounds [regions(G)][K] (null: none), which the plain path (J < 0) reads
// region by region.  `count`: a device counter to which the kernel adds the bytes of PDM
// planes it loads (null: none).
cudaError_t launch_update_fused(const uint8_t* pdm, int64_t plane, int64_t G, const float* tf,
                                int N, int K, int J, const Borders& bd, int uniform,
                                const uint16_t* order, const uint8_t* rmin, uint16_t* act,
                                int32_t* nact, uint64_t* smask, uint64_t* smask_out,
                                uint8_t* out, int num_sms, unsigned long long* count,
                                cudaStream_t s);

// D' = byte-wise min over the active planes (Eq. 1); 255 when S is empty.  `count` as in
// launch_update_fused.
cudaError_t launch_combine(const uint8_t* pdm, int64_t plane, int64_t G, const uint16_t* act,
                           const int32_t* nact, uint8_t* out, int num_sms,
                           unsigned long long* count, cudaStream_t s);

// ---------------------------------------------------------------- batched update
constexpr int kMaxBatch = 64;          // groups per launch pair (descriptors as parameters)
constexpr int kMaxGroupEdits = 8;      // TFs of one volume that share their plane reads

// One volume and up to kMaxGroupEdits TFs for it.  list / emask / count: where the
// active-set kernel leaves the group's planes (batch_list_entries(planes) entries each; for
// E == 1 emask is not used).
struct BatchGroup {
    const uint8_t* pdm;
    int64_t plane, G;
    const uint8_t* lut;                // the volume's partition table (its scratch)
    const uint16_t* order;             // the volume's plane order (its scratch; null: ascending)
    uint16_t* list;
    uint8_t* emask;
    int32_t* count;
    int32_t N, K;
    int32_t J;                         // index levels (-1: no index)
    int32_t E;
    const float* tf[kMaxGroupEdits];
    uint8_t* out[kMaxGroupEdits];
};

struct BatchTuning {
    int ctas_per_sm;                   // combine grid: CTAs per SM (<= 0: 24)
    int loads_per_stage;               // plane loads per pipeline stage: 4 (default) or 8
};

// Entries of a group's plane list, padding included, for a buffer of `planes` planes.
size_t batch_list_entries(int planes);

// Active sets of up to kMaxBatch groups (one CTA each), then one combine over all their
// work units (PDL).  `count`: a device counter to which the combine adds the bytes of PDM
// planes it loads (null: none).
cudaError_t launch_update_batch(const BatchGroup* groups, int n, const BatchTuning& tune,
                                int num_sms, unsigned long long* count, cudaStream_t s);

}  // namespace dmk
