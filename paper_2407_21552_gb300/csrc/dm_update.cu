// dm_update.cu -- the per-TF update: active partitions from the TF, then the combine.
//
// §3.1 step 1: S = partitions holding at least one intensity whose TF alpha is non-zero.
// One CTA turns the N alphas into a visibility prefix count cnt[0..N] (also what the plain
// min/max recompute needs), then partition p is active iff cnt[hi_p + 1] > cnt[lo_p]; the
// active indices are compacted in ascending order with warp ballots.  S never leaves the
// device.
//
// §3.1 step 2, Eq. 1: D'(x,y,z) = min over p in S of PDM_p(x,y,z).  A pure streaming
// kernel: each thread owns 16-byte chunks of the map, reads the same chunk of every active
// plane (independent 16-byte loads, several in flight) and folds them byte-wise, two bytes
// per min.u16x2 (ByteMin16).  On large maps the chunks are taken in plane-major tiles: a
// warp reads 4 KiB of one plane per step and keeps 8 accumulators per thread.  An empty S
// yields 255.
//
// A byte minimum of 0 is final, so a chunk stops loading planes once its minimum is 0 in
// every byte, and the active planes are read in the context's plane order: most-covered
// (most zero bytes on a sample) first, which brings most chunks to 0 soonest.  The HBM
// traffic is at most (|S| + 1) * G bytes; D' is the same in any order.
#include "dm_build_batch.cuh"
#include "dm_internal.cuh"

namespace dmk {
namespace {

constexpr int kActThreads = 1024;
constexpr int DM_MAX_TF_WORDS = 65536 / 32;
constexpr int kCombineThreads = 256;

__global__ void __launch_bounds__(kActThreads)
k_tf_active(const float* __restrict__ tf, int N, int K, Borders bd, int32_t* __restrict__ cnt,
            uint16_t* __restrict__ act, int32_t* __restrict__ nact, uint64_t* __restrict__ smask,
            uint64_t* __restrict__ smask_out)
{
    __shared__ int32_t s_warp[32];
    __shared__ int32_t s_actw[8];
    __shared__ uint32_t s_bits[8];
    pdl_trigger();     // the next kernel's CTAs may launch; they wait for this grid
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // contiguous chunk of intensities per thread; visibility kept as bits (chunk <= 64)
    const int per = (N + kActThreads - 1) / kActThreads;
    const int i0 = min(N, tid * per), i1 = min(N, i0 + per);
    uint64_t vbits = 0;
#pragma unroll 8
    for (int i = i0; i < i1; ++i)
        vbits |= uint64_t(__ldg(tf + 4 * int64_t(i) + 3) > 0.0f) << (i - i0);
    const int c = __popcll(vbits);
    // block exclusive scan of c
    int incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = s_warp[lane];
        int wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int v = __shfl_up_sync(0xFFFFFFFFu, wi, d);
            if (lane >= d) wi += v;
        }
        s_warp[lane] = wi - w;                 // exclusive warp offsets
    }
    __syncthreads();
    int run = s_warp[warp] + incl - c;
    for (int i = i0; i < i1; ++i) {
        cnt[i] = run;
        run += int((vbits >> (i - i0)) & 1u);
    }
    if (i1 == N && i0 < i1) cnt[N] = run;   // the thread holding intensity N-1
    __syncthreads();                          // cnt is visible to the whole block
    // active partitions, ascending, compacted with ballots (K <= 256 -> warps 0..7)
    const int p = tid;
    const bool on = (p < K) && (cnt[bd.v[p + 1]] > cnt[bd.v[p]]);
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, on);
    if (lane == 0 && warp < 8) {
        s_actw[warp] = __popc(bal);
        s_bits[warp] = bal;
    }
    __syncthreads();
    if (tid < 256) {
        int off = 0;
        for (int w = 0; w < warp; ++w) off += s_actw[w];
        if (on) act[off + __popc(bal & ((1u << lane) - 1))] = uint16_t(p);
        if (tid == 0) {
            int tot = 0;
            for (int w = 0; w < 8; ++w) tot += s_actw[w];
            *nact = tot;
        }
        if (tid < 4) {
            uint64_t v = uint64_t(s_bits[2 * tid]) | (uint64_t(s_bits[2 * tid + 1]) << 32);
            smask[tid] = v;
            if (smask_out && tid < (K + 63) / 64) smask_out[tid] = v;
        }
    }
}

// Step 1 of §3.1 for the update path: visibility bits from warp ballots (all loads of a
// batch issued before any is used), then partition p is active iff a visibility bit in
// [lo_p, hi_p] is set; compacted ascending.  Lets the combine's CTAs launch at once.
__global__ void __launch_bounds__(kActThreads)
k_active_set(const float* __restrict__ tf, int N, int K, int J, Borders bd,
             const uint16_t* __restrict__ order, uint16_t* __restrict__ act,
             int32_t* __restrict__ nact, uint64_t* __restrict__ smask,
             uint64_t* __restrict__ smask_out)
{
    pdl_trigger();
    constexpr int kBatch = 8;
    __shared__ uint32_t s_vis[DM_MAX_TF_WORDS];
    __shared__ uint32_t s_bits[8];
    __shared__ uint16_t s_list[kMaxPartitions + 8];
    __shared__ int s_scan[9];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mine = order && tid < K ? int(order[tid]) : tid;     // this thread's plane
    for (int base = 0; base < N; base += kActThreads * kBatch) {
        float a[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int i = base + k * kActThreads + tid;
            a[k] = i < N ? __ldg(tf + 4 * int64_t(i) + 3) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int i0 = base + k * kActThreads;          // uniform over the block
            if (i0 < N) {
                const unsigned bal = __ballot_sync(0xFFFFFFFFu, a[k] > 0.0f);
                if (lane == 0 && i0 + warp * 32 < N) s_vis[(i0 >> 5) + warp] = bal;
            }
        }
    }
    __syncthreads();
    bool on = false;
    const int p = tid;
    if (p < K) {
        const int lo = bd.v[p], hi = bd.v[p + 1] - 1;
        for (int w = lo >> 5; w <= (hi >> 5) && !on; ++w) {
            uint32_t m = s_vis[w];
            if (w == (lo >> 5)) m &= 0xFFFFFFFFu << (lo & 31);
            if (w == (hi >> 5)) m &= 0xFFFFFFFFu >> (31 - (hi & 31));
            on = m != 0;
        }
    }
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, on);
    if (lane == 0 && warp < 8) s_bits[warp] = bal;
    __syncthreads();
    const int n = plan_maps(s_bits, K, J, s_list, s_scan, mine);
    for (int j = tid; j < n; j += kActThreads) act[j] = s_list[j];
    if (tid == 0) *nact = n;
    if (tid < 4) {
        const uint64_t v = uint64_t(s_bits[2 * tid]) | (uint64_t(s_bits[2 * tid + 1]) << 32);
        smask[tid] = v;
        if (smask_out && tid < (K + 63) / 64) smask_out[tid] = v;
    }
}

__device__ __forceinline__ uint4 vmin4(uint4 a, uint4 b)
{
    return make_uint4(__vminu4(a.x, b.x), __vminu4(a.y, b.y), __vminu4(a.z, b.z),
                      __vminu4(a.w, b.w));
}

__device__ __forceinline__ void cp_async16(void* smem, const uint8_t* gmem)
{
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global.L2::256B [%0], [%1], 16;" ::"r"(sa), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Measurement aid: the combine functions add the bytes of PDM planes each thread loads to
// *loads (a per-thread counter; null: not counted), and the kernel adds each warp's total
// to the caller's device counter once, at its end (add_warp_count).

template <int N>
__device__ __forceinline__ void cp_async_wait_n()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// D' for `nvec` 16-byte chunks through cp.async: each thread streams its chunk of every
// active plane into its own shared-memory slots, kAsyncBatch planes per group with S
// groups in flight (no registers held by the loads), and folds a group once it landed.
// `stage` is this thread's [S][kAsyncBatch] slot array (stride `ld` uint4 between slots);
// s_off holds the n plane offsets followed by kAsyncBatch copies of the first one, so a
// last, partial batch reads plane 0 again (same bytes, no effect on the min).
// A chunk whose minimum has reached 0 in every byte is final: its later batches are
// neither loaded nor folded.
constexpr int kAsyncBatch = 8;

template <int S>
__device__ __forceinline__ void combine_chunks_async(const uint8_t* __restrict__ pdm,
                                                     const int64_t* s_off, int n, int64_t nvec,
                                                     int64_t t0, int64_t stride, uint4* stage,
                                                     int ld, uint8_t* __restrict__ out,
                                                     unsigned* loads)
{
    const int nb = (n + kAsyncBatch - 1) / kAsyncBatch;       // batches per chunk
    if (nb == 0) {
        for (int64_t v = t0; v < nvec; v += stride)
            __stcs(reinterpret_cast<uint4*>(out + (v << 4)), make_uint4(~0u, ~0u, ~0u, ~0u));
        return;
    }
    int64_t v = t0;
    if (v >= nvec) return;
    ByteMin16 acc;                                            // chunk v, batches before jb
    acc.reset();
    bool live = true;                                         // acc may still fall
    // the flattened sequence of (chunk, batch) steps; a step is issued S - 1 steps before
    // it is folded, and loads nothing when the minimum of its chunk is already final
    auto issue = [&](int64_t vv, int b, int slot) {
        const bool load = vv < nvec && (vv != v || live);
        if (load) {
            const uint8_t* src = pdm + (vv << 4);
#pragma unroll
            for (int k = 0; k < kAsyncBatch; ++k)
                cp_async16(stage + (slot * kAsyncBatch + k) * ld,
                           src + s_off[b * kAsyncBatch + k]);
            if (loads) *loads += 16u * unsigned(min(kAsyncBatch, n - b * kAsyncBatch));
        }
        cp_async_commit();
    };
    int64_t iv = v;                                           // next step to issue
    int ib = 0, islot = 0;
    auto advance = [&](int64_t& vv, int& b) {
        if (++b == nb) { b = 0; vv += stride; }
    };
#pragma unroll
    for (int a = 0; a < S - 1; ++a) {
        issue(iv, ib, islot);
        advance(iv, ib);
        islot = islot + 1 == S ? 0 : islot + 1;
    }
    int jb = 0, slot = 0;
    while (true) {
        issue(iv, ib, islot);
        advance(iv, ib);
        islot = islot + 1 == S ? 0 : islot + 1;
        cp_async_wait_n<S - 1>();                             // step (v, jb) landed
        if (live) {
#pragma unroll
            for (int k = 0; k < kAsyncBatch; ++k)
                acc.fold(stage[(slot * kAsyncBatch + k) * ld]);
            live = acc.nonzero();
        }
        if (jb == nb - 1) {
            __stcs(reinterpret_cast<uint4*>(out + (v << 4)), acc.value());
            acc.reset();
            live = true;
        }
        advance(v, jb);
        if (v >= nvec) break;
        slot = slot + 1 == S ? 0 : slot + 1;
    }
    cp_async_wait0();
}

// D' for large maps, plane-major: a CTA walks tiles of kTileChunks chunks; within a tile a
// warp owns 256 consecutive chunks (4 KiB), lane l chunks base + 32 k + l for k < 8.
// One step loads the warp's 4 KiB of one plane (8 cp.async per thread, each instruction
// 512 contiguous bytes), so every DRAM burst of a step is 4 KiB of one plane; the 8
// per-thread accumulators fold the planes and are stored once per tile.  A step is issued
// S - 1 steps before it is folded.  As in the per-chunk path, a chunk whose minimum is 0
// in every byte loads no further plane.
constexpr int kPM = 8;                                        // chunks per thread per tile
template <int S>
__device__ __forceinline__ void combine_tiles_planar(const uint8_t* __restrict__ pdm,
                                                     const int64_t* s_off, int n, int64_t ntiles,
                                                     int64_t tile0, int64_t tstride, uint4* stage,
                                                     int ld, uint8_t* __restrict__ out, int warp,
                                                     int lane, int warps,
                                                     unsigned* loads)
{
    const int64_t tile_chunks = int64_t(warps) * 32 * kPM;
    auto chunk_of = [&](int64_t t, int k) {
        return t * tile_chunks + int64_t(warp) * (32 * kPM) + k * 32 + lane;
    };
    int64_t t = tile0;
    if (t >= ntiles) return;
    if (n == 0) {
        for (; t < ntiles; t += tstride)
#pragma unroll
            for (int k = 0; k < kPM; ++k)
                __stcs(reinterpret_cast<uint4*>(out) + chunk_of(t, k), make_uint4(~0u, ~0u, ~0u, ~0u));
        return;
    }
    ByteMin16 acc[kPM];                                       // tile t, planes before p
#pragma unroll
    for (int k = 0; k < kPM; ++k) acc[k].reset();
    unsigned live = (1u << kPM) - 1;                          // bit k: acc[k] may still fall
    // a step of another tile than t loads every chunk (the accumulators hold tile t)
    auto issue = [&](int64_t tt, int pp, int slot) {
        if (tt < ntiles && (tt != t || live != 0u)) {
            const uint8_t* src = pdm + s_off[pp];
            unsigned issued = 0;
#pragma unroll
            for (int k = 0; k < kPM; ++k)
                if (tt != t || ((live >> k) & 1u)) {
                    cp_async16(stage + (slot * kPM + k) * ld, src + (chunk_of(tt, k) << 4));
                    ++issued;
                }
            if (loads) *loads += 16u * issued;
        }
        cp_async_commit();
    };
    auto advance = [&](int64_t& tt, int& pp) {
        if (++pp == n) { pp = 0; tt += tstride; }
    };
    int64_t it = t;                                           // next step to issue
    int ip = 0, islot = 0;
#pragma unroll
    for (int a = 0; a < S - 1; ++a) {
        issue(it, ip, islot);
        advance(it, ip);
        islot = islot + 1 == S ? 0 : islot + 1;
    }
    int p = 0, slot = 0;
    while (true) {
        issue(it, ip, islot);
        advance(it, ip);
        islot = islot + 1 == S ? 0 : islot + 1;
        cp_async_wait_n<S - 1>();                             // step (t, p) landed
        if (live != 0u) {
#pragma unroll
            for (int k = 0; k < kPM; ++k)
                if ((live >> k) & 1u) {
                    acc[k].fold(stage[(slot * kPM + k) * ld]);
                    if (!acc[k].nonzero()) live &= ~(1u << k);
                }
        }
        if (p == n - 1) {
#pragma unroll
            for (int k = 0; k < kPM; ++k) {
                __stcs(reinterpret_cast<uint4*>(out) + chunk_of(t, k), acc[k].value());
                acc[k].reset();
            }
            live = (1u << kPM) - 1;
        }
        advance(t, p);
        if (t >= ntiles) break;
        slot = slot + 1 == S ? 0 : slot + 1;
    }
    cp_async_wait0();
}

// D' region by region, without the range index: warp w of the grid (w = warp * gridDim.x
// + block, so that small maps spread over every SM) takes regions w, w + warps, ...  For a
// region it lists the active planes (the CTA's list, in the plane order) in ascending order
// of their minimum over the region, ties kept in list order, and reads them one plane per
// step, lane l loading chunks r * 256 + 32 k + l (k < 8) of the plane: 512 contiguous bytes
// per instruction.  A chunk whose minimum is 0 loads no further plane, and the region stops
// as soon as the next plane's regional minimum is at least the largest minimum of the
// region so far: that plane, and every later one, is at least every byte of D' there.
// The first plane is folded before the second is issued (a region that one plane settles
// reads one plane); after that a plane is issued while the one before it is folded, and
// the bound it is checked against is the region's maximum one plane earlier.
// Each warp keeps its sorted list in w_list / w_bnd (kMaxPartitions entries) and uses
// w_key as scratch; `stage` is the thread's [2][kPM] slot array.
__device__ __forceinline__ void combine_regions(const uint8_t* __restrict__ pdm, int64_t plane,
                                                const uint16_t* s_list, int n, int K,
                                                const uint8_t* __restrict__ rmin, int64_t nvec,
                                                int64_t nreg, uint4* stage, int ld,
                                                uint8_t* __restrict__ out, uint16_t* w_list,
                                                uint8_t* w_bnd, uint32_t* w_key, int lane,
                                                int64_t w0, int64_t warps, unsigned* loads)
{
    for (int64_t r = w0; r < nreg; r += warps) {
        // ---- the region's plane list, by regional minimum
        for (int j = lane; j < n; j += 32) {
            const int p = s_list[j];
            w_key[j] = (uint32_t(rmin[r * K + p]) << 16) | uint32_t(j);
        }
        __syncwarp();
        for (int j = lane; j < n; j += 32) {
            const uint32_t key = w_key[j];
            int rank = 0;
            for (int q = 0; q < n; ++q) rank += w_key[q] < key ? 1 : 0;
            w_list[rank] = s_list[j];
            w_bnd[rank] = uint8_t(key >> 16);
        }
        __syncwarp();
        // ---- stream the planes
        const int64_t c0 = r * kRegionChunks + lane;
        unsigned live = 0;                                    // bit k: chunk k may still fall
#pragma unroll
        for (int k = 0; k < kPM; ++k)
            if (c0 + 32 * k < nvec) live |= 1u << k;
        const unsigned valid = live;
        ByteMin16 acc[kPM];
#pragma unroll
        for (int k = 0; k < kPM; ++k) acc[k].reset();
        auto issue = [&](int q, int slot) {
            const uint8_t* src = pdm + int64_t(w_list[q]) * plane;
            unsigned issued = 0;
#pragma unroll
            for (int k = 0; k < kPM; ++k)
                if ((live >> k) & 1u) {
                    cp_async16(stage + (slot * kPM + k) * ld, src + ((c0 + 32 * k) << 4));
                    ++issued;
                }
            cp_async_commit();
            if (loads) *loads += 16u * issued;
        };
        unsigned wmax = 255u;                                 // largest minimum so far
        auto fold = [&](int slot) {
            unsigned tmax = 0;
#pragma unroll
            for (int k = 0; k < kPM; ++k) {
                if ((live >> k) & 1u) {
                    acc[k].fold(stage[(slot * kPM + k) * ld]);
                    const unsigned mk = acc[k].max_byte();
                    if (mk == 0u) live &= ~(1u << k);
                    tmax = max(tmax, mk);
                }
            }
            wmax = __reduce_max_sync(0xFFFFFFFFu, tmax);
        };
        if (n > 0 && w_bnd[0] < wmax) {                       // warp-uniform from here on
            // the first plane alone: the region's minima after it decide the second
            issue(0, 0);
            cp_async_wait_n<0>();
            fold(0);
            int q = 1, slot = 1;
            bool go = q < n && w_bnd[q] < wmax;
            if (go) issue(q, slot);
            while (go) {                                      // then one plane ahead
                const bool next = q + 1 < n && w_bnd[q + 1] < wmax;
                if (next) issue(q + 1, slot ^ 1); else cp_async_commit();
                cp_async_wait_n<1>();                         // plane q landed
                fold(slot);
                go = next;
                ++q;
                slot ^= 1;
            }
        }
#pragma unroll
        for (int k = 0; k < kPM; ++k)
            if ((valid >> k) & 1u)
                __stcs(reinterpret_cast<uint4*>(out) + c0 + 32 * k, acc[k].value());
        __syncwarp();                                         // w_key / w_list are reused
    }
    cp_async_wait0();
}

// COUNT: the measurement build, which adds the PDM bytes it loads to *count.
template <bool COUNT>
__global__ void __launch_bounds__(kCombineThreads)
k_combine(const uint8_t* __restrict__ pdm, int64_t plane, int64_t G,
          const uint16_t* __restrict__ act, const int32_t* __restrict__ nact,
          uint8_t* __restrict__ out, int vec_ok, unsigned long long* __restrict__ count)
{
    constexpr int kBatch = 8;                          // plane loads issued before any use
    __shared__ int64_t s_off[kMaxPartitions + kBatch];
    __shared__ int s_n;
    extern __shared__ uint4 s_stage[];                 // [2][kAsyncBatch][kCombineThreads]
    pdl_wait();        // the active set written by the previous kernel is visible now
    if (threadIdx.x == 0) s_n = *nact;
    __syncthreads();
    const int n = s_n;
    for (int j = threadIdx.x; j < kMaxPartitions + kBatch; j += kCombineThreads)
        s_off[j] = int64_t(act[j < n ? j : 0]) * plane;      // padding: copies of plane 0
    __syncthreads();
    const int64_t stride = int64_t(gridDim.x) * kCombineThreads;
    const int64_t t0 = int64_t(blockIdx.x) * kCombineThreads + threadIdx.x;
    int64_t done = 0;
    unsigned loaded = 0;
    unsigned* lp = COUNT ? &loaded : nullptr;
    if (vec_ok) {
        combine_chunks_async<2>(pdm, s_off, n, G >> 4, t0, stride, s_stage + threadIdx.x,
                                kCombineThreads, out, lp);
        done = (G >> 4) << 4;
    }
    // bytes not covered by whole aligned chunks
    for (int64_t i = done + t0; i < G; i += stride) {
        unsigned acc = 255;
        for (int j = 0; j < n; ++j) acc = min(acc, unsigned(pdm[s_off[j] + i]));
        out[i] = uint8_t(acc);
        if (COUNT) loaded += unsigned(n);
    }
    if (COUNT) add_warp_count(count, loaded);
}

// Step 1 and step 2 in one launch (TFs with N <= kFusedMaxN): every CTA derives S from
// the alpha channel itself (independent loads, ballots into a visibility bit set in shared
// memory, one scan per partition), so the combine waits on no other kernel.  CTA 0 also
// publishes S (list, count, bit set) for callers that read it back.
constexpr int kFusedThreads = 512;
constexpr int kFusedMaxN = 8192;
// plane loads in flight per thread: kFusedStages - 1 steps ahead of the fold (128 KiB of
// staging for 2 stages; 3 stages, 192 KiB, measured no faster on the large map and slower
// on the smaller ones)
constexpr int kFusedStages = 2;
static_assert(kPM == kAsyncBatch, "both paths use the same slots");

// COUNT: the measurement build, which adds the PDM bytes it loads to *count.
template <bool COUNT>
__global__ void __launch_bounds__(kFusedThreads)
k_update_fused(const uint8_t* __restrict__ pdm, int64_t plane, int64_t G,
               const float* __restrict__ tf, int N, int K, int J, Borders bd, int uniform,
               const uint16_t* __restrict__ order, const uint8_t* __restrict__ rmin,
               uint16_t* __restrict__ act, int32_t* __restrict__ nact,
               uint64_t* __restrict__ smask, uint64_t* __restrict__ smask_out,
               uint8_t* __restrict__ out, int vec_ok, unsigned long long* __restrict__ count)
{
    constexpr int kBatch = 8;
    constexpr int kPer = kFusedMaxN / kFusedThreads;          // alphas per thread (max)
    constexpr int kWarps = kFusedThreads / 32;
    __shared__ uint32_t s_vis[kFusedMaxN / 32];
    __shared__ uint32_t s_wkey[kWarps][kMaxPartitions];       // per warp: region plan
    __shared__ uint16_t s_wlist[kWarps][kMaxPartitions];
    __shared__ uint8_t s_wbnd[kWarps][kMaxPartitions];
    __shared__ int64_t s_off[kMaxPartitions + kBatch];
    __shared__ uint32_t s_bits[8];
    __shared__ uint16_t s_list[kMaxPartitions + kBatch];
    __shared__ int s_scan[9];
    extern __shared__ uint4 s_stage[];      // [kFusedStages][kAsyncBatch][kFusedThreads]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    pdl_wait();
    const int mine = order && tid < K ? int(order[tid]) : tid;     // this thread's plane
    // ---- visibility bits: thread t holds intensities t + k * blockDim
    float a[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int i = k * kFusedThreads + tid;
        a[k] = i < N ? __ldg(tf + 4 * int64_t(i) + 3) : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        if (k * kFusedThreads < N) {                          // uniform over the block
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, a[k] > 0.0f);
            const int word = (k * kFusedThreads >> 5) + warp;
            if (lane == 0 && word * 32 < N) s_vis[word] = bal;
        }
    }
    __syncthreads();
    // ---- S: partition p active iff a visibility bit in [lo_p, hi_p] is set
    bool on = false;
    if (tid < K) {
        // uniform borders are computed: indexing the parameter array by thread serialises
        // the constant-cache reads of a warp
        const int lo = uniform ? (tid * N) / K : bd.v[tid];
        const int hi = (uniform ? ((tid + 1) * N) / K : bd.v[tid + 1]) - 1;
        for (int w = lo >> 5; w <= (hi >> 5) && !on; ++w) {
            uint32_t m = s_vis[w];
            if (w == (lo >> 5)) m &= 0xFFFFFFFFu << (lo & 31);
            if (w == (hi >> 5)) m &= 0xFFFFFFFFu >> (31 - (hi & 31));
            on = m != 0;
        }
    }
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, on);
    if (lane == 0 && warp < 8) s_bits[warp] = bal;
    __syncthreads();
    // ---- planes to combine: the active partitions, or index planes covering their runs
    const int n = plan_maps(s_bits, K, J, s_list, s_scan, mine);
    for (int j = tid; j < kMaxPartitions + kBatch; j += kFusedThreads)
        s_off[j] = int64_t(s_list[j < n ? j : 0]) * plane;     // padding: copies of plane 0
    if (blockIdx.x == 0) {
        for (int j = tid; j < n; j += kFusedThreads) act[j] = s_list[j];
        if (tid == 0) *nact = n;
        if (tid < 4) {
            const uint64_t v = uint64_t(s_bits[2 * tid]) | (uint64_t(s_bits[2 * tid + 1]) << 32);
            smask[tid] = v;
            if (smask_out && tid < (K + 63) / 64) smask_out[tid] = v;
        }
    }
    __syncthreads();
    // ---- Eq. 1 over the active planes
    const int64_t stride = int64_t(gridDim.x) * kFusedThreads;
    const int64_t t0 = int64_t(blockIdx.x) * kFusedThreads + tid;
    int64_t done = 0;
    unsigned loaded = 0;                                       // plane bytes (COUNT only)
    unsigned* lp = COUNT ? &loaded : nullptr;
    if (vec_ok) {
        // Large maps: whole plane-major tiles while every CTA gets at least two and they
        // spread evenly (all of them when the last round fills three quarters of the CTAs,
        // else a multiple of the grid); every other chunk through the per-chunk path.
        const int64_t nvec = G >> 4;
        if (J < 0 && rmin && 2 * num_regions(G) >= int64_t(kWarps) * gridDim.x) {
            // the plain planes with their region bounds, region by region, when there are
            // regions for at least half of the warps (a smaller map is bound by the latency
            // of its plane steps, which the per-chunk path overlaps 8 planes at a time)
            combine_regions(pdm, plane, s_list, n, K, rmin, nvec, num_regions(G),
                            s_stage + tid, kFusedThreads, out, s_wlist[warp], s_wbnd[warp],
                            s_wkey[warp], lane, int64_t(warp) * gridDim.x + blockIdx.x,
                            int64_t(kWarps) * gridDim.x, lp);
        } else {
            const int64_t tile_chunks = int64_t(kFusedThreads) * kPM;
            const int64_t grid = gridDim.x;
            int64_t ntiles = nvec / tile_chunks;
            if (ntiles < 2 * grid) ntiles = 0;
            else if (ntiles % grid != 0 && 4 * (ntiles % grid) < 3 * grid)
                ntiles -= ntiles % grid;
            if (ntiles > 0)
                combine_tiles_planar<kFusedStages>(pdm, s_off, n, ntiles, blockIdx.x, grid,
                                                   s_stage + tid, kFusedThreads, out, warp,
                                                   lane, kWarps, lp);
            combine_chunks_async<kFusedStages>(pdm, s_off, n, nvec, ntiles * tile_chunks + t0,
                                               stride, s_stage + tid, kFusedThreads, out, lp);
        }
        done = nvec << 4;
    }
    for (int64_t i = done + t0; i < G; i += stride) {
        unsigned acc = 255;
        for (int j = 0; j < n; ++j) acc = min(acc, unsigned(pdm[s_off[j] + i]));
        out[i] = uint8_t(acc);
        if (COUNT) loaded += unsigned(n);
    }
    if (COUNT) add_warp_count(count, loaded);
}

// One level of the partition-range index: plane (k, i) = min(plane (k-1, i),
// plane (k-1, i + 2^(k-1))), 16 bytes per thread (bytes for a ragged tail).
__global__ void __launch_bounds__(256)
k_index_level(uint8_t* __restrict__ pdm, int64_t plane, int64_t G, int prev_base, int base,
              int half, int vec_ok)
{
    pdl_wait();
    const int i = blockIdx.y;
    const uint8_t* a = pdm + int64_t(prev_base + i) * plane;
    const uint8_t* b = pdm + int64_t(prev_base + i + half) * plane;
    uint8_t* o = pdm + int64_t(base + i) * plane;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t t0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t done = 0;
    if (vec_ok) {
        const int64_t nvec = G >> 4;
        for (int64_t v = t0; v < nvec; v += stride)
            reinterpret_cast<uint4*>(o)[v] = vmin4(__ldcs(reinterpret_cast<const uint4*>(a) + v),
                                                   __ldcs(reinterpret_cast<const uint4*>(b) + v));
        done = nvec << 4;
    }
    for (int64_t j = done + t0; j < G; j += stride) o[j] = min(a[j], b[j]);
}

// ---------------------------------------------------------------- plane order
// Zero bytes of each plane on a fixed sample (kCoverSamples 16-byte chunks at an even
// stride, or bytes where the plane is not 16-byte aligned): kCoverSplit CTAs per plane,
// each writing its part of the count (no atomics, so the count is the same on every run);
// a thread issues all its loads before it uses any.
constexpr int kCoverSamples = 8192;
constexpr int kOrderThreads = 256;
constexpr int kCoverPer = kCoverSamples / kOrderThreads;
static_assert(kCoverPer % kCoverSplit == 0, "each CTA of a plane takes whole rounds");
static_assert(kMaxPartitions <= kOrderThreads, "one thread per partition ranks the planes");

struct PlaneOrderBatch {
    int n;
    int start[kMaxBuildBatch + 1];             // first CTA (plane) of each context
    int rstart[kMaxBuildBatch + 1];            // first CTA of each context's region minima
    PlaneOrderItem it[kMaxBuildBatch];
};

constexpr int kRminWarps = 8;                  // (region, plane) pairs per CTA



__global__ void __launch_bounds__(kOrderThreads)
k_plane_cover(const __grid_constant__ PlaneOrderBatch B)
{
    __shared__ uint32_t s_w[kOrderThreads / 32];
    const int i = batch_item_of(B.start, B.n, int(blockIdx.x));
    const PlaneOrderItem& it = B.it[i];
    const int local = int(blockIdx.x) - B.start[i];
    const int p = local / kCoverSplit, q = local - p * kCoverSplit;   // plane, its part
    const uint8_t* src = it.pdm + int64_t(p) * it.plane;
    const int tid = threadIdx.x;
    pdl_wait();
    uint32_t z = 0;                                            // zero bytes x 8
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0 && it.G >= 16) {
        const int64_t nvec = it.G >> 4;
        const int64_t ns = nvec < kCoverSamples ? nvec : kCoverSamples;
        const int64_t step = nvec / ns;
        const uint4* v4 = reinterpret_cast<const uint4*>(src);
        constexpr int kPer = kCoverPer / kCoverSplit;          // loads per thread, all at once
        uint4 v[kPer];
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int64_t j = int64_t(r * kCoverSplit + q) * kOrderThreads + tid;
            v[r] = j < ns ? __ldcs(v4 + j * step) : make_uint4(1u, 1u, 1u, 1u);
        }
#pragma unroll
        for (int r = 0; r < kPer; ++r)
            z += __popc(__vcmpeq4(v[r].x, 0u)) + __popc(__vcmpeq4(v[r].y, 0u)) +
                 __popc(__vcmpeq4(v[r].z, 0u)) + __popc(__vcmpeq4(v[r].w, 0u));
    } else {
        const int64_t ns = it.G < 16 * kCoverSamples ? it.G : 16 * kCoverSamples;
        const int64_t step = ns > 0 ? it.G / ns : 1;
        for (int64_t j = int64_t(q) * kOrderThreads + tid; j < ns;
             j += int64_t(kOrderThreads) * kCoverSplit)
            z += src[j * step] == 0 ? 8u : 0u;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) z += __shfl_xor_sync(0xFFFFFFFFu, z, d);
    if ((tid & 31) == 0) s_w[tid >> 5] = z;
    __syncthreads();
    if (tid == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kOrderThreads / 32; ++w) t += s_w[w];
        it.cover[p * kCoverSplit + q] = t >> 3;
    }
}

// Rank of partition t: the planes with more zero bytes, and those with as many and a lower
// index, come before it.
__global__ void __launch_bounds__(kOrderThreads)
k_plane_order(const __grid_constant__ PlaneOrderBatch B)
{
    __shared__ uint32_t s_c[kMaxPartitions];
    const PlaneOrderItem& it = B.it[blockIdx.x];
    const int tid = threadIdx.x;
    pdl_wait();
    if (tid < it.K) {
        uint32_t c = 0;
        for (int q = 0; q < kCoverSplit; ++q) c += it.cover[tid * kCoverSplit + q];
        s_c[tid] = c;
    }
    __syncthreads();
    if (tid < it.K) {
        const uint32_t c = s_c[tid];
        int r = 0;
        for (int q = 0; q < it.K; ++q) {
            const uint32_t d = s_c[q];
            r += (d > c || (d == c && q < tid)) ? 1 : 0;
        }
        it.order[r] = uint16_t(tid);
    }
}

// The minimum of plane p over region r: one warp per (region, plane), plane-major so that
// neighbouring warps read neighbouring regions; 16-byte loads where the plane is aligned,
// the bytes past the last whole chunk one by one.
__global__ void __launch_bounds__(kRminWarps * 32)
k_region_min(const __grid_constant__ PlaneOrderBatch B)
{
    const int i = batch_item_of(B.rstart, B.n, int(blockIdx.x));
    const PlaneOrderItem& it = B.it[i];
    const int lane = threadIdx.x & 31;
    const int64_t nreg = num_regions(it.G);
    const int64_t u = int64_t(int(blockIdx.x) - B.rstart[i]) * kRminWarps + (threadIdx.x >> 5);
    pdl_wait();
    if (u >= nreg * it.K) return;                            // warp-uniform
    const int p = int(u / nreg);
    const int64_t r = u - int64_t(p) * nreg;
    const uint8_t* src = it.pdm + int64_t(p) * it.plane;
    const int64_t b0 = r * kRegionBlocks;
    const int64_t b1 = b0 + kRegionBlocks < it.G ? b0 + kRegionBlocks : it.G;
    unsigned m = 255u;
    int64_t done = b0;
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const int64_t c0 = b0 >> 4, c1 = b1 >> 4;           // b0 is a multiple of 16
        const uint4* v4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
        for (int k = 0; k < kRegionChunks / 32; ++k) {
            const int64_t c = c0 + k * 32 + lane;
            if (c < c1) m = min(m, bytemin16(__ldcs(v4 + c)));
        }
        done = c1 << 4;
    }
    for (int64_t b = done + lane; b < b1; b += 32) m = min(m, unsigned(src[b]));
    m = __reduce_min_sync(0xFFFFFFFFu, m);
    if (lane == 0) it.rmin[r * it.K + p] = uint8_t(m);
}

// ---------------------------------------------------------------- region bounds by rows
// Where a region is whole rows of blocks (4096 a multiple of gx), the minimum of a PDM over
// a region is the minimum over its rows (y, z) of D2(y, z), the 2D chessboard distance
// transform of the partition's occupancy ORed along x: a block of the row can sit above
// the nearest occupied block in x, so x adds nothing to the distance.  D2 is built with
// the x pass and the line pass over the projected masks (y as x, z as y), about gx times
// fewer bytes than the PDMs; the regional minima then come from D2.

// P[row][w] = OR over x of mask[(row * gx + x) * W + w]: one warp per row.
__global__ void __launch_bounds__(256)
k_row_project(const uint64_t* __restrict__ mask, int W, int gx, int64_t rows,
              uint64_t* __restrict__ proj)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = int64_t(blockIdx.x) * 8 + (threadIdx.x >> 5);
    pdl_wait();
    if (row >= rows) return;                                 // warp-uniform
    const uint64_t* src = mask + row * gx * W;
    for (int w = 0; w < W; ++w) {
        uint64_t m = 0;
        for (int x = lane; x < gx; x += 32) m |= src[int64_t(x) * W + w];
        const unsigned lo = __reduce_or_sync(0xFFFFFFFFu, unsigned(m));
        const unsigned hi = __reduce_or_sync(0xFFFFFFFFu, unsigned(m >> 32));
        if (lane == 0) proj[row * W + w] = (uint64_t(hi) << 32) | lo;
    }
}

// rmin[r][p] = min over the rows of region r of D2_p: one thread per (plane, region), so
// that neighbouring threads read neighbouring regions' rows; 16-byte loads where a region
// is whole 16-row vectors.
__global__ void __launch_bounds__(256)
k_region_min_rows(const uint8_t* __restrict__ d2, int64_t plane2, int64_t rows,
                  int rows_per_region, int K, int64_t nreg, uint8_t* __restrict__ rmin)
{
    const int64_t u = int64_t(blockIdx.x) * 256 + threadIdx.x;
    pdl_wait();
    if (u >= nreg * K) return;
    const int p = int(u / nreg);
    const int64_t r = u - int64_t(p) * nreg;
    const int64_t q0 = r * rows_per_region;
    const int64_t q1 = q0 + rows_per_region < rows ? q0 + rows_per_region : rows;
    const uint8_t* src = d2 + int64_t(p) * plane2;           // plane2: a multiple of 64
    unsigned m = 255u;
    int64_t q = q0;
    if (rows_per_region % 16 == 0)
        for (; q + 16 <= q1; q += 16)
            m = min(m, bytemin16(*reinterpret_cast<const uint4*>(src + q)));
    for (; q < q1; ++q) m = min(m, unsigned(src[q]));
    rmin[r * K + p] = uint8_t(m);
}

}  // namespace

cudaError_t launch_build_index(uint8_t* pdm, int64_t plane, int64_t G, int K, cudaStream_t s)
{
    const int J = index_levels(K);
    const int vec_ok = ((reinterpret_cast<uintptr_t>(pdm) & 15) == 0) && (plane % 16 == 0);
    for (int k = 1; k <= J; ++k) {
        const int count = K - (1 << k) + 1;
        const int64_t work = vec_ok ? (G >> 4) : G;
        int64_t bx = (work + 255) / 256;
        if (bx > 1024) bx = 1024;
        if (bx < 1) bx = 1;
        cudaError_t e = launch_pdl(k_index_level, dim3(unsigned(bx), unsigned(count)), dim3(256), 0, s,
                                   pdm, plane, G, index_level_base(K, k - 1), index_level_base(K, k),
                                   1 << (k - 1), vec_ok);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

bool update_fused_ok(int N) { return N <= kFusedMaxN; }

cudaError_t launch_update_fused(const uint8_t* pdm, int64_t plane, int64_t G, const float* tf,
                                int N, int K, int J, const Borders& bd, int uniform,
                                const uint16_t* order, const uint8_t* rmin, uint16_t* act,
                                int32_t* nact, uint64_t* smask, uint64_t* smask_out,
                                uint8_t* out, int num_sms, unsigned long long* count,
                                cudaStream_t s)
{
    if (N > kFusedMaxN) return cudaErrorInvalidValue;
    const int vec_ok = ((reinterpret_cast<uintptr_t>(pdm) & 15) == 0) &&
                       ((reinterpret_cast<uintptr_t>(out) & 15) == 0) && (plane % 16 == 0);
    const int64_t work = vec_ok ? (G >> 4) : G;
    const int64_t want = (work + kFusedThreads - 1) / kFusedThreads;
    const size_t smem =
        vec_ok ? size_t(kFusedStages) * kAsyncBatch * kFusedThreads * sizeof(uint4) : 0;
    const int64_t cap = int64_t(num_sms > 0 ? num_sms : 152);  // one 512-thread CTA per SM
    const int blocks = int(want < cap ? (want > 0 ? want : 1) : cap);
    auto kern = count ? k_update_fused<true> : k_update_fused<false>;
    cudaError_t e = count ? ensure_dynamic_smem<k_update_fused<true>>(int(smem))
                          : ensure_dynamic_smem<k_update_fused<false>>(int(smem));
    if (e != cudaSuccess) return e;
    kern<<<blocks, kFusedThreads, smem, s>>>(pdm, plane, G, tf, N, K, J, bd, uniform, order,
                                            rmin, act, nact, smask, smask_out, out, vec_ok,
                                            count);
    return cudaGetLastError();
}

cudaError_t launch_tf_active(const float* tf, int N, int K, const Borders& bd, int32_t* cnt,
                             uint16_t* act, int32_t* nact, uint64_t* smask,
                             uint64_t* smask_out, cudaStream_t s)
{
    k_tf_active<<<1, kActThreads, 0, s>>>(tf, N, K, bd, cnt, act, nact, smask, smask_out);
    return cudaGetLastError();
}

cudaError_t launch_active_set(const float* tf, int N, int K, int J, const Borders& bd,
                              const uint16_t* order, uint16_t* act, int32_t* nact,
                              uint64_t* smask, uint64_t* smask_out, cudaStream_t s)
{
    k_active_set<<<1, kActThreads, 0, s>>>(tf, N, K, J, bd, order, act, nact, smask, smask_out);
    return cudaGetLastError();
}

cudaError_t launch_combine(const uint8_t* pdm, int64_t plane, int64_t G, const uint16_t* act,
                           const int32_t* nact, uint8_t* out, int num_sms,
                           unsigned long long* count, cudaStream_t s)
{
    const int vec_ok = ((reinterpret_cast<uintptr_t>(pdm) & 15) == 0) &&
                       ((reinterpret_cast<uintptr_t>(out) & 15) == 0) && (plane % 16 == 0);
    int64_t work = vec_ok ? (G >> 4) : G;
    int64_t want = (work + kCombineThreads - 1) / kCombineThreads;
    const size_t smem = vec_ok ? size_t(2) * kAsyncBatch * kCombineThreads * sizeof(uint4) : 0;
    int64_t cap = int64_t(num_sms > 0 ? num_sms : 152) * 3;   // 3 resident CTAs per SM
    int blocks = int(want < cap ? (want > 0 ? want : 1) : cap);
    cudaError_t e = count ? ensure_dynamic_smem<k_combine<true>>(int(smem))
                          : ensure_dynamic_smem<k_combine<false>>(int(smem));
    if (e != cudaSuccess) return e;
    return launch_pdl(count ? k_combine<true> : k_combine<false>, dim3(blocks),
                      dim3(kCombineThreads), smem, s, pdm, plane, G, act, nact, out, vec_ok,
                      count);
}

cudaError_t launch_plane_order(const PlaneOrderItem* items, int n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (n > kMaxBuildBatch) return cudaErrorInvalidValue;
    PlaneOrderBatch B;
    B.n = n;
    int ctas = 0;
    for (int k = 0; k < n; ++k) {
        if (items[k].K < 1 || items[k].K > kMaxPartitions) return cudaErrorInvalidValue;
        B.it[k] = items[k];
        B.start[k] = ctas;
        ctas += items[k].K * kCoverSplit;
    }
    B.start[n] = ctas;
    cudaError_t e = launch_pdl(k_plane_cover, dim3(unsigned(ctas)), dim3(kOrderThreads), 0, s, B);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_plane_order, dim3(unsigned(n)), dim3(kOrderThreads), 0, s, B);
    if (e != cudaSuccess) return e;
    // the region minima read from the planes, for the items that ask for it
    PlaneOrderBatch R;
    R.n = 0;
    int64_t rctas = 0;
    for (int k = 0; k < n; ++k) {
        if (!items[k].bounds_from_planes) continue;
        R.it[R.n] = items[k];
        R.rstart[R.n++] = int(rctas);
        rctas += (num_regions(items[k].G) * items[k].K + kRminWarps - 1) / kRminWarps;
        if (rctas > int64_t(0x7FFFFFFF)) return cudaErrorInvalidConfiguration;
    }
    if (R.n == 0) return cudaSuccess;
    R.rstart[R.n] = int(rctas);
    return launch_pdl(k_region_min, dim3(unsigned(rctas)), dim3(kRminWarps * 32), 0, s, R);
}

// The projected grid: rows (y, z) of the volume's grid as a one-slice grid, y along x.
static Geometry row_geometry(const Geometry& g)
{
    Geometry g2 = g;
    g2.gx = g.gy;
    g2.gy = g.gz;
    g2.gz = 1;
    g2.G = int64_t(g.gy) * g.gz;
    g2.plane = (g2.G + 63) / 64 * 64;
    return g2;
}

bool bounds_from_rows_ok(const Geometry& g, int K)
{
    if (g.gx < 32 || kRegionBlocks % g.gx != 0) return false;
    const Geometry g2 = row_geometry(g);
    return g2.gx <= 10240 && xpass_smem(g2.gx, K) <= size_t(kXpassSmemLimit) &&
           line_pass_smem(g2.gy) <= size_t(kLineSmemLimit);
}

size_t bounds_rows_proj_bytes(const Geometry& g, int K)
{
    return size_t(row_geometry(g).G) * size_t((K + 63) / 64) * 8;
}

size_t bounds_rows_d2_bytes(const Geometry& g, int K)
{
    return size_t(row_geometry(g).plane) * size_t(K);
}

cudaError_t launch_bounds_from_rows(const uint64_t* mask, const Geometry& g, int K,
                                    uint64_t* proj, bool projected, uint8_t* d2, uint8_t* rmin,
                                    cudaStream_t s)
{
    const Geometry g2 = row_geometry(g);
    const int W = (K + 63) / 64;
    cudaError_t e = cudaSuccess;
    if (!projected) {                                        // the x pass did not write proj
        e = launch_pdl(k_row_project, dim3(unsigned((g2.G + 7) / 8)), dim3(256), 0, s, mask, W,
                       int(g.gx), g2.G, proj);
        if (e != cudaSuccess) return e;
    }
    e = launch_xpass_mask(proj, K, g2, d2, s);              // distance along y
    if (e != cudaSuccess) return e;
    e = launch_line_pass(d2, K, g2.plane, g2, 1, s);        // then the max-min along z
    if (e != cudaSuccess) return e;
    const int64_t nreg = num_regions(g.G);
    const int64_t n = nreg * K;
    return launch_pdl(k_region_min_rows, dim3(unsigned((n + 255) / 256)), dim3(256), 0, s, d2,
                      g2.plane, g2.G, int(kRegionBlocks / g.gx), K, nreg, rmin);
}

}  // namespace dmk
