// dm_batch.cu -- the per-TF update for many volumes and many TF edits at once.
//
// A group is one volume's resident PDMs (§3.1) with up to kMaxGroupEdits TFs.  Two launches
// cover up to kMaxBatch groups: an active-set kernel with one CTA per group (§3.1 step 1
// for each of the group's TFs, from the partition table built at precompute time; all
// loads of a batch issued before any is used), then a combine (Eq. 1) over one flattened
// list of 4 KiB work units of all groups, launched with programmatic dependent launch.
// The active-set CTA writes the union of the group's plane lists with, per plane, the set
// of the group's TFs that take it; the combine reads each plane of that union once per work
// unit and folds it into the running minimum of every TF that takes it, so a volume's
// edits share their plane reads.  By default each combine CTA takes one unit.  The bytes
// past a group's last whole 16-byte chunk are folded by one warp per group, its lanes over
// the planes.  Per-group descriptors are passed by value as kernel parameters, so the pair
// needs no device-side setup and can be captured in a CUDA graph.
#include "dm_internal.cuh"

namespace dmk {
namespace {

constexpr int kActThreads = 1024;
constexpr int kThreads = 256;                  // combine CTA; one work unit = 256 x 16 B
constexpr int kMaxPlanes = 2048;               // planes of a PDM buffer with the range index
constexpr int kPad = 8;                        // list padding: covers the largest load group
static_assert(kMaxPartitions + kPad >= kThreads, "a list buffer covers one entry per thread");

struct Group {
    const uint8_t* pdm;
    int64_t plane;
    int64_t G;
    const uint8_t* lut;                        // partition of each intensity (precompute)
    const uint16_t* order;                     // plane order (precompute; null: ascending)
    uint16_t* list;                            // plane list, padded (workspace or scratch)
    uint8_t* emask;                            // per list entry: the TFs taking the plane
    int32_t* count;
    int32_t N, K, J;                           // J: index levels (-1: none)
    int32_t E;                                 // TFs of the group, 1..kMaxGroupEdits
    int32_t vec;                               // 16-byte units (else bytes)
    const float* tf[kMaxGroupEdits];
    uint8_t* out[kMaxGroupEdits];
};

struct Params {
    int n;
    unsigned long long* count;                 // PDM bytes loaded (measurement; may be null)
    int64_t q, r;                              // CTA b takes q units, plus one if b < r
    int64_t unit_prefix[kMaxBatch + 1];        // work units before group i (256 lanes each)
    Group g[kMaxBatch];
};

__device__ __forceinline__ void cp_async16(void* smem, const uint8_t* gmem)
{
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global.L2::256B [%0], [%1], 16;" ::"r"(sa), "l"(gmem)
                 : "memory");
}

// §3.1 step 1 for every TF of group blockIdx.x: partition lut[i] is active when
// alpha_i > 0.  A warp holds 32 consecutive intensities, so its visible partitions fall in
// few mask words: it ORs each word over the warp and one lane sets it, with no
// same-address shared atomics between the lanes.  Each TF's planes (the active partitions,
// or index planes covering their runs) are marked in a per-plane TF set; the planes any TF
// takes are then listed with their TF sets (in the volume's plane order without the index,
// else ascending), followed by kPad copies of the first entry, so that the combine can read
// the list in groups of up to kPad without knowing its length first (a repeated plane
// changes no minimum).
template <int EMAX>
__global__ void __launch_bounds__(kActThreads) k_active_group(const __grid_constant__ Params P)
{
    pdl_trigger();
    __shared__ uint32_t s_S[kMaxPartitions / 32];
    __shared__ uint16_t s_list[kMaxPartitions + 8];
    __shared__ uint8_t s_em[EMAX > 1 ? kMaxPlanes : 1];
    __shared__ uint16_t s_ord[EMAX > 1 ? kMaxPartitions : 1];
    __shared__ int s_scan[33];
    const Group& g = P.g[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mine = g.order && tid < g.K ? int(g.order[tid]) : tid;   // this thread's plane
    const bool ordered = EMAX > 1 && g.J < 0 && g.order != nullptr;
    if (ordered && tid < g.K) s_ord[tid] = uint16_t(mine);
    const int planes = EMAX > 1 ? (g.J < 0 ? g.K : index_level_base(g.K, g.J + 1)) : 0;
    if (EMAX > 1)
        for (int j = tid; j < planes; j += kActThreads) s_em[j] = 0;
    int n = 0;
    for (int e = 0; e < g.E; ++e) {
        if (tid < kMaxPartitions / 32) s_S[tid] = 0;
        __syncthreads();
        constexpr int kLB = 8;                                // loads issued before any use
        const float* tf = g.tf[e];
        for (int base = 0; base < g.N; base += kActThreads * kLB) {
            float a[kLB];
            uint8_t c[kLB];
#pragma unroll
            for (int k = 0; k < kLB; ++k) {
                const int i = base + k * kActThreads + tid;
                a[k] = i < g.N ? __ldg(tf + 4 * int64_t(i) + 3) : 0.0f;
                c[k] = i < g.N ? g.lut[i] : uint8_t(0);
            }
#pragma unroll
            for (int k = 0; k < kLB; ++k) {
                const bool vis = a[k] > 0.0f;
                const unsigned w = c[k] >> 5;
                const unsigned wlo = __reduce_min_sync(0xFFFFFFFFu, vis ? w : 8u);
                const unsigned whi = __reduce_max_sync(0xFFFFFFFFu, vis ? w : 0u);
                for (unsigned ww = wlo; ww <= whi; ++ww) {    // usually one word
                    const unsigned bit = (vis && w == ww) ? 1u << (c[k] & 31) : 0u;
                    const unsigned m = __reduce_or_sync(0xFFFFFFFFu, bit);
                    if (lane == 0 && m) atomicOr(&s_S[ww], m);
                }
            }
        }
        __syncthreads();
        n = plan_maps(s_S, g.K, g.J, s_list, s_scan, mine);  // ends with a CTA barrier
        if (EMAX > 1)
            for (int j = tid; j < n; j += kActThreads) s_em[s_list[j]] |= uint8_t(1u << e);
    }
    if (EMAX == 1) {                                          // one TF: its plan is the list
        for (int j = tid; j < n + kPad; j += kActThreads)
            g.list[j] = n ? s_list[j < n ? j : 0] : uint16_t(0);
        if (tid == 0) *g.count = n;
        return;
    }
    __syncthreads();
    // list the planes some TF takes: each thread scans two consecutive list positions, the
    // planes at those positions of the plane order (or those positions themselves)
    const int p0 = 2 * tid;
    const int q0 = p0 < planes ? (ordered ? int(s_ord[p0]) : p0) : 0;
    const int q1 = p0 + 1 < planes ? (ordered ? int(s_ord[p0 + 1]) : p0 + 1) : 0;
    const int c0 = p0 < planes && s_em[q0] ? 1 : 0;
    const int c1 = p0 + 1 < planes && s_em[q1] ? 1 : 0;
    int incl = c0 + c1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31) s_scan[warp] = incl;
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int w = 0; w < 32; ++w) {
            const int t = s_scan[w];
            s_scan[w] = run;
            run += t;
        }
        s_scan[32] = run;
    }
    __syncthreads();
    int pos = s_scan[warp] + incl - c0 - c1;
    if (c0) {
        g.list[pos] = uint16_t(q0);
        g.emask[pos] = s_em[q0];
        ++pos;
    }
    if (c1) {
        g.list[pos] = uint16_t(q1);
        g.emask[pos] = s_em[q1];
    }
    const int u = s_scan[32];
    __syncthreads();                                          // the first entry is written
    if (tid < kPad) {
        g.list[u + tid] = u ? g.list[0] : uint16_t(0);
        g.emask[u + tid] = u ? g.emask[0] : uint8_t(0);
    }
    if (tid == 0) *g.count = u;
}

// Running byte minimum of one 16-byte chunk for each TF of a group.
template <int EMAX>
struct GroupMin {
    ByteMin16 acc[EMAX];
    __device__ __forceinline__ void reset()
    {
#pragma unroll
        for (int e = 0; e < EMAX; ++e) acc[e].reset();
    }
    __device__ __forceinline__ void fold(const uint4& v, unsigned em)
    {
#pragma unroll
        for (int e = 0; e < EMAX; ++e)
            if (EMAX == 1 || ((em >> e) & 1u)) acc[e].fold(v);
    }
    // some TF of the group (e < E) still has a byte above 0: later planes may lower it
    __device__ __forceinline__ bool live(int E) const
    {
        bool any = false;
#pragma unroll
        for (int e = 0; e < EMAX; ++e)
            if (EMAX == 1 || e < E) any = any || acc[e].nonzero();
        return any;
    }
};

// Bytes past the last whole 16-byte chunk of a group (fewer than 16): one warp, the lanes
// over the group's planes, then a warp min per byte and TF.
template <int EMAX, bool COUNT>
__device__ __forceinline__ void group_tail(const Group& g, int lane, unsigned& loaded)
{
    const int64_t g0 = (g.G >> 4) << 4;
    const int rem = int(g.G - g0);
    if (rem == 0) return;                                     // warp-uniform
    const int n = *g.count;
    const int E = EMAX == 1 ? 1 : g.E;
    for (int e = 0; e < E; ++e) {
        unsigned m[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) m[r] = 255;
        for (int j = lane; j < n; j += 32) {
            if (EMAX > 1 && !((g.emask[j] >> e) & 1u)) continue;
            const uint8_t* src = g.pdm + int64_t(g.list[j]) * g.plane + g0;
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (r < rem) m[r] = min(m[r], unsigned(src[r]));
            if (COUNT) loaded += unsigned(rem);
        }
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if (r < rem) {
                const unsigned v = __reduce_min_sync(0xFFFFFFFFu, m[r]);
                if (lane == 0) g.out[e][g0 + r] = uint8_t(v);
            }
        }
    }
}

// Eq. 1 over every group's work units; CTA b takes a contiguous range of units.  KB plane
// loads per stage, two stages in flight.  With one TF per group, at most 40 registers a
// thread, so that 6 CTAs fit an SM next to their 6 x 34 KiB of shared memory.  COUNT: the
// measurement variant, which adds the PDM bytes it loads to *P.count (its own
// instantiation, so that the counter costs the timed kernel no register).
template <int EMAX, int KB, bool COUNT>
__global__ void __launch_bounds__(kThreads, EMAX == 1 ? 6 : 2)
k_combine_group(const __grid_constant__ Params P)
{
    static_assert(KB <= kPad, "the list padding covers one load group");
    constexpr int kList = (EMAX > 1 ? kMaxPlanes : kMaxPartitions) + kPad;   // longest list
    __shared__ int64_t s_off[kList];
    __shared__ uint8_t s_emk[EMAX > 1 ? kList : 1];
    extern __shared__ uint4 s_dyn[];                          // [2][KB][kThreads] staging
    uint4 (*s_stage)[KB][kThreads] = reinterpret_cast<uint4 (*)[KB][kThreads]>(s_dyn);
    const int tid = threadIdx.x;
    // this CTA's units and the group holding the first one (the last i with unit_prefix[i]
    // <= u0, by binary search): kernel parameters only, found while the active sets build
    const int64_t cta = blockIdx.x;                           // balanced: q or q + 1 units
    const int64_t u0 = cta * P.q + min(cta, P.r);
    const int64_t u1 = u0 + P.q + (cta < P.r ? 1 : 0);
    int gi = 0;
    for (int lo = 0, hi = P.n - 1; lo <= hi;) {
        const int mid = (lo + hi) >> 1;
        if (P.unit_prefix[mid] <= u0) { gi = mid; lo = mid + 1; } else hi = mid - 1;
    }
    while (gi < P.n && P.unit_prefix[gi + 1] <= u0) ++gi;     // skip empty groups
    pdl_wait();                                               // active sets are visible
    unsigned bytes = 0;                                       // PDM bytes loaded (P.count)
    // bytes past the last whole chunk of each vectorised group: one warp per group
    for (int i = int(blockIdx.x) * (kThreads / 32) + (tid >> 5); i < P.n;
         i += int(gridDim.x) * (kThreads / 32))
        if (P.g[i].vec) group_tail<EMAX, COUNT>(P.g[i], tid & 31, bytes);
    int loaded = -1, n = 0;
    for (int64_t u = u0; u < u1; ++u) {
        while (P.unit_prefix[gi + 1] <= u) ++gi;
        const Group& g = P.g[gi];
        if (gi != loaded) {                                   // this group's planes
            if (loaded >= 0) __syncthreads();                 // the last group's offsets are read
            // the count and the first kThreads list entries in one round trip: every list
            // buffer holds at least kMaxPartitions + kPad >= kThreads entries
            const unsigned l0 = g.list[tid];
            const unsigned e0 = EMAX > 1 ? unsigned(g.emask[tid]) : 0u;
            n = *g.count;
            const int cap = min(n + kPad, kList);
            if (tid < cap) {
                s_off[tid] = int64_t(l0) * g.plane;
                if (EMAX > 1) s_emk[tid] = uint8_t(e0);
            }
            for (int j = tid + kThreads; j < cap; j += kThreads) {
                s_off[j] = int64_t(g.list[j]) * g.plane;
                if (EMAX > 1) s_emk[j] = g.emask[j];
            }
            __syncthreads();
            loaded = gi;
        }
        const int64_t lane_unit = (u - P.unit_prefix[gi]) * kThreads + tid;
        if (g.vec) {
            const int64_t nvec = g.G >> 4;
            if (lane_unit < nvec) {
                const uint8_t* src = g.pdm + (lane_unit << 4);
                GroupMin<EMAX> acc;
                acc.reset();
                const int nb = (n + KB - 1) / KB;
                if (nb > 0) {
                    for (int k = 0; k < KB; ++k) cp_async16(&s_stage[0][k][tid], src + s_off[k]);
                    asm volatile("cp.async.commit_group;" ::: "memory");
                    if (COUNT) bytes += 16u * unsigned(min(KB, n));
                }
                for (int b = 0; b < nb; ++b) {
                    // a chunk at 0 in every byte of every TF is final: its later planes are
                    // not loaded, and their stale slots fold into minima of 0
                    if (b + 1 < nb && acc.live(g.E)) {
                        for (int k = 0; k < KB; ++k)
                            cp_async16(&s_stage[(b + 1) & 1][k][tid], src + s_off[(b + 1) * KB + k]);
                        if (COUNT) bytes += 16u * unsigned(min(KB, n - (b + 1) * KB));
                    }
                    asm volatile("cp.async.commit_group;" ::: "memory");
                    asm volatile("cp.async.wait_group 1;" ::: "memory");
#pragma unroll
                    for (int k = 0; k < KB; ++k)
                        acc.fold(s_stage[b & 1][k][tid], EMAX > 1 ? unsigned(s_emk[b * KB + k]) : 1u);
                }
                asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
                for (int e = 0; e < EMAX; ++e)
                    if (EMAX == 1 || e < g.E)
                        __stcs(reinterpret_cast<uint4*>(g.out[e] + (lane_unit << 4)),
                               acc.acc[e].value());
            }
        } else if (lane_unit < g.G) {
            unsigned a[EMAX];
#pragma unroll
            for (int e = 0; e < EMAX; ++e) a[e] = 255;
            if (COUNT) bytes += unsigned(n);
            for (int j = 0; j < n; ++j) {
                const unsigned v = g.pdm[s_off[j] + lane_unit];
                const unsigned em = EMAX > 1 ? unsigned(s_emk[j]) : 1u;
#pragma unroll
                for (int e = 0; e < EMAX; ++e)
                    if ((em >> e) & 1u) a[e] = min(a[e], v);
            }
#pragma unroll
            for (int e = 0; e < EMAX; ++e)
                if (EMAX == 1 || e < g.E) g.out[e][lane_unit] = uint8_t(a[e]);
        }
    }
    if (COUNT) add_warp_count(P.count, bytes);
}

template <int EMAX, int KB, bool COUNT>
cudaError_t launch_combine_group_t(const Params& P, int64_t ctas, cudaStream_t s)
{
    const size_t smem = size_t(2) * KB * kThreads * sizeof(uint4);
    cudaError_t e = ensure_dynamic_smem<k_combine_group<EMAX, KB, COUNT>>(int(smem));
    if (e != cudaSuccess) return e;
    return launch_pdl(k_combine_group<EMAX, KB, COUNT>, dim3(unsigned(ctas)), dim3(kThreads),
                      smem, s, P);
}

template <int EMAX, int KB>
cudaError_t launch_combine_group(const Params& P, int64_t ctas, cudaStream_t s)
{
    return P.count ? launch_combine_group_t<EMAX, KB, true>(P, ctas, s)
                   : launch_combine_group_t<EMAX, KB, false>(P, ctas, s);
}

template <int EMAX>
cudaError_t launch_pair(const Params& P, int64_t ctas, int kb, cudaStream_t s)
{
    k_active_group<EMAX><<<P.n, kActThreads, 0, s>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return kb == 8 ? launch_combine_group<EMAX, 8>(P, ctas, s)
                   : launch_combine_group<EMAX, 4>(P, ctas, s);
}

}  // namespace

size_t batch_list_entries(int planes) { return size_t(planes) + kPad; }

cudaError_t launch_update_batch(const BatchGroup* groups, int n, const BatchTuning& tune,
                                int num_sms, unsigned long long* count, cudaStream_t s)
{
    if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
    Params P;
    P.n = n;
    P.count = count;
    P.unit_prefix[0] = 0;
    int emax = 1;
    for (int i = 0; i < n; ++i) {
        const BatchGroup& d = groups[i];
        if (d.E < 1 || d.E > kMaxGroupEdits) return cudaErrorInvalidValue;
        Group& g = P.g[i];
        g.pdm = d.pdm;
        g.plane = d.plane;
        g.G = d.G;
        g.lut = d.lut;
        g.order = d.order;
        g.list = d.list;
        g.emask = d.emask;
        g.count = d.count;
        g.N = d.N;
        g.K = d.K;
        g.J = d.J;
        g.E = d.E;
        bool vec = ((reinterpret_cast<uintptr_t>(d.pdm) & 15) == 0) && (d.plane % 16 == 0);
        for (int e = 0; e < kMaxGroupEdits; ++e) {
            g.tf[e] = e < d.E ? d.tf[e] : nullptr;
            g.out[e] = e < d.E ? d.out[e] : nullptr;
            if (e < d.E) vec = vec && ((reinterpret_cast<uintptr_t>(d.out[e]) & 15) == 0);
        }
        g.vec = vec ? 1 : 0;
        if (d.E > emax) emax = d.E;
        const int64_t units = g.vec ? (d.G >> 4) : d.G;
        P.unit_prefix[i + 1] = P.unit_prefix[i] + (units + kThreads - 1) / kThreads + (units == 0);
    }
    const int64_t total = P.unit_prefix[n];
    // many small CTAs (32 KiB of staging each, 6 resident per SM) over 4 KiB units,
    // by default one unit each on batches of up to 24 units per SM: the hardware's CTA
    // scheduling balances groups of different cost
    int64_t ctas = int64_t(num_sms > 0 ? num_sms : 152) *
                   (tune.ctas_per_sm > 0 ? tune.ctas_per_sm : 24);
    if (ctas > total) ctas = total;
    P.q = total / ctas;
    P.r = total % ctas;
    const int kb = tune.loads_per_stage == 8 ? 8 : 4;
    if (emax == 1) return launch_pair<1>(P, ctas, kb, s);
    if (emax == 2) return launch_pair<2>(P, ctas, kb, s);
    if (emax <= 4) return launch_pair<4>(P, ctas, kb, s);
    return launch_pair<8>(P, ctas, kb, s);
}

}  // namespace dmk
