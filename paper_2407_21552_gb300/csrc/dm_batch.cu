// dm_batch.cu -- the per-TF update for many volumes at once.
//
// Each item is one volume's resident PDMs (§3.1) with its own TF.  Two launches cover up
// to kMaxBatch items: an active-set kernel with one CTA per item (§3.1 step 1, from the
// item's partition table built at precompute time; all loads of a batch issued before any
// is used), then a combine (Eq. 1) over one flattened list of 4 KiB work units of all
// items, launched with programmatic dependent launch; by default each combine CTA takes
// one unit.  The bytes past an item's last whole 16-byte chunk are folded by one warp per
// item, its lanes over the planes.  Per-item descriptors are passed by value as kernel
// parameters, so the pair needs no device-side setup and can be captured in a CUDA graph.
#include "dm_internal.cuh"

namespace dmk {
namespace {

constexpr int kActThreads = 1024;
constexpr int kThreads = 256;                  // combine CTA; one work unit = 256 x 16 B

struct Item {
    const uint8_t* pdm;
    int64_t plane;
    int64_t G;
    const float* tf;
    uint8_t* out;
    const uint8_t* lut;                        // partition of each intensity (precompute)
    uint16_t* act;                             // active list and count (item's scratch)
    int32_t* nact;
    int32_t N, K, J;                           // J: index levels (-1: none)
    int32_t vec;                               // 16-byte units (else bytes)
};

struct Params {
    int n;
    int64_t q, r;                              // CTA b takes q units, plus one if b < r
    int64_t unit_prefix[kMaxBatch + 1];        // work units before item i (256 lanes each)
    Item it[kMaxBatch];
};

__device__ __forceinline__ void cp_async16(void* smem, const uint8_t* gmem)
{
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global.L2::256B [%0], [%1], 16;" ::"r"(sa), "l"(gmem)
                 : "memory");
}

// §3.1 step 1 for item blockIdx.x: partition lut[i] is active when alpha_i > 0.  A warp
// holds 32 consecutive intensities, so its visible partitions fall in few mask words: it
// ORs each word over the warp and one lane sets it, with no same-address shared atomics
// between the lanes.  The list is followed by kPad copies of its first entry, so that the
// combine can read it in groups of kPad without knowing its length first.
constexpr int kPad = 4;

__global__ void __launch_bounds__(kActThreads) k_active_batch(const __grid_constant__ Params P)
{
    pdl_trigger();
    __shared__ uint32_t s_S[kMaxPartitions / 32];
    __shared__ uint16_t s_list[kMaxPartitions + 8];
    __shared__ int s_scan[9];
    const Item& it = P.it[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < kMaxPartitions / 32) s_S[tid] = 0;
    __syncthreads();
    constexpr int kLB = 8;                                    // loads issued before any use
    for (int base = 0; base < it.N; base += kActThreads * kLB) {
        float a[kLB];
        uint8_t c[kLB];
#pragma unroll
        for (int k = 0; k < kLB; ++k) {
            const int i = base + k * kActThreads + tid;
            a[k] = i < it.N ? __ldg(it.tf + 4 * int64_t(i) + 3) : 0.0f;
            c[k] = i < it.N ? it.lut[i] : uint8_t(0);
        }
#pragma unroll
        for (int k = 0; k < kLB; ++k) {
            const bool vis = a[k] > 0.0f;
            const unsigned w = c[k] >> 5;
            const unsigned wlo = __reduce_min_sync(0xFFFFFFFFu, vis ? w : 8u);
            const unsigned whi = __reduce_max_sync(0xFFFFFFFFu, vis ? w : 0u);
            for (unsigned ww = wlo; ww <= whi; ++ww) {        // usually one word
                const unsigned bit = (vis && w == ww) ? 1u << (c[k] & 31) : 0u;
                const unsigned m = __reduce_or_sync(0xFFFFFFFFu, bit);
                if (lane == 0 && m) atomicOr(&s_S[ww], m);
            }
        }
    }
    __syncthreads();
    const int n = plan_maps(s_S, it.K, it.J, s_list, s_scan);
    for (int j = tid; j < n + kPad; j += kActThreads)
        it.act[j] = n ? s_list[j < n ? j : 0] : uint16_t(0);
    if (tid == 0) *it.nact = n;
}

// Bytes past the last whole 16-byte chunk of an item (fewer than 16): one warp, the lanes
// over the item's active planes, then a warp min per byte.
__device__ __forceinline__ void item_tail(const Item& it, int lane)
{
    const int64_t g0 = (it.G >> 4) << 4;
    const int rem = int(it.G - g0);
    if (rem == 0) return;                                     // warp-uniform
    const int n = *it.nact;
    unsigned m[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) m[r] = 255;
    for (int j = lane; j < n; j += 32) {
        const uint8_t* src = it.pdm + int64_t(it.act[j]) * it.plane + g0;
#pragma unroll
        for (int r = 0; r < 16; ++r)
            if (r < rem) m[r] = min(m[r], unsigned(src[r]));
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        if (r < rem) {
            const unsigned v = __reduce_min_sync(0xFFFFFFFFu, m[r]);
            if (lane == 0) it.out[g0 + r] = uint8_t(v);
        }
    }
}

// Eq. 1 over every item's work units; CTA b takes a contiguous range of units.  At most 40
// registers a thread, so that 6 CTAs fit an SM next to their 6 x 34 KiB of shared memory.
__global__ void __launch_bounds__(kThreads, 6) k_combine_batch(const __grid_constant__ Params P)
{
    constexpr int kB = 4;                                     // plane loads per group
    static_assert(kB == kPad, "the list padding covers one load group");
    __shared__ int64_t s_off[kMaxPartitions + kB];
    extern __shared__ uint4 s_dyn[];                          // [2][kB][kThreads] staging
    uint4 (*s_stage)[kB][kThreads] = reinterpret_cast<uint4 (*)[kB][kThreads]>(s_dyn);
    const int tid = threadIdx.x;
    // this CTA's units and the item holding the first one (the last i with unit_prefix[i]
    // <= u0, by binary search): kernel parameters only, found while the active sets build
    const int64_t cta = blockIdx.x;                           // balanced: q or q + 1 units
    const int64_t u0 = cta * P.q + min(cta, P.r);
    const int64_t u1 = u0 + P.q + (cta < P.r ? 1 : 0);
    int item = 0;
    for (int lo = 0, hi = P.n - 1; lo <= hi;) {
        const int mid = (lo + hi) >> 1;
        if (P.unit_prefix[mid] <= u0) { item = mid; lo = mid + 1; } else hi = mid - 1;
    }
    while (item < P.n && P.unit_prefix[item + 1] <= u0) ++item;   // skip empty items
    pdl_wait();                                               // active sets are visible
    // bytes past the last whole chunk of each vectorised item: one warp per item
    for (int i = int(blockIdx.x) * (kThreads / 32) + (tid >> 5); i < P.n;
         i += int(gridDim.x) * (kThreads / 32))
        if (P.it[i].vec) item_tail(P.it[i], tid & 31);
    int loaded = -1, n = 0;
    for (int64_t u = u0; u < u1; ++u) {
        while (P.unit_prefix[item + 1] <= u) ++item;
        const Item& it = P.it[item];
        if (item != loaded) {                                 // this item's active planes
            if (loaded >= 0) __syncthreads();                 // the last item's offsets are read
            n = *it.nact;                                     // issued with the list loads
            for (int j = tid; j < kMaxPartitions + kB; j += kThreads)
                s_off[j] = int64_t(it.act[j]) * it.plane;     // only [0, n + kB) is ever used
            __syncthreads();
            loaded = item;
        }
        const int64_t lane_unit = (u - P.unit_prefix[item]) * kThreads + tid;
        if (it.vec) {
            const int64_t nvec = it.G >> 4;
            if (lane_unit < nvec) {
                const uint8_t* src = it.pdm + (lane_unit << 4);
                ByteMin16 acc;
                acc.reset();
                const int nb = (n + kB - 1) / kB;
                if (nb > 0) {
                    for (int k = 0; k < kB; ++k) cp_async16(&s_stage[0][k][tid], src + s_off[k]);
                    asm volatile("cp.async.commit_group;" ::: "memory");
                }
                for (int b = 0; b < nb; ++b) {
                    if (b + 1 < nb)
                        for (int k = 0; k < kB; ++k)
                            cp_async16(&s_stage[(b + 1) & 1][k][tid], src + s_off[(b + 1) * kB + k]);
                    asm volatile("cp.async.commit_group;" ::: "memory");
                    asm volatile("cp.async.wait_group 1;" ::: "memory");
#pragma unroll
                    for (int k = 0; k < kB; ++k) acc.fold(s_stage[b & 1][k][tid]);
                }
                asm volatile("cp.async.wait_group 0;" ::: "memory");
                __stcs(reinterpret_cast<uint4*>(it.out + (lane_unit << 4)), acc.value());
            }
        } else if (lane_unit < it.G) {
            unsigned a = 255;
            for (int j = 0; j < n; ++j) a = min(a, unsigned(it.pdm[s_off[j] + lane_unit]));
            it.out[lane_unit] = uint8_t(a);
        }
    }
}

}  // namespace

cudaError_t launch_update_batch(const BatchDesc* items, int n, int ctas_per_sm, int num_sms,
                                cudaStream_t s)
{
    if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
    Params P;
    P.n = n;
    P.unit_prefix[0] = 0;
    for (int i = 0; i < n; ++i) {
        const BatchDesc& d = items[i];
        Item& it = P.it[i];
        it.pdm = d.pdm;
        it.plane = d.plane;
        it.G = d.G;
        it.tf = d.tf;
        it.out = d.out;
        it.lut = d.lut;
        it.act = d.act;
        it.nact = d.nact;
        it.N = d.N;
        it.K = d.K;
        it.J = d.J;
        it.vec = ((reinterpret_cast<uintptr_t>(d.pdm) & 15) == 0) &&
                 ((reinterpret_cast<uintptr_t>(d.out) & 15) == 0) && (d.plane % 16 == 0);
        const int64_t units = it.vec ? (d.G >> 4) : d.G;
        P.unit_prefix[i + 1] = P.unit_prefix[i] + (units + kThreads - 1) / kThreads + (units == 0);
    }
    k_active_batch<<<n, kActThreads, 0, s>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = P.unit_prefix[n];
    // many small CTAs (32 KiB of staging each, 6 resident per SM) over 4 KiB units,
    // by default one unit each on batches of up to 24 units per SM: the hardware's CTA
    // scheduling balances items of different cost
    int64_t ctas = int64_t(num_sms > 0 ? num_sms : 152) * (ctas_per_sm > 0 ? ctas_per_sm : 24);
    if (ctas > total) ctas = total;
    P.q = total / ctas;
    P.r = total % ctas;
    const size_t smem = size_t(2) * 4 * kThreads * sizeof(uint4);
    e = ensure_dynamic_smem<k_combine_batch>(int(smem));
    if (e != cudaSuccess) return e;
    return launch_pdl(k_combine_batch, dim3(unsigned(ctas)), dim3(kThreads), smem, s, P);
}

}  // namespace dmk
