// dm_noalloc.cu -- a per-TF update for callers that cannot allocate device memory.
//
// dm_update_tf needs a small device scratch buffer (active list, count, active bit set)
// that the caller allocates and binds to a context.  Some callers cannot do that: a
// plug-in running inside a host renderer that owns every device allocation and hands out
// only the buffers it manages, or an interactive render loop that must not call cudaMalloc
// between frames because an allocation can synchronize the device and stall the frame.
// dm_update_tf_noalloc needs no context and no scratch from the caller: its working memory
// is a fixed-size array in the library's own device memory (g_noalloc_scratch below),
// which every GPU that loads the library holds until the process exits.  The caller still
// passes the PDM planes, the TF and the output map.
//
// Host code cannot use the array's name as a device address (on the host it names a
// stand-in), so the first call on each device looks up the real address with
// cudaGetSymbolAddress, with that device current, and caches it.
//
// All calls share the one array and it keeps the last call's contents.  The active-set
// kernel writes every word that the combine later reads (each visibility word, the count
// and the list entries below the count), so nothing needs clearing between calls.  Two
// calls whose work overlaps on the GPU (different streams, no ordering) race on the array.
// The cached address belongs to the device's current context: after cudaDeviceReset the
// library's module is loaded again and the array may move, so the cache is not valid
// across a reset.
#include <mutex>

#include "../../include/dm.h"
#include "dm_internal.cuh"

namespace {

constexpr int kMaxDevices = 64;
constexpr int kThreads = 1024;
// layout of the static array
constexpr size_t kOffCount = 0;                   // int32: number of active partitions
constexpr size_t kOffAct = 128;                   // uint16[256]: ascending active list
constexpr size_t kOffVis = 1024;                  // uint32[N/32]: visibility bits
static_assert(kOffAct + 2 * dmk::kMaxPartitions <= kOffVis, "active list overlaps");
static_assert(kOffVis + DM_NOALLOC_MAX_TF_SIZE / 8 <= DM_NOALLOC_SCRATCH_BYTES,
              "visibility bits do not fit the static scratch");

static __device__ __align__(256) unsigned char g_noalloc_scratch[DM_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
unsigned char* g_addr[kMaxDevices];               // device address per device ordinal

// Step 1 of §3.1 with the working memory in `scratch`: visibility bits by warp ballots,
// then partition p is active iff a bit in [lo_p, hi_p] is set; compacted ascending.
__global__ void __launch_bounds__(kThreads)
k_noalloc_active(const float* __restrict__ tf, int N, int K, dmk::Borders bd,
                 unsigned char* scratch)
{
    __shared__ int s_cnt[8];
    uint32_t* vis = reinterpret_cast<uint32_t*>(scratch + kOffVis);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int base = 0; base < N; base += kThreads) {
        const int i = base + tid;
        const bool v = i < N && __ldg(tf + 4 * int64_t(i) + 3) > 0.0f;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, v);
        if (lane == 0 && base + warp * 32 < N) vis[(base >> 5) + warp] = bal;
    }
    __syncthreads();
    bool on = false;
    const int p = tid;
    if (p < K) {
        const int lo = bd.v[p], hi = bd.v[p + 1] - 1;
        for (int w = lo >> 5; w <= (hi >> 5) && !on; ++w) {
            uint32_t m = vis[w];
            if (w == (lo >> 5)) m &= 0xFFFFFFFFu << (lo & 31);
            if (w == (hi >> 5)) m &= 0xFFFFFFFFu >> (31 - (hi & 31));
            on = m != 0;
        }
    }
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, on);
    if (lane == 0 && warp < 8) s_cnt[warp] = __popc(bal);
    __syncthreads();
    if (tid < 256) {
        int off = 0;
        for (int w = 0; w < warp; ++w) off += s_cnt[w];
        uint16_t* act = reinterpret_cast<uint16_t*>(scratch + kOffAct);
        if (on) act[off + __popc(bal & ((1u << lane) - 1))] = uint16_t(p);
        if (tid == 0) {
            int tot = 0;
            for (int w = 0; w < 8; ++w) tot += s_cnt[w];
            *reinterpret_cast<int32_t*>(scratch + kOffCount) = tot;
        }
    }
}

// Device address of the static array on the current device, looked up once per device.
dm_status scratch_on_current_device(unsigned char** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return DM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return DM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DM_ERR_CUDA;
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return DM_OK;
}

}  // namespace

extern "C" dm_status dm_update_tf_noalloc(const uint8_t* d_pdm, size_t plane_stride,
                                          int64_t num_blocks, int32_t num_partitions,
                                          const int32_t* borders, int32_t tf_size,
                                          const float* d_tf_rgba, uint8_t* d_out, void* stream)
{
    const int K = num_partitions, N = tf_size;
    if (!d_pdm || !d_tf_rgba || !d_out || num_blocks < 1 || K < 1 || N < 2 || K > N ||
        plane_stride < size_t(num_blocks) || (reinterpret_cast<uintptr_t>(d_tf_rgba) & 3))
        return DM_ERR_INVALID_ARG;
    if (K > DM_MAX_PARTITIONS || N > DM_NOALLOC_MAX_TF_SIZE) return DM_ERR_UNSUPPORTED;
    dmk::Borders bd;
    for (int p = 0; p <= K; ++p) bd.v[p] = borders ? borders[p] : int32_t((int64_t(p) * N) / K);
    if (bd.v[0] != 0 || bd.v[K] != N) return DM_ERR_INVALID_ARG;
    for (int p = 0; p < K; ++p)
        if (bd.v[p + 1] <= bd.v[p]) return DM_ERR_INVALID_ARG;
    for (int p = K + 1; p <= dmk::kMaxPartitions; ++p) bd.v[p] = N;
    unsigned char* scratch = nullptr;
    dm_status st = scratch_on_current_device(&scratch);
    if (st != DM_OK) return st;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DM_ERR_CUDA;
    // An error left by earlier work of the caller is reported, not cleared: it stays with
    // the caller, and only a failure of the launches below is this call's own.
    if (cudaPeekAtLastError() != cudaSuccess) return DM_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_noalloc_active<<<1, kThreads, 0, s>>>(d_tf_rgba, N, K, bd, scratch);
    if (cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();
        return DM_ERR_CUDA;
    }
    cudaError_t e = dmk::launch_combine(d_pdm, int64_t(plane_stride), num_blocks,
                                        reinterpret_cast<const uint16_t*>(scratch + kOffAct),
                                        reinterpret_cast<const int32_t*>(scratch + kOffCount),
                                        d_out, sms, nullptr, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DM_ERR_CUDA;
    }
    return DM_OK;
}
