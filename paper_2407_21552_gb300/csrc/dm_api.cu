// dm_api.cu -- the C ABI of libdm (declared in include/dm.h).
//
// Host-side validation, buffer bookkeeping and launch sequencing.  Every step of the
// method runs in the kernels of dm_footprint.cu, dm_dt.cu and dm_update.cu; this file only
// checks arguments, lays out the caller's scratch buffer and enqueues work on the caller's
// stream.  No device memory is allocated here.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/dm.h"
#include "dm_build_batch.cuh"
#include "dm_internal.cuh"

struct dm_ctx {
    dm_config cfg;
    dmk::Borders borders;
    bool uniform_borders;           // borders[p] == floor(p N / K) for every p
    dmk::Geometry geo;
    dm_sizes sizes;
    int W;
    int J;                          // range-index levels (-1: none)
    int planes;                     // planes in the pdm buffer
    int num_sms;
    // scratch layout (byte offsets)
    size_t off_lut, off_cnt, off_act, off_nact, off_smask, off_cover, off_order, off_rmin, off_tf,
        off_out;
    bool rows_ok;                   // region bounds from the masks' rows (the single build)
    size_t off_proj, off_d2;        // their scratch (rows_ok)
    void* d_mask;
    void* d_pdm;
    void* d_minmax;
    void* d_scratch;
    bool built;
    bool minmax_built;
    cudaEvent_t ev_begin, ev_end;   // optional, caller-owned (dm_set_profile_events)
    uint64_t* prof_bytes;           // optional, caller-owned (dm_set_profile_counter)
    char err[256];
};

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

dm_status fail(dm_ctx* c, dm_status s, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

dm_status cuda_fail(dm_ctx* c, cudaError_t e, const char* where)
{
    return fail(c, DM_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// Report an earlier asynchronous error without clearing it from a healthy context.
dm_status check_sticky(dm_ctx* c, const char* where)
{
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(c, e, where);
    }
    return DM_OK;
}

}  // namespace

extern "C" {

int32_t dm_version(void) { return 10000; }

const char* dm_status_string(dm_status s)
{
    switch (s) {
    case DM_OK: return "DM_OK";
    case DM_ERR_INVALID_ARG: return "DM_ERR_INVALID_ARG";
    case DM_ERR_UNSUPPORTED: return "DM_ERR_UNSUPPORTED";
    case DM_ERR_CUDA: return "DM_ERR_CUDA";
    case DM_ERR_NOT_BOUND: return "DM_ERR_NOT_BOUND";
    default: return "DM_ERR_UNKNOWN";
    }
}

const char* dm_last_error_string(const dm_ctx* ctx) { return ctx ? ctx->err : "null context"; }

dm_status dm_create(dm_ctx** out, const dm_config* cfg)
{
    if (!out || !cfg) return DM_ERR_INVALID_ARG;
    *out = nullptr;
    const dm_config& c = *cfg;
    for (int i = 0; i < 3; ++i)
        if (c.dims[i] < 1) return DM_ERR_INVALID_ARG;
    if (c.dtype != DM_U8 && c.dtype != DM_U16) return DM_ERR_INVALID_ARG;
    if (c.block < 1 || c.apron < 0) return DM_ERR_INVALID_ARG;
    if (c.block > DM_MAX_BLOCK || c.apron > c.block) return DM_ERR_UNSUPPORTED;
    if (c.num_partitions < 1 || c.tf_size < 2) return DM_ERR_INVALID_ARG;
    if (c.num_partitions > DM_MAX_PARTITIONS || c.tf_size > DM_MAX_TF_SIZE)
        return DM_ERR_UNSUPPORTED;
    if (c.num_partitions > c.tf_size) return DM_ERR_INVALID_ARG;
    if (c.occ_mode != DM_OCC_MINMAX && c.occ_mode != DM_OCC_EXACT) return DM_ERR_INVALID_ARG;
    if (c.index_mode != DM_INDEX_NONE && c.index_mode != DM_INDEX_RANGES) return DM_ERR_INVALID_ARG;
    const int K = c.num_partitions, N = c.tf_size;
    if (c.borders) {
        if (c.borders[0] != 0 || c.borders[K] != N) return DM_ERR_INVALID_ARG;
        for (int p = 0; p < K; ++p)
            if (c.borders[p + 1] <= c.borders[p]) return DM_ERR_INVALID_ARG;
    }
    dm_ctx* x = new (std::nothrow) dm_ctx();
    if (!x) return DM_ERR_INVALID_ARG;
    x->cfg = c;
    x->cfg.borders = nullptr;
    for (int p = 0; p <= K; ++p)
        x->borders.v[p] = c.borders ? c.borders[p] : int32_t((int64_t(p) * N) / K);
    for (int p = K + 1; p <= dmk::kMaxPartitions; ++p) x->borders.v[p] = N;
    x->uniform_borders = true;
    for (int p = 0; p <= K; ++p)
        x->uniform_borders &= x->borders.v[p] == int32_t((int64_t(p) * N) / K);
    dmk::Geometry& g = x->geo;
    g.X = c.dims[0];
    g.Y = c.dims[1];
    g.Z = c.dims[2];
    g.b = c.block;
    g.a = c.apron;
    g.bpv = c.dtype;
    g.gx = (g.X + g.b - 1) / g.b;
    g.gy = (g.Y + g.b - 1) / g.b;
    g.gz = (g.Z + g.b - 1) / g.b;
    g.G = int64_t(g.gx) * g.gy * g.gz;
    g.plane = int64_t(align_up(size_t(g.G), 64));
    x->W = (K + 63) / 64;
    x->J = c.index_mode == DM_INDEX_RANGES ? dmk::index_levels(K) : -1;
    x->planes = x->J < 0 ? K : dmk::index_level_base(K, x->J + 1);
    // limits of the kernels' tilings
    if (g.gx > 10240 || dmk::xpass_smem(g.gx, K) > size_t(dmk::kXpassSmemLimit) ||
        dmk::line_pass_smem(g.gy) > size_t(dmk::kLineSmemLimit) ||
        dmk::line_pass_smem(g.gz) > size_t(dmk::kLineSmemLimit) || g.gz > 65535 ||
        g.gy > 65535) {
        delete x;
        return DM_ERR_UNSUPPORTED;
    }
    dm_sizes& s = x->sizes;
    s.mask_bytes = size_t(g.G) * x->W * 8;
    s.plane_stride = size_t(g.plane);
    s.pdm_bytes = size_t(x->planes) * s.plane_stride;
    s.pdm_planes = x->planes;
    s.minmax_bytes = size_t(g.G) * 2 * g.bpv;
    s.out_bytes = size_t(g.G);
    s.grid[0] = g.gx;
    s.grid[1] = g.gy;
    s.grid[2] = g.gz;
    s.mask_words = x->W;
    size_t o = 0;
    x->off_lut = o;   o = align_up(o + size_t(N), 256);
    x->off_cnt = o;   o = align_up(o + size_t(N + 1) * 4, 256);
    x->off_act = o;   o = align_up(o + size_t(dmk::kMaxPartitions + 8) * 2, 256);
    x->off_nact = o;  o = align_up(o + 64, 64);
    x->off_smask = o; o = align_up(o + 64, 256);
    x->off_cover = o; o = align_up(o + size_t(dmk::kMaxPartitions) * dmk::kCoverSplit * 4, 256);
    x->off_order = o; o = align_up(o + size_t(dmk::kMaxPartitions) * 2, 256);
    x->off_rmin = o;  o = align_up(o + size_t(dmk::num_regions(g.G)) * size_t(K), 256);
    x->off_tf = o;    o = align_up(o + size_t(N) * 16, 256);
    x->off_out = o;   o = align_up(o + size_t(g.G), 256);
    x->rows_ok = dmk::bounds_from_rows_ok(g, K);
    x->off_proj = o;
    if (x->rows_ok) o = align_up(o + dmk::bounds_rows_proj_bytes(g, K), 256);
    x->off_d2 = o;
    if (x->rows_ok) o = align_up(o + dmk::bounds_rows_d2_bytes(g, K), 256);
    s.scratch_bytes = o;
    int dev = 0;
    x->num_sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            x->num_sms = n;
    }
    cudaGetLastError();   // no GPU is not an error at create time
    x->err[0] = 0;
    *out = x;
    return DM_OK;
}

dm_status dm_query_sizes(const dm_ctx* ctx, dm_sizes* out)
{
    if (!ctx || !out) return DM_ERR_INVALID_ARG;
    *out = ctx->sizes;
    return DM_OK;
}

dm_status dm_bind(dm_ctx* ctx, void* d_mask, void* d_pdm, void* d_minmax, void* d_scratch)
{
    if (!ctx) return DM_ERR_INVALID_ARG;
    if ((d_mask && !aligned(d_mask, 16)) || (d_pdm && !aligned(d_pdm, 16)) ||
        (d_minmax && !aligned(d_minmax, 16)) || (d_scratch && !aligned(d_scratch, 256)))
        return fail(ctx, DM_ERR_INVALID_ARG, "dm_bind: misaligned buffer (mask/pdm/minmax need "
                    "16 bytes, scratch 256)");
    // the scratch holds the partition table that dm_build_partitions / dm_mark_built write:
    // another pdm or scratch buffer needs one of them again
    if (d_pdm != ctx->d_pdm || d_scratch != ctx->d_scratch) ctx->built = false;
    if (d_minmax != ctx->d_minmax) ctx->minmax_built = false;
    ctx->d_mask = d_mask;
    ctx->d_pdm = d_pdm;
    ctx->d_minmax = d_minmax;
    ctx->d_scratch = d_scratch;
    ctx->err[0] = 0;
    return DM_OK;
}

// The plane order of a context (in its scratch, next to the partition table): written by
// dm_build_partitions, dm_build_partitions_batch and dm_mark_built, read by the updates.
static dmk::PlaneOrderItem plane_order_item(const dm_ctx* c)
{
    uint8_t* scratch = static_cast<uint8_t*>(c->d_scratch);
    dmk::PlaneOrderItem it;
    it.pdm = static_cast<const uint8_t*>(c->d_pdm);
    it.plane = c->geo.plane;
    it.G = c->geo.G;
    it.K = c->cfg.num_partitions;
    it.cover = reinterpret_cast<uint32_t*>(scratch + c->off_cover);
    it.order = reinterpret_cast<uint16_t*>(scratch + c->off_order);
    it.rmin = scratch + c->off_rmin;
    it.bounds_from_planes = 1;
    return it;
}

static unsigned long long* prof_count(const dm_ctx* c)
{
    static_assert(sizeof(unsigned long long) == sizeof(uint64_t), "64-bit counter");
    return reinterpret_cast<unsigned long long*>(c->prof_bytes);
}

static const uint8_t* region_bounds(const dm_ctx* c)
{
    return static_cast<const uint8_t*>(c->d_scratch) + c->off_rmin;
}

static const uint16_t* plane_order(const dm_ctx* c)
{
    return reinterpret_cast<const uint16_t*>(static_cast<const uint8_t*>(c->d_scratch) +
                                             c->off_order);
}

// Uniform partitions of a power-of-two width: the partition of intensity i is i >> shift.
// Else -1.
static int pom_shift(const dm_ctx* c)
{
    const int K = c->cfg.num_partitions, N = c->cfg.tf_size;
    if (!c->uniform_borders || N % K != 0 || ((N / K) & (N / K - 1)) != 0) return -1;
    int shift = 0;
    while ((1 << shift) < N / K) ++shift;
    return shift;
}

dm_status dm_build_partitions(dm_ctx* ctx, const void* d_volume, void* stream)
{
    if (!ctx) return DM_ERR_INVALID_ARG;
    if (!d_volume || !aligned(d_volume, size_t(ctx->geo.bpv)))
        return fail(ctx, DM_ERR_INVALID_ARG, "dm_build_partitions: null or misaligned volume");
    if (!ctx->d_mask || !ctx->d_pdm || !ctx->d_scratch)
        return fail(ctx, DM_ERR_NOT_BOUND, "dm_build_partitions: mask, pdm and scratch must be bound");
    dm_status st = check_sticky(ctx, "dm_build_partitions (earlier work)");
    if (st != DM_OK) return st;
    const int K = ctx->cfg.num_partitions, N = ctx->cfg.tf_size;
    cudaStream_t s = as_stream(stream);
    uint8_t* scratch = static_cast<uint8_t*>(ctx->d_scratch);
    uint8_t* lut = scratch + ctx->off_lut;
    uint8_t* pdm = static_cast<uint8_t*>(ctx->d_pdm);
    cudaError_t e = dmk::launch_partition_lut(lut, N, K, ctx->borders, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "partition table");
    const int shift = pom_shift(ctx);
    e = dmk::launch_pom_build(d_volume, ctx->geo, N, K, lut, static_cast<uint64_t*>(ctx->d_mask),
                              ctx->d_minmax, shift, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "POM build");
    uint64_t* proj = reinterpret_cast<uint64_t*>(scratch + ctx->off_proj);
    bool projected = false;                  // the row ORs for the region bounds, if taken
    e = dmk::launch_xpass_mask(static_cast<const uint64_t*>(ctx->d_mask), K, ctx->geo, pdm, s,
                               ctx->rows_ok ? proj : nullptr, &projected);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "PDM x pass");
    e = dmk::launch_line_pass(pdm, K, ctx->geo.plane, ctx->geo, 1, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "PDM y pass");
    e = dmk::launch_line_pass(pdm, K, ctx->geo.plane, ctx->geo, 2, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "PDM z pass");
    dmk::PlaneOrderItem po = plane_order_item(ctx);
    po.bounds_from_planes = ctx->rows_ok ? 0 : 1;
    e = dmk::launch_plane_order(&po, 1, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plane order");
    if (ctx->rows_ok) {
        e = dmk::launch_bounds_from_rows(static_cast<const uint64_t*>(ctx->d_mask), ctx->geo, K,
                                         proj, projected, scratch + ctx->off_d2,
                                         scratch + ctx->off_rmin, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "region bounds");
    }
    if (ctx->J > 0) {
        e = dmk::launch_build_index(pdm, ctx->geo.plane, ctx->geo.G, K, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "range index");
    }
    ctx->built = true;
    ctx->minmax_built = ctx->d_minmax != nullptr;
    ctx->err[0] = 0;
    return DM_OK;
}

// Host checks of a batched precompute: every context bound, every volume aligned, no
// context twice and no buffer bound to two contexts (by sorting the buffer addresses).
static dm_status check_build_batch(dm_ctx* const* ctxs, const void* const* vols, int32_t n)
{
    for (int32_t i = 0; i < n; ++i)        // a refusal leaves its message in one context only
        if (ctxs[i]) ctxs[i]->err[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        dm_ctx* c = ctxs[i];
        if (!c)
            return ctxs[0] ? fail(ctxs[0], DM_ERR_INVALID_ARG, "dm_build_partitions_batch: item "
                                  "%d: null context", i) : DM_ERR_INVALID_ARG;
        if (!vols[i] || !aligned(vols[i], size_t(c->geo.bpv)))
            return fail(c, DM_ERR_INVALID_ARG, "dm_build_partitions_batch: item %d: null or "
                        "misaligned volume", i);
        if (!c->d_mask || !c->d_pdm || !c->d_scratch)
            return fail(c, DM_ERR_NOT_BOUND, "dm_build_partitions_batch: item %d: mask, pdm and "
                        "scratch must be bound", i);
    }
    struct Buf {
        uintptr_t p;
        int32_t item;
    };
    Buf* bufs = new (std::nothrow) Buf[size_t(n) * 5];
    if (!bufs)
        return fail(ctxs[0], DM_ERR_INVALID_ARG, "dm_build_partitions_batch: out of host memory");
    size_t nb = 0;
    for (int32_t i = 0; i < n; ++i) {
        const dm_ctx* c = ctxs[i];
        // the context itself counts as a buffer, so that a context listed twice is caught
        const void* own[5] = {c, c->d_mask, c->d_pdm, c->d_scratch, c->d_minmax};
        for (const void* p : own)
            if (p) bufs[nb++] = Buf{reinterpret_cast<uintptr_t>(p), i};
    }
    std::sort(bufs, bufs + nb, [](const Buf& a, const Buf& b) {
        return a.p < b.p || (a.p == b.p && a.item < b.item);
    });
    dm_status st = DM_OK;
    for (size_t k = 1; k < nb && st == DM_OK; ++k)
        if (bufs[k].p == bufs[k - 1].p && bufs[k].item != bufs[k - 1].item)
            st = fail(ctxs[bufs[k].item], DM_ERR_INVALID_ARG, "dm_build_partitions_batch: items "
                      "%d and %d share a context or a buffer", bufs[k - 1].item, bufs[k].item);
    delete[] bufs;
    return st;
}

dm_status dm_build_partitions_batch(dm_ctx* const* ctxs, const void* const* d_volumes, int32_t n,
                                    void* stream)
{
    if (!ctxs || !d_volumes || n < 0) return DM_ERR_INVALID_ARG;
    if (n == 0) return DM_OK;
    dm_status st = check_build_batch(ctxs, d_volumes, n);
    if (st != DM_OK) return st;
    st = check_sticky(ctxs[0], "dm_build_partitions_batch (earlier work)");
    if (st != DM_OK) return st;
    cudaStream_t s = as_stream(stream);
    dmk::BuildItem items[dmk::kMaxBuildBatch];
    for (int32_t i0 = 0; i0 < n; i0 += dmk::kMaxBuildBatch) {
        const int m = (n - i0) < dmk::kMaxBuildBatch ? (n - i0) : dmk::kMaxBuildBatch;
        for (int k = 0; k < m; ++k) {
            dm_ctx* c = ctxs[i0 + k];
            dmk::BuildItem& b = items[k];
            b.vol = d_volumes[i0 + k];
            b.g = c->geo;
            b.N = c->cfg.tf_size;
            b.K = c->cfg.num_partitions;
            b.shift = pom_shift(c);
            b.borders = &c->borders;
            b.lut = static_cast<uint8_t*>(c->d_scratch) + c->off_lut;
            b.mask = static_cast<uint64_t*>(c->d_mask);
            b.minmax = c->d_minmax;
            b.pdm = static_cast<uint8_t*>(c->d_pdm);
            c->built = false;
            c->minmax_built = false;
        }
        dm_ctx* first = ctxs[i0];
        cudaError_t e = dmk::launch_partition_lut_batch(items, m, s);
        if (e != cudaSuccess) return cuda_fail(first, e, "batched precompute: partition tables");
        e = dmk::launch_pom_build_batch(items, m, s);
        if (e != cudaSuccess) return cuda_fail(first, e, "batched precompute: POM build");
        e = dmk::launch_xpass_mask_batch(items, m, s);
        if (e != cudaSuccess) return cuda_fail(first, e, "batched precompute: x pass");
        e = dmk::launch_line_pass_batch(items, m, 1, s);
        if (e != cudaSuccess) return cuda_fail(first, e, "batched precompute: y pass");
        e = dmk::launch_line_pass_batch(items, m, 2, s);
        if (e != cudaSuccess) return cuda_fail(first, e, "batched precompute: z pass");
        dmk::PlaneOrderItem po[dmk::kMaxBuildBatch];
        for (int k = 0; k < m; ++k) po[k] = plane_order_item(ctxs[i0 + k]);
        e = dmk::launch_plane_order(po, m, s);
        if (e != cudaSuccess) return cuda_fail(first, e, "batched precompute: plane order");
        for (int k = 0; k < m; ++k) {
            dm_ctx* c = ctxs[i0 + k];
            if (c->J > 0) {
                e = dmk::launch_build_index(items[k].pdm, c->geo.plane, c->geo.G,
                                            c->cfg.num_partitions, s);
                if (e != cudaSuccess) return cuda_fail(c, e, "batched precompute: range index");
            }
        }
        for (int k = 0; k < m; ++k) {
            dm_ctx* c = ctxs[i0 + k];
            c->built = true;
            c->minmax_built = c->d_minmax != nullptr;
            c->err[0] = 0;
        }
    }
    return DM_OK;
}

static dm_status check_update(dm_ctx* ctx, const void* tf, const void* out, const char* who)
{
    if (!tf || !out || !aligned(tf, 4))
        return fail(ctx, DM_ERR_INVALID_ARG, "%s: null or misaligned tf / out", who);
    if (!ctx->d_pdm || !ctx->d_scratch)
        return fail(ctx, DM_ERR_NOT_BOUND, "%s: pdm and scratch must be bound", who);
    if (!ctx->built)
        return fail(ctx, DM_ERR_NOT_BOUND, "%s: dm_build_partitions (or dm_mark_built) has not "
                    "run on the bound pdm and scratch", who);
    return DM_OK;
}

static dm_status update_into(dm_ctx* ctx, const float* d_tf, uint8_t* d_out,
                             uint64_t* d_active_mask_out, cudaStream_t s)
{
    uint8_t* scratch = static_cast<uint8_t*>(ctx->d_scratch);
    const int K = ctx->cfg.num_partitions, N = ctx->cfg.tf_size;
    uint16_t* act = reinterpret_cast<uint16_t*>(scratch + ctx->off_act);
    int32_t* nact = reinterpret_cast<int32_t*>(scratch + ctx->off_nact);
    uint64_t* smask = reinterpret_cast<uint64_t*>(scratch + ctx->off_smask);
    if (dmk::update_fused_ok(N)) {          // one launch: every CTA derives S itself
        if (ctx->ev_begin) {
            cudaError_t e = cudaEventRecord(ctx->ev_begin, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "profile event");
        }
        cudaError_t e = dmk::launch_update_fused(static_cast<const uint8_t*>(ctx->d_pdm),
                                                 ctx->geo.plane, ctx->geo.G, d_tf, N, K,
                                                 ctx->J, ctx->borders, ctx->uniform_borders ? 1 : 0,
                                                 plane_order(ctx), region_bounds(ctx), act,
                                                 nact, smask,
                                                 d_active_mask_out, d_out, ctx->num_sms,
                                                 prof_count(ctx), s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "update");
        if (ctx->ev_end && (e = cudaEventRecord(ctx->ev_end, s)) != cudaSuccess)
            return cuda_fail(ctx, e, "profile event");
        ctx->err[0] = 0;
        return DM_OK;
    }
    cudaError_t e = dmk::launch_active_set(d_tf, N, K, ctx->J, ctx->borders, plane_order(ctx),
                                           act, nact, smask, d_active_mask_out, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "active set");
    if (ctx->ev_begin && (e = cudaEventRecord(ctx->ev_begin, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "profile event");
    e = dmk::launch_combine(static_cast<const uint8_t*>(ctx->d_pdm), ctx->geo.plane, ctx->geo.G,
                            act, nact, d_out, ctx->num_sms, prof_count(ctx), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "combine");
    if (ctx->ev_end && (e = cudaEventRecord(ctx->ev_end, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "profile event");
    ctx->err[0] = 0;
    return DM_OK;
}

dm_status dm_update_tf(dm_ctx* ctx, const float* d_tf_rgba, uint8_t* d_out,
                       uint64_t* d_active_mask_out, void* stream)
{
    if (!ctx) return DM_ERR_INVALID_ARG;
    if (d_active_mask_out && !aligned(d_active_mask_out, 8))
        return fail(ctx, DM_ERR_INVALID_ARG, "dm_update_tf: misaligned active-mask output");
    dm_status st = check_update(ctx, d_tf_rgba, d_out, "dm_update_tf");
    if (st != DM_OK) return st;
    st = check_sticky(ctx, "dm_update_tf (earlier work)");
    if (st != DM_OK) return st;
    return update_into(ctx, d_tf_rgba, d_out, d_active_mask_out, as_stream(stream));
}

dm_status dm_update_tf_host(dm_ctx* ctx, const float* h_tf_rgba, uint8_t* h_out, void* stream)
{
    if (!ctx) return DM_ERR_INVALID_ARG;
    if (!h_tf_rgba || !h_out) return fail(ctx, DM_ERR_INVALID_ARG, "dm_update_tf_host: null buffer");
    dm_status st = check_update(ctx, h_tf_rgba, h_out, "dm_update_tf_host");
    if (st != DM_OK) return st;
    st = check_sticky(ctx, "dm_update_tf_host (earlier work)");
    if (st != DM_OK) return st;
    cudaStream_t s = as_stream(stream);
    uint8_t* scratch = static_cast<uint8_t*>(ctx->d_scratch);
    float* d_tf = reinterpret_cast<float*>(scratch + ctx->off_tf);
    uint8_t* d_out = scratch + ctx->off_out;
    const size_t tf_bytes = size_t(ctx->cfg.tf_size) * 16;
    cudaError_t e = cudaMemcpyAsync(d_tf, h_tf_rgba, tf_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dm_update_tf_host: TF upload");
    // Pinned (page-locked, mapped) host output: the update writes D' into it directly
    // (over the CPU-GPU link, overlapped with its reads); otherwise through scratch and a
    // device-to-host copy.
    cudaPointerAttributes pa;
    uint8_t* mapped = nullptr;
    if (cudaPointerGetAttributes(&pa, h_out) == cudaSuccess) {
        if (pa.type == cudaMemoryTypeHost && pa.devicePointer)
            mapped = static_cast<uint8_t*>(pa.devicePointer);
    } else {
        cudaGetLastError();
    }
    st = update_into(ctx, d_tf, mapped ? mapped : d_out, nullptr, s);
    if (st != DM_OK) return st;
    if (!mapped) {
        e = cudaMemcpyAsync(h_out, d_out, size_t(ctx->geo.G), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "dm_update_tf_host: D' download");
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dm_update_tf_host: sync");
    return DM_OK;
}

dm_status dm_full_recompute(dm_ctx* ctx, const void* d_volume, const float* d_tf_rgba,
                            uint8_t* d_out, void* stream)
{
    if (!ctx) return DM_ERR_INVALID_ARG;
    if (!d_tf_rgba || !d_out || !aligned(d_tf_rgba, 4))
        return fail(ctx, DM_ERR_INVALID_ARG, "dm_full_recompute: null or misaligned tf / out");
    if (!ctx->d_scratch)
        return fail(ctx, DM_ERR_NOT_BOUND, "dm_full_recompute: scratch must be bound");
    const bool exact = ctx->cfg.occ_mode == DM_OCC_EXACT;
    if (exact && (!d_volume || !aligned(d_volume, size_t(ctx->geo.bpv))))
        return fail(ctx, DM_ERR_INVALID_ARG, "dm_full_recompute: exact mode needs the volume");
    if (!exact && (!ctx->d_minmax || !ctx->minmax_built))
        return fail(ctx, DM_ERR_NOT_BOUND,
                    "dm_full_recompute: min/max mode needs a bound min/max built by dm_build_partitions");
    dm_status st = check_sticky(ctx, "dm_full_recompute (earlier work)");
    if (st != DM_OK) return st;
    cudaStream_t s = as_stream(stream);
    uint8_t* scratch = static_cast<uint8_t*>(ctx->d_scratch);
    const int K = ctx->cfg.num_partitions, N = ctx->cfg.tf_size;
    int32_t* cnt = reinterpret_cast<int32_t*>(scratch + ctx->off_cnt);
    uint16_t* act = reinterpret_cast<uint16_t*>(scratch + ctx->off_act);
    int32_t* nact = reinterpret_cast<int32_t*>(scratch + ctx->off_nact);
    uint64_t* smask = reinterpret_cast<uint64_t*>(scratch + ctx->off_smask);
    cudaError_t e = dmk::launch_tf_active(d_tf_rgba, N, K, ctx->borders, cnt, act, nact, smask,
                                          nullptr, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "visibility prefix");
    if (exact) {
        e = dmk::launch_occ_exact(d_volume, ctx->geo, N, cnt, d_out, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "exact occupancy");
        e = dmk::launch_xpass_occ(d_out, ctx->geo, s);
    } else {
        e = dmk::launch_xpass_minmax(ctx->d_minmax, cnt, ctx->geo, d_out, s);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "DT x pass");
    e = dmk::launch_line_pass(d_out, 1, 0, ctx->geo, 1, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "DT y pass");
    e = dmk::launch_line_pass(d_out, 1, 0, ctx->geo, 2, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "DT z pass");
    ctx->err[0] = 0;
    return DM_OK;
}

static uint64_t fnv1a(uint64_t h, const void* p, size_t n)
{
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

static uint64_t ctx_hash(const dm_ctx* c)
{
    uint64_t h = 1469598103934665603ull;
    const int32_t layout_version = 1;
    h = fnv1a(h, &layout_version, sizeof(layout_version));
    const int32_t f[] = {c->cfg.dims[0], c->cfg.dims[1], c->cfg.dims[2], c->cfg.dtype,
                         c->cfg.block, c->cfg.apron, c->cfg.num_partitions, c->cfg.tf_size,
                         c->cfg.index_mode};
    h = fnv1a(h, f, sizeof(f));
    h = fnv1a(h, c->borders.v, sizeof(int32_t) * size_t(c->cfg.num_partitions + 1));
    return h;
}

dm_status dm_config_hash(const dm_ctx* ctx, uint64_t* out)
{
    if (!ctx || !out) return DM_ERR_INVALID_ARG;
    *out = ctx_hash(ctx);
    return DM_OK;
}

dm_status dm_mark_built(dm_ctx* ctx, uint64_t hash, int32_t with_minmax, void* stream)
{
    if (!ctx) return DM_ERR_INVALID_ARG;
    if (hash != ctx_hash(ctx))
        return fail(ctx, DM_ERR_INVALID_ARG, "dm_mark_built: maps were built for another configuration");
    if (!ctx->d_pdm || !ctx->d_scratch || (with_minmax && !ctx->d_minmax))
        return fail(ctx, DM_ERR_NOT_BOUND, "dm_mark_built: pdm, scratch (and min/max) must be bound");
    dm_status st = check_sticky(ctx, "dm_mark_built (earlier work)");
    if (st != DM_OK) return st;
    uint8_t* lut = static_cast<uint8_t*>(ctx->d_scratch) + ctx->off_lut;
    cudaError_t e = dmk::launch_partition_lut(lut, ctx->cfg.tf_size, ctx->cfg.num_partitions,
                                              ctx->borders, as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "partition table");
    const dmk::PlaneOrderItem po = plane_order_item(ctx);
    e = dmk::launch_plane_order(&po, 1, as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plane order");
    ctx->built = true;
    ctx->minmax_built = with_minmax != 0;
    ctx->err[0] = 0;
    return DM_OK;
}

static dm_status check_batch_items(const dm_batch_item* items, int32_t n, bool unique)
{
    for (int32_t i = 0; i < n; ++i) {
        dm_ctx* c = items[i].ctx;
        if (!c || !items[i].d_tf_rgba || !items[i].d_out ||
            (reinterpret_cast<uintptr_t>(items[i].d_tf_rgba) & 3))
            return c ? fail(c, DM_ERR_INVALID_ARG, "batched update: item %d: null or "
                            "misaligned buffer", i) : DM_ERR_INVALID_ARG;
        if (!c->d_pdm || !c->d_scratch || !c->built)
            return fail(c, DM_ERR_NOT_BOUND, "batched update: item %d: context not built", i);
        if (unique)
            for (int32_t j = 0; j < i; ++j)
                if (items[j].ctx == c)
                    return fail(c, DM_ERR_INVALID_ARG, "dm_update_tf_batch: context repeated "
                                "(items %d and %d)", j, i);
    }
    return DM_OK;
}

static dmk::BatchTuning batch_tuning(const dm_batch_tuning* t)
{
    dmk::BatchTuning bt;
    bt.ctas_per_sm = t ? t->combine_ctas_per_sm : 0;
    bt.loads_per_stage = t ? t->loads_per_stage : 0;
    return bt;
}

static void group_of(dm_ctx* c, dmk::BatchGroup& d)
{
    uint8_t* scratch = static_cast<uint8_t*>(c->d_scratch);
    d.pdm = static_cast<const uint8_t*>(c->d_pdm);
    d.plane = c->geo.plane;
    d.G = c->geo.G;
    d.lut = scratch + c->off_lut;
    d.order = plane_order(c);
    d.N = c->cfg.tf_size;
    d.K = c->cfg.num_partitions;
    d.J = c->J;
    d.E = 0;
}

dm_status dm_update_tf_batch(const dm_batch_item* items, int32_t n, const dm_batch_tuning* tuning,
                             void* stream)
{
    if (!items || n < 0) return DM_ERR_INVALID_ARG;
    if (n == 0) return DM_OK;
    dm_status st = check_batch_items(items, n, true);
    if (st != DM_OK) return st;
    dm_ctx* first = items[0].ctx;
    st = check_sticky(first, "dm_update_tf_batch (earlier work)");
    if (st != DM_OK) return st;
    cudaStream_t s = as_stream(stream);
    const dmk::BatchTuning bt = batch_tuning(tuning);
    dmk::BatchGroup desc[dmk::kMaxBatch];
    for (int32_t i0 = 0; i0 < n; i0 += dmk::kMaxBatch) {
        const int m = (n - i0) < dmk::kMaxBatch ? (n - i0) : dmk::kMaxBatch;
        for (int k = 0; k < m; ++k) {                   // one TF per group; the plane list
            dm_ctx* c = items[i0 + k].ctx;             // lives in the context's scratch
            uint8_t* scratch = static_cast<uint8_t*>(c->d_scratch);
            dmk::BatchGroup& d = desc[k];
            group_of(c, d);
            d.list = reinterpret_cast<uint16_t*>(scratch + c->off_act);
            d.emask = nullptr;
            d.count = reinterpret_cast<int32_t*>(scratch + c->off_nact);
            d.E = 1;
            d.tf[0] = items[i0 + k].d_tf_rgba;
            d.out[0] = items[i0 + k].d_out;
        }
        cudaError_t e = dmk::launch_update_batch(desc, m, bt, first->num_sms,
                                                 prof_count(first), s);
        if (e != cudaSuccess) return cuda_fail(first, e, "batched update");
    }
    return DM_OK;
}

// Workspace slot of one group: the plane count, then the padded plane list and TF sets.
static size_t ws_slot_bytes()
{
    const size_t entries = dmk::batch_list_entries(2048);
    return align_up(16 + entries * 3, 256);
}

size_t dm_batch_workspace_bytes(int32_t n) { return n > 0 ? size_t(n) * ws_slot_bytes() : 0; }

dm_status dm_update_tf_batch_ws(const dm_batch_item* items, int32_t n,
                                const dm_batch_tuning* tuning, void* d_workspace,
                                size_t workspace_bytes, void* stream)
{
    if (!items || n < 0) return DM_ERR_INVALID_ARG;
    if (n == 0) return DM_OK;
    dm_ctx* first = items[0].ctx;
    if (!first) return DM_ERR_INVALID_ARG;
    if (!d_workspace || !aligned(d_workspace, 256) || workspace_bytes < dm_batch_workspace_bytes(n))
        return fail(first, DM_ERR_INVALID_ARG, "dm_update_tf_batch_ws: workspace null, not "
                    "256-byte aligned or smaller than dm_batch_workspace_bytes(%d)", n);
    dm_status st = check_batch_items(items, n, false);
    if (st != DM_OK) return st;
    st = check_sticky(first, "dm_update_tf_batch_ws (earlier work)");
    if (st != DM_OK) return st;
    cudaStream_t s = as_stream(stream);
    const dmk::BatchTuning bt = batch_tuning(tuning);
    const size_t slot = ws_slot_bytes();
    const size_t entries = dmk::batch_list_entries(2048);
    uint8_t* ws = static_cast<uint8_t*>(d_workspace);
    // groups: the items of one context in their order, up to kMaxGroupEdits per group
    dmk::BatchGroup desc[dmk::kMaxBatch];
    int m = 0, used_slots = 0;
    bool* taken = new (std::nothrow) bool[size_t(n)]();
    if (!taken) return fail(first, DM_ERR_INVALID_ARG, "dm_update_tf_batch_ws: out of host memory");
    for (int32_t i = 0; i < n; ++i) {
        if (taken[i]) continue;
        dm_ctx* c = items[i].ctx;
        for (int32_t j = i; j < n;) {              // fill groups of this context
            dmk::BatchGroup& d = desc[m];
            group_of(c, d);
            uint8_t* sl = ws + size_t(used_slots++) * slot;
            d.count = reinterpret_cast<int32_t*>(sl);
            d.list = reinterpret_cast<uint16_t*>(sl + 16);
            d.emask = sl + 16 + entries * 2;
            for (; j < n && d.E < dmk::kMaxGroupEdits; ++j) {
                if (taken[j] || items[j].ctx != c) continue;
                taken[j] = true;
                d.tf[d.E] = items[j].d_tf_rgba;
                d.out[d.E] = items[j].d_out;
                ++d.E;
            }
            if (++m == dmk::kMaxBatch) {
                cudaError_t e = dmk::launch_update_batch(desc, m, bt, first->num_sms,
                                                 prof_count(first), s);
                if (e != cudaSuccess) {
                    delete[] taken;
                    return cuda_fail(first, e, "batched update");
                }
                m = 0;
            }
            while (j < n && (taken[j] || items[j].ctx != c)) ++j;
        }
    }
    delete[] taken;
    if (m > 0) {
        cudaError_t e = dmk::launch_update_batch(desc, m, bt, first->num_sms,
                                                 prof_count(first), s);
        if (e != cudaSuccess) return cuda_fail(first, e, "batched update");
    }
    return DM_OK;
}

dm_status dm_set_profile_events(dm_ctx* ctx, void* ev_begin, void* ev_end)
{
    if (!ctx) return DM_ERR_INVALID_ARG;
    if ((ev_begin == nullptr) != (ev_end == nullptr))
        return fail(ctx, DM_ERR_INVALID_ARG, "dm_set_profile_events: set both events or neither");
    ctx->ev_begin = static_cast<cudaEvent_t>(ev_begin);
    ctx->ev_end = static_cast<cudaEvent_t>(ev_end);
    return DM_OK;
}

dm_status dm_set_profile_counter(dm_ctx* ctx, uint64_t* d_bytes)
{
    if (!ctx) return DM_ERR_INVALID_ARG;
    if (d_bytes && !aligned(d_bytes, 8))
        return fail(ctx, DM_ERR_INVALID_ARG, "dm_set_profile_counter: misaligned counter");
    ctx->prof_bytes = d_bytes;
    return DM_OK;
}

dm_status dm_sync(dm_ctx* ctx, void* stream)
{
    cudaError_t e = cudaStreamSynchronize(as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dm_sync");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dm_sync (sticky)");
    if (ctx) ctx->err[0] = 0;
    return DM_OK;
}

void dm_destroy(dm_ctx* ctx) { delete ctx; }

}  // extern "C"
