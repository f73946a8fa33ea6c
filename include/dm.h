/*
 * dm.h -- C ABI of libdm: partitioned distance maps for fast transfer-function updates of
 * distance-map empty-space skipping (Rauter, Zimmermann & Zeilinger, IEEE VIS 2024).
 *
 * The method (§3.1): cut the intensity range into K partitions; once per volume build one
 * block-reduced occupancy map (POM) per partition and its Chebyshev distance map (PDM);
 * on every TF change, (step 1) find the set S of partitions holding an intensity with
 * non-zero alpha and (step 2, Eq. 1) take the element-wise min of the PDMs in S.  The
 * plain full recompute it replaces (occupancy of the TF, then a fresh distance transform,
 * as in Deakin & Knackstedt, §2) is provided next to it.
 *
 * Conventions shared by every call
 *  - The library allocates no device memory.  The caller allocates every device buffer,
 *    sized by dm_query_sizes(), and hands them over with dm_bind(); the library keeps only
 *    the pointers.  Buffers stay owned by the caller and must outlive their use.
 *  - Device pointers are plain CUDA device addresses; `stream` is a cudaStream_t (NULL =
 *    the legacy default stream).  Work is enqueued on `stream` and the calls return
 *    without waiting for it, except dm_update_tf_host() and dm_sync(), which wait.
 *  - Every call returns a dm_status.  On DM_ERR_* nothing was enqueued by that call, except
 *    DM_ERR_CUDA, which can also report a failure of earlier asynchronous work (a sticky
 *    CUDA error).  dm_last_error_string() gives a one-line reason.  No C++ exception
 *    crosses this interface.
 *  - A context is not thread-safe: use it from one host thread / stream at a time.
 *  - Layouts: the volume is [Z][Y][X], x fastest, uint8 or uint16.  The block grid is
 *    Gx = ceil(X/b), Gy = ceil(Y/b), Gz = ceil(Z/b), G = Gx*Gy*Gz, stored [Gz][Gy][Gx].
 *    Distance maps are uint8 [Gz][Gy][Gx]; the K PDMs are planar, plane p at byte offset
 *    p * plane_stride (plane_stride = G rounded up to 64 bytes), followed by the planes of
 *    the optional range index (dm_config.index_mode).  Distances are in block
 *    units, 0 on occupied blocks, clamped to 255, and 255 for an empty map (§3.2).
 */
#ifndef DM_H
#define DM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t dm_status;
#define DM_OK 0
#define DM_ERR_INVALID_ARG 1   /* null / misaligned pointer, bad size or value */
#define DM_ERR_UNSUPPORTED 2   /* valid but outside what this library version handles */
#define DM_ERR_CUDA 3          /* a CUDA launch or an earlier asynchronous CUDA error */
#define DM_ERR_NOT_BOUND 4     /* buffers not bound with dm_bind() */

#define DM_U8 1                /* dtype: bytes per voxel */
#define DM_U16 2

#define DM_OCC_MINMAX 0        /* full recompute: block min/max occupancy (default) */
#define DM_OCC_EXACT 1         /* full recompute: per-voxel occupancy (re-reads volume) */

#define DM_MAX_PARTITIONS 256
#define DM_MAX_TF_SIZE 65536
#define DM_MAX_BLOCK 16

typedef struct dm_ctx dm_ctx;

typedef struct dm_config {
    int32_t dims[3];          /* X, Y, Z in voxels, each >= 1 */
    int32_t dtype;            /* DM_U8 or DM_U16 */
    int32_t block;            /* b, the block edge in voxels, 1..DM_MAX_BLOCK (paper: 4) */
    int32_t apron;            /* voxels of interpolation apron added on every side of a
                                 block's footprint (clipped at the volume), 0..block */
    int32_t num_partitions;   /* K (the paper's n), 1..DM_MAX_PARTITIONS, K <= tf_size */
    const int32_t *borders;   /* host, K+1 strictly increasing lower borders with
                                 borders[0] = 0 and borders[K] = tf_size; partition p is
                                 [borders[p], borders[p+1]-1].  NULL = uniform:
                                 borders[p] = floor(p * tf_size / K).  Copied at create. */
    int32_t tf_size;          /* N, entries of the 1D TF, 2..DM_MAX_TF_SIZE; entry i maps
                                 intensity i; voxels >= N are treated as N-1 */
    int32_t occ_mode;         /* DM_OCC_MINMAX or DM_OCC_EXACT, for dm_full_recompute */
    int32_t index_mode;       /* DM_INDEX_NONE (the K PDMs only, as in the paper) or
                                 DM_INDEX_RANGES: also keep, for k = 1..floor(log2 K),
                                 plane (k, i) = min of PDM_i .. PDM_{i+2^k-1}, so that an
                                 update reads two planes per run of consecutive active
                                 partitions instead of one per active partition (same D');
                                 costs about K*log2(K) planes of memory instead of K */
} dm_config;

#define DM_INDEX_NONE 0
#define DM_INDEX_RANGES 1

typedef struct dm_sizes {
    size_t mask_bytes;        /* POM bit masks: G * ceil(K/64) uint64 words */
    size_t pdm_bytes;         /* K * plane_stride; equals K*G (§5) when G % 64 == 0 */
    size_t plane_stride;      /* bytes between PDM planes */
    size_t minmax_bytes;      /* block footprint min/max: G pairs of the voxel type */
    size_t scratch_bytes;     /* small per-context working memory */
    size_t out_bytes;         /* one distance map: G */
    int32_t grid[3];          /* Gx, Gy, Gz */
    int32_t mask_words;       /* ceil(K/64) */
    int32_t pdm_planes;       /* planes in the pdm buffer: K, or K plus the range index */
} dm_sizes;

/*
 * Validate `cfg` and create a context (host memory only).  Returns DM_ERR_INVALID_ARG for
 * a malformed config and DM_ERR_UNSUPPORTED for limits of this library version.  *out is set only
 * on DM_OK.  Partition borders: §3.1 (integer borders rho_min^p, rho_max^p; uniform split
 * or not, e.g. a separate partition for the minimum intensity).
 */
dm_status dm_create(dm_ctx **out, const dm_config *cfg);

/* Sizes of every buffer the caller must allocate for this context (host only). */
dm_status dm_query_sizes(const dm_ctx *ctx, dm_sizes *out);

/*
 * Bind caller-owned device buffers: d_mask (mask_bytes, 16-byte aligned), d_pdm
 * (pdm_bytes, 16-byte aligned), d_minmax (minmax_bytes, 16-byte aligned; may be NULL if
 * the full recompute is never used in DM_OCC_MINMAX mode), d_scratch (scratch_bytes,
 * 256-byte aligned).  d_mask is only written and read by dm_build_partitions (the POMs are
 * an intermediate, §5) and may be released afterwards by binding NULL.  Rebinding is
 * allowed between calls.  The scratch buffer holds per-context tables that
 * dm_build_partitions and dm_mark_built write: the partition of every intensity, and the
 * plane order and region bounds with which the updates read the planes (below).  Binding
 * another pdm or scratch buffer marks the context unbuilt, and the updates return
 * DM_ERR_NOT_BOUND until one of those two calls has run on the new buffers.
 */
dm_status dm_bind(dm_ctx *ctx, void *d_mask, void *d_pdm, void *d_minmax, void *d_scratch);

/*
 * One-time precompute (§3.1, "one-time initialization step"): from the device volume
 * (dims / dtype of the config) build the partition table, the K POMs as per-block bit
 * masks over each block's footprint (b^3 voxels plus the apron), the block min/max (if
 * d_minmax is bound), and the K PDMs as Chebyshev distance transforms of the POMs,
 * clamped to uint8 (§3.2).  Last, what the update uses to read few bytes: the plane order
 * (the K planes ranked by their count of zero bytes on a fixed sample, most first) and the
 * region bounds (each plane's minimum over every region of 4096 blocks), in the scratch.
 * Asynchronous on `stream`.
 */
dm_status dm_build_partitions(dm_ctx *ctx, const void *d_volume, void *stream);

/*
 * The same one-time precompute (§3.1, §3.2) for n volumes in one call: ctxs[i] is built
 * from d_volumes[i] exactly as dm_build_partitions(ctxs[i], d_volumes[i], stream) would
 * build it.  Contexts may differ in size, voxel type, block, K and N.  Each step of the
 * precompute (partition tables, POM masks, x pass, y pass, z pass) runs as one launch per
 * kernel variant over the CTAs of all the volumes, DM_BUILD_BATCH_MAX_ITEMS volumes at a
 * time.  POM builds go to the 16-byte vector kernel where it takes the volume (b = 4,
 * apron 1, K <= 32 for uint8 and K <= 64 for uint16; rows of any length, a volume aligned
 * to its voxel size), else to the general kernel (K <= 64); a volume with K > 64 gets its
 * own POM launch within the batch.  The range-index levels (DM_INDEX_RANGES) are built
 * per volume after the z pass.  Asynchronous on `stream`.  The call first clears the
 * message of every listed context.  Errors, all found on the host before anything is
 * enqueued: DM_ERR_INVALID_ARG
 * (null arrays or n < 0, a null context, a null or misaligned volume, a context listed
 * twice, two contexts bound to the same mask, pdm, min/max or scratch buffer) and
 * DM_ERR_NOT_BOUND (mask, pdm or scratch not bound), reported in the context concerned
 * (dm_last_error_string), else in ctxs[0].  The buffers of different contexts must not
 * overlap.  A launch failure returns DM_ERR_CUDA; the volumes of the failing group of
 * DM_BUILD_BATCH_MAX_ITEMS are then unbuilt and those of later groups untouched.
 */
#define DM_BUILD_BATCH_MAX_ITEMS 64
dm_status dm_build_partitions_batch(dm_ctx *const *ctxs, const void *const *d_volumes,
                                    int32_t n, void *stream);

/*
 * Per-TF update (§3.1 steps 1 and 2, Eq. 1).  d_tf_rgba: device float32 [N][4] (RGBA);
 * a partition is active when one of its intensities has alpha > 0.0f (NaN is not).
 * d_out: device uint8 [G], D' = min over active p of PDM_p, 255 where no partition is
 * active.  d_active_mask_out: optional device uint64 [ceil(K/64)] receiving S as a bit
 * set.  Reads the PDMs built by dm_build_partitions.  Asynchronous; no host round trip.
 * Without the range index the active planes are read in the context's plane order, and a
 * 16-byte chunk of D' whose minimum is already 0 in every byte reads no further plane; on
 * maps of about 5 M blocks or more each region of 4096 blocks reads its planes in
 * ascending order of their minimum over the region (bounds built with the maps) and stops
 * once the next plane's regional minimum is at least the region's largest minimum so far.
 * The traffic is at most (|S| + 1) * G bytes and D' is the same as when every active plane
 * is read.
 */
dm_status dm_update_tf(dm_ctx *ctx, const float *d_tf_rgba, uint8_t *d_out,
                       uint64_t *d_active_mask_out, void *stream);

/*
 * The same update with HOST buffers: copies h_tf_rgba (float32 [N][4]) to the device,
 * runs dm_update_tf and waits for `stream`.  When h_out (uint8 [G]) is pinned host memory
 * the GPU can address, the update writes D' into it directly; otherwise it writes into the
 * context's scratch and D' is copied back.  Pageable buffers work too (slower copies).
 */
dm_status dm_update_tf_host(dm_ctx *ctx, const float *h_tf_rgba, uint8_t *h_out,
                            void *stream);

/*
 * The plain full recompute that the method replaces (§2 Deakin & Knackstedt; compared in
 * Table 1): occupancy of the TF per block, then a fresh Chebyshev distance transform,
 * clamped to 255.  DM_OCC_MINMAX: a block is occupied when one intensity in [min, max]
 * of its footprint has alpha > 0 (Krueger & Westermann min/max blocks, §2); needs the
 * min/max built by dm_build_partitions.  DM_OCC_EXACT: a block is occupied when one voxel
 * of its footprint has alpha > 0; re-reads d_volume (ignored in DM_OCC_MINMAX mode).
 * d_out: device uint8 [G].  Asynchronous.
 */
dm_status dm_full_recompute(dm_ctx *ctx, const void *d_volume, const float *d_tf_rgba,
                            uint8_t *d_out, void *stream);

/*
 * Checkpoint / resume of a session without recomputing the maps.  dm_config_hash() gives
 * a 64-bit FNV-1a hash of everything that determines the maps' bytes (dims, voxel type,
 * block, apron, K, borders, N, index mode) and of the library's layout version.  A caller
 * that saved the PDM planes (pdm_bytes) and, if used, the min/max (minmax_bytes) of a built
 * context, and later copies them back into the bound buffers of a context with the same
 * hash, declares them built with dm_mark_built(ctx, hash); the call fails with
 * DM_ERR_INVALID_ARG when the hash differs, and with DM_ERR_NOT_BOUND when pdm / scratch
 * are not bound.  The partition table, the plane order and the region bounds in scratch
 * are rebuilt on `stream` (from the planes as they are at that point of the stream).  The
 * paper recomputes the maps at every load (§3.1, one-time initialisation).
 */
dm_status dm_config_hash(const dm_ctx *ctx, uint64_t *out);
dm_status dm_mark_built(dm_ctx *ctx, uint64_t hash, int32_t with_minmax, void *stream);

/*
 * Batched per-TF update over several volumes (§3.1 steps 1 and 2 for each item).  Item i
 * updates context items[i].ctx with its device TF (float32 [N_i][4]) into its device
 * output (uint8 [G_i]); results are those of dm_update_tf on each item alone.  Contexts may
 * differ in size, voxel type, K and N; each must have been built (dm_build_partitions or
 * dm_mark_built) on its bound pdm and scratch, and a context may appear at most once per
 * call (its scratch holds the item's active set; dm_update_tf_batch_ws below takes several
 * TFs per context).  Up to DM_BATCH_MAX_ITEMS items share one launch pair (an active-set
 * kernel with one CTA per item, then one combine over all items); longer batches are split.
 * tuning may be NULL (defaults).  Asynchronous on `stream`; the launch pair has no
 * host-side dependency on the items, so it can be captured in a CUDA graph.  Errors, all
 * found on the host before anything is enqueued: DM_ERR_INVALID_ARG (null / repeated
 * context, null buffers, a TF not 4-byte aligned), DM_ERR_NOT_BOUND (a context not built).
 */
#define DM_BATCH_MAX_ITEMS 64
#define DM_BATCH_MAX_EDITS_PER_GROUP 8
typedef struct dm_batch_item {
    dm_ctx *ctx;
    const float *d_tf_rgba;
    uint8_t *d_out;
} dm_batch_item;

typedef struct dm_batch_tuning {
    int32_t combine_ctas_per_sm;   /* combine grid: CTAs per SM (0 = default 24) */
    int32_t loads_per_stage;       /* plane loads per combine pipeline stage: 4 (0 = default)
                                      or 8 */
    int32_t reserved[2];
} dm_batch_tuning;

dm_status dm_update_tf_batch(const dm_batch_item *items, int32_t n,
                             const dm_batch_tuning *tuning, void *stream);

/*
 * Batched update in which a context may appear several times: several TF edits of one
 * volume in one call, next to other volumes (§3.1 steps 1 and 2 for each item; results
 * are those of dm_update_tf on each item alone).  The items of one context, in their
 * order, form groups of up to DM_BATCH_MAX_EDITS_PER_GROUP; the combine reads every PDM
 * plane that one of a group's TFs needs once and folds it into each of those TFs' maps,
 * so a group's HBM traffic is at most (|S_1 u ... u S_E| + E) * G bytes instead of
 * sum_e (|S_e| + 1) * G (planes in the plane order; a chunk at 0 in every byte of every
 * TF of the group reads no further plane).  The active sets live in d_workspace, a
 * caller-allocated device buffer of at least dm_batch_workspace_bytes(n) bytes, 256-byte
 * aligned, which must not be used by other work while the call's kernels run (no
 * context's scratch is written, so calls on other streams may share contexts but not a
 * workspace).  Up to
 * DM_BATCH_MAX_ITEMS groups share a launch pair; more are split.  Outputs must not overlap.
 * Errors as for dm_update_tf_batch (a repeated context is allowed), plus
 * DM_ERR_INVALID_ARG for a missing, misaligned or short workspace.  Asynchronous;
 * capturable in a CUDA graph.
 */
size_t dm_batch_workspace_bytes(int32_t n);
dm_status dm_update_tf_batch_ws(const dm_batch_item *items, int32_t n,
                                const dm_batch_tuning *tuning, void *d_workspace,
                                size_t workspace_bytes, void *stream);

/*
 * Instrumentation: when set, dm_update_tf() records `ev_begin` on its stream right before
 * the combine kernel (Eq. 1) is launched and `ev_end` right after it, so a caller can time
 * that kernel alone with cudaEventElapsedTime (for tf_size <= 8192 the combine kernel also
 * derives the active set, so the events bracket the whole update).  Both are cudaEvent_t created by the caller
 * (owned by the caller); pass NULL, NULL to stop.  No effect on results.
 */
dm_status dm_set_profile_events(dm_ctx *ctx, void *ev_begin, void *ev_end);

/*
 * Instrumentation: when d_bytes (device memory, 8-byte aligned, owned and zeroed by the
 * caller) is set, every later dm_update_tf() / dm_update_tf_host() on the context adds to
 * *d_bytes the bytes of PDM planes its combine loads (Eq. 1): 16 per 16-byte chunk of a
 * plane, 1 per byte past the last whole chunk.  With the plane order and the stop at 0 of
 * the update this is at most |S| * G; it is the update's algorithmic read traffic, which a
 * caller divides by the kernel time for its bandwidth.  dm_update_tf_batch and
 * dm_update_tf_batch_ws add the bytes of the whole call to the counter of items[0].ctx (a
 * separate build of their combine kernel does the counting).  The count costs a few
 * instructions per load and one atomic per warp; pass NULL to stop.  No effect on D'.
 */
dm_status dm_set_profile_counter(dm_ctx *ctx, uint64_t *d_bytes);

/*
 * TF update for callers that cannot allocate device memory.  The paper has no counterpart:
 * this is a deployment variant of dm_update_tf (same results, bit for bit).
 *
 * Who needs it: code that is not allowed to call cudaMalloc -- for example a plug-in
 * inside a host renderer that owns all device allocations and only hands out the buffers
 * it manages, or a render loop that must not allocate between frames because an
 * allocation can synchronize the device and stall the frame.  dm_update_tf needs a small
 * scratch buffer bound to a context; this call needs neither a context nor scratch from
 * the caller.  Its working memory is a fixed array of DM_NOALLOC_SCRATCH_BYTES inside the
 * library's own device memory, which every GPU that loads the library keeps until the
 * process exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Inputs: d_pdm, the K PDM planes (uint8, plane p at byte p * plane_stride, each [G] =
 * num_blocks bytes, as built by dm_build_partitions); borders, host, K+1 lower borders as
 * in dm_config (NULL = uniform); tf_size N; d_tf_rgba, device float32 [N][4].  Output:
 * d_out, device uint8 [G], D' = min over active p of PDM_p (255 if none is active).
 * Errors: DM_ERR_INVALID_ARG for null pointers, plane_stride < num_blocks, bad borders;
 * DM_ERR_UNSUPPORTED when K > DM_MAX_PARTITIONS or N > DM_NOALLOC_MAX_TF_SIZE (the fixed
 * array holds one visibility bit per TF entry); DM_ERR_CUDA for a launch failure.  Sizes
 * are checked on the host before anything is enqueued.
 *
 * The first call on each device looks up the array's device address (with that device
 * current) and caches it; make that first call outside any stream capture.  The cached
 * address is not valid after cudaDeviceReset() (the array may move when the library's
 * device code is loaded again): do not call this entry point after resetting a device it
 * was used on.  Every call shares the array and it keeps the last call's contents (each
 * call rewrites all of the array that it reads); calls whose work overlaps on the GPU,
 * e.g. on two unordered streams, race on it.  An error left by earlier CUDA work of the
 * caller is returned as DM_ERR_CUDA and left in place (not cleared).  Asynchronous on
 * `stream`.
 */
#define DM_NOALLOC_MAX_TF_SIZE 16384
#define DM_NOALLOC_SCRATCH_BYTES 4096
dm_status dm_update_tf_noalloc(const uint8_t *d_pdm, size_t plane_stride, int64_t num_blocks,
                               int32_t num_partitions, const int32_t *borders,
                               int32_t tf_size, const float *d_tf_rgba, uint8_t *d_out,
                               void *stream);

/*
 * Consumer of the distance map (not part of the update path): a headless orthographic ray
 * caster with empty-space skipping, the renderer the distance map serves (§1; §4.1: early
 * ray termination at 0.98).  Pixel (i, j) casts origin + i*pixel_dx + j*pixel_dy +
 * t*direction; samples lie on t_k = t_in + k*step inside the box of voxel centres and are
 * pre-classified trilinear (the RGBA of the 8 corner voxels are blended).  With d_dmap
 * (uint8 [G] Chebyshev distances in blocks of `block` voxels, built with an apron >= 1,
 * e.g. D' from dm_update_tf) the ray jumps over every cube of blocks the map proves empty,
 * landing on the same sample lattice, so the image equals the one rendered with d_dmap =
 * NULL (no skipping).  d_image_rgba: device float32 [height][width][4], premultiplied
 * colour and accumulated alpha.  d_samples (nullable): device uint32 [height][width],
 * samples evaluated per ray.  Asynchronous on `stream`.
 */
typedef struct dm_camera {
    float origin[3], pixel_dx[3], pixel_dy[3], direction[3];
    int32_t width, height;
    float step;                 /* sample spacing in voxels along the ray, > 0 */
    float ert;                  /* early ray termination threshold (accumulated alpha) */
} dm_camera;

dm_status dm_render(const void *d_volume, int32_t dtype, const int32_t dims[3], int32_t block,
                    const uint8_t *d_dmap, const float *d_tf_rgba, int32_t tf_size,
                    const dm_camera *cam, float *d_image_rgba, uint32_t *d_samples,
                    void *stream);

/* Wait for `stream` and report any asynchronous CUDA error as DM_ERR_CUDA. */
dm_status dm_sync(dm_ctx *ctx, void *stream);

/* Free the context (host memory only; bound buffers stay with the caller).  NULL is ok. */
void dm_destroy(dm_ctx *ctx);

/* One-line reason for the context's last error ("" if none); valid until the next call. */
const char *dm_last_error_string(const dm_ctx *ctx);

/* Static name of a status code. */
const char *dm_status_string(dm_status s);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int32_t dm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DM_H */
