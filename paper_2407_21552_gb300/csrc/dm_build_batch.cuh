// dm_build_batch.cuh -- the batched one-time precompute: launchers shared between the
// C-ABI layer and the kernel files.  Internal to libdm.
#pragma once

#include "dm_internal.cuh"

namespace dmk {

// ---------------------------------------------------------------- batched precompute
constexpr int kMaxBuildBatch = 64;     // volumes per batched launch (descriptors as parameters)

// One volume of a batched precompute: the buffers of its one-volume build.
struct BuildItem {
    const void* vol;
    Geometry g;
    int N, K;
    int shift;                         // as in launch_pom_build
    const Borders* borders;            // host memory, read while the launches are set up
    uint8_t* lut;
    uint64_t* mask;
    void* minmax;                      // may be null
    uint8_t* pdm;                      // K planes, g.plane bytes apart
};

// The CTA of a grid that concatenates several volumes' grids: the last i < n with
// start[i] <= cta (start ascending from start[0] = 0, no volume without CTAs).
__device__ __forceinline__ int batch_item_of(const int* start, int n, int cta)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= cta) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Each step of the precompute of up to kMaxBuildBatch volumes as one launch per kernel
// variant over all their CTAs.  Partition tables; POM build (volumes that the 16-byte
// vector kernel does not take run their one-volume kernels); x pass; y pass; z pass.
cudaError_t launch_partition_lut_batch(const BuildItem* items, int n, cudaStream_t s);
cudaError_t launch_pom_build_batch(const BuildItem* items, int n, cudaStream_t s);
cudaError_t launch_xpass_mask_batch(const BuildItem* items, int n, cudaStream_t s);
cudaError_t launch_line_pass_batch(const BuildItem* items, int n, int axis, cudaStream_t s);

// ---------------------------------------------------------------- plane order, bounds
// What the combine needs to read few bytes (D' does not depend on either):
//  * the plane order: descending count of zero bytes (occupied blocks) on a fixed sample of
//    each plane, ties by partition index;
//  * the region bounds: for each region of kRegionBlocks consecutive blocks and each plane,
//    the plane's minimum over the region.  No byte of D' in a region can be lowered by a
//    plane whose regional minimum is at least the region's current maximum.
constexpr int kCoverSplit = 8;         // CTAs that count one plane's sampled zero bytes

struct PlaneOrderItem {
    const uint8_t* pdm;                // K planes, `plane` bytes apart
    int64_t plane;
    int64_t G;
    int K;
    uint32_t* cover;                   // [K][kCoverSplit] sampled zero-byte counts (written)
    uint16_t* order;                   // [K] partitions, most covered first (device, written)
    uint8_t* rmin;                     // [regions(G)][K] regional minima (device, written)
    int bounds_from_planes;            // 1: rmin from the planes; 0: the caller fills it
};

// Three launches over up to kMaxBuildBatch contexts: one CTA per plane counts, one CTA per
// context ranks, one warp per (region, plane) takes the minimum.  Runs after the context's
// z pass on the same stream.
cudaError_t launch_plane_order(const PlaneOrderItem* items, int n, cudaStream_t s);

// The region bounds of a context whose regions are whole rows (bounds_from_rows_ok), from
// its POM masks rather than its planes: the masks ORed along each row, a 2D distance
// transform of those (x pass and line pass over the rows), the minimum over each region's
// rows.  proj and d2 are scratch of bounds_rows_proj_bytes / bounds_rows_d2_bytes;
// projected: the x pass already wrote proj (launch_xpass_mask's proj argument).
bool bounds_from_rows_ok(const Geometry& g, int K);
size_t bounds_rows_proj_bytes(const Geometry& g, int K);
size_t bounds_rows_d2_bytes(const Geometry& g, int K);
cudaError_t launch_bounds_from_rows(const uint64_t* mask, const Geometry& g, int K,
                                    uint64_t* proj, bool projected, uint8_t* d2, uint8_t* rmin,
                                    cudaStream_t s);

}  // namespace dmk
