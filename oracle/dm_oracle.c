/*
 * dm_oracle.c -- plain, slow, single-threaded CPU oracle for partitioned distance maps.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or includes this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg use it.  It
 * shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (Rauter, Zimmermann & Zeilinger, "Accelerating Transfer Function Update
 * for Distance Map based Volume Rendering", IEEE VIS 2024):
 *
 *   partitions   §3.1: the intensity range is cut into K partitions [lo_p, hi_p] (integer
 *                borders; uniform by default: lo_p = floor(p*N/K), hi_p = floor((p+1)N/K)-1).
 *   POM_p        §3.1: a block is occupied for p if one voxel of its footprint has an
 *                intensity in [lo_p, hi_p].  Blocks are b^3, non-overlapping; the footprint
 *                adds `a` voxels of interpolation apron per side, clipped at the volume.
 *   PDM_p        §3.1: Chebyshev (chessboard) distance, in block units, from each block to
 *                the nearest occupied block of POM_p; 0 on occupied blocks; §3.2: stored as
 *                uint8 with distances above 255 clamped; an empty map is all 255.
 *   S            §3.1 step 1: partitions holding one intensity whose TF alpha is non-zero
 *                (float32 alpha > 0.0f; NaN and -0.0 are not visible).
 *   D'           §3.1 step 2, Eq. 1: element-wise min over p in S of PDM_p; 255 if S empty.
 *   D (exact)    the plain distance map of the TF: occupancy = one footprint voxel visible.
 *   D (min/max)  the plain full recompute it replaces: occupancy = one visible intensity in
 *                [min, max] of the footprint (Krueger & Westermann style block min/max, §2).
 *
 * Intensities >= N are clamped to N-1 before use.  The distance transform here is the
 * two-pass raster chamfer with unit weights over the 26-neighbourhood, which is exact for
 * the chessboard metric (Rosenfeld & Pfaltz in 2D; Borgefors for n-D): deliberately a
 * different algorithm from the separable passes of the CUDA path.
 *
 * Layouts: volume [Z][Y][X] (x fastest) as uint8 or uint16; block grid [Gz][Gy][Gx] with
 * Gx = ceil(X/b) etc.; masks [G][W] uint64 words, W = ceil(K/64), bit p%64 of word p/64;
 * PDMs [K][G] uint8.  Every function returns 0 on success and -1 on a bad argument.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_INF 0x3fffffff

static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

static int grid_of(const int32_t dims[3], int32_t b, int64_t g[3])
{
    if (!dims || b < 1 || dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return -1;
    for (int i = 0; i < 3; ++i) g[i] = cdiv(dims[i], b);
    return 0;
}

/* §3.1: lower border of partition p; borders == NULL means the uniform split. */
static int64_t part_lo(int32_t N, int32_t K, const int32_t *borders, int32_t p)
{
    if (borders) return borders[p];
    return ((int64_t)p * N) / K;
}

/* Partition index of every intensity i in [0, N): the p with lo_p <= i <= hi_p. */
int oracle_partition_lut(int32_t N, int32_t K, const int32_t *borders, uint8_t *lut)
{
    if (N < 1 || K < 1 || K > 256 || K > N || !lut) return -1;
    if (borders) {
        if (borders[0] != 0 || borders[K] != N) return -1;
        for (int32_t p = 0; p < K; ++p)
            if (borders[p + 1] <= borders[p]) return -1;
    }
    for (int32_t i = 0; i < N; ++i) {
        int found = -1;
        for (int32_t p = 0; p < K; ++p) {
            int64_t lo = part_lo(N, K, borders, p);
            int64_t hi = part_lo(N, K, borders, p + 1) - 1;
            if (lo <= i && i <= hi) { found = p; break; }
        }
        if (found < 0) return -1;
        lut[i] = (uint8_t)found;
    }
    return 0;
}

static int64_t voxel_at(const void *vol, int32_t bytes_per_voxel, int64_t idx, int32_t N)
{
    int64_t v = bytes_per_voxel == 1 ? ((const uint8_t *)vol)[idx]
                                     : ((const uint16_t *)vol)[idx];
    return v > N - 1 ? N - 1 : v;
}

/* Footprint of block coordinate c along an axis of length n: [c*b - a, c*b + b - 1 + a]
 * clipped to [0, n-1]. */
static void footprint(int64_t c, int32_t b, int32_t a, int64_t n, int64_t *lo, int64_t *hi)
{
    *lo = c * b - a;
    *hi = c * b + b - 1 + a;
    if (*lo < 0) *lo = 0;
    if (*hi > n - 1) *hi = n - 1;
}

/*
 * POMs (§3.1) for all K partitions at once as per-block bit masks, plus the footprint
 * minimum and maximum of the (clamped) intensity.  vmin / vmax may be NULL.
 */
int oracle_pom(const void *vol, int32_t bytes_per_voxel, const int32_t dims[3],
               int32_t b, int32_t a, int32_t N, int32_t K, const uint8_t *lut,
               uint64_t *mask, uint16_t *vmin, uint16_t *vmax)
{
    int64_t g[3];
    if (!vol || !lut || !mask || (bytes_per_voxel != 1 && bytes_per_voxel != 2)) return -1;
    if (a < 0 || grid_of(dims, b, g)) return -1;
    const int64_t X = dims[0], Y = dims[1];
    const int32_t W = (K + 63) / 64;
    for (int64_t bz = 0; bz < g[2]; ++bz)
        for (int64_t by = 0; by < g[1]; ++by)
            for (int64_t bx = 0; bx < g[0]; ++bx) {
                int64_t blk = (bz * g[1] + by) * g[0] + bx;
                int64_t x0, x1, y0, y1, z0, z1;
                footprint(bx, b, a, X, &x0, &x1);
                footprint(by, b, a, Y, &y0, &y1);
                footprint(bz, b, a, dims[2], &z0, &z1);
                for (int32_t w = 0; w < W; ++w) mask[blk * W + w] = 0;
                int64_t mn = N, mx = -1;
                for (int64_t z = z0; z <= z1; ++z)
                    for (int64_t y = y0; y <= y1; ++y)
                        for (int64_t x = x0; x <= x1; ++x) {
                            int64_t i = voxel_at(vol, bytes_per_voxel, (z * Y + y) * X + x, N);
                            int32_t p = lut[i];
                            mask[blk * W + p / 64] |= (uint64_t)1 << (p % 64);
                            if (i < mn) mn = i;
                            if (i > mx) mx = i;
                        }
                if (vmin) vmin[blk] = (uint16_t)mn;
                if (vmax) vmax[blk] = (uint16_t)mx;
            }
    return 0;
}

/*
 * Chessboard distance transform of a block occupancy grid (occ != 0 = occupied), clamped
 * to 255; 255 everywhere when nothing is occupied.  Two raster passes over the grid, each
 * taking the 13 neighbours of the 26-neighbourhood already visited in its scan order, with
 * unit step cost.
 */
int oracle_chamfer_dt(const uint8_t *occ, const int32_t grid[3], uint8_t *out)
{
    if (!occ || !out || !grid || grid[0] < 1 || grid[1] < 1 || grid[2] < 1) return -1;
    const int64_t gx = grid[0], gy = grid[1], gz = grid[2];
    const int64_t G = gx * gy * gz;
    int32_t *d = (int32_t *)malloc((size_t)G * sizeof(int32_t));
    if (!d) return -1;
    for (int64_t i = 0; i < G; ++i) d[i] = occ[i] ? 0 : OR_INF;
    /* forward: neighbours that precede (z, y, x) in z-major, y, x raster order */
    for (int64_t z = 0; z < gz; ++z)
        for (int64_t y = 0; y < gy; ++y)
            for (int64_t x = 0; x < gx; ++x) {
                int64_t i = (z * gy + y) * gx + x;
                int32_t best = d[i];
                for (int dz = -1; dz <= 0; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int before = dz < 0 || (dz == 0 && (dy < 0 || (dy == 0 && dx < 0)));
                            if (!before) continue;
                            int64_t nz = z + dz, ny = y + dy, nx = x + dx;
                            if (nz < 0 || ny < 0 || ny >= gy || nx < 0 || nx >= gx) continue;
                            int32_t c = d[(nz * gy + ny) * gx + nx];
                            if (c < OR_INF && c + 1 < best) best = c + 1;
                        }
                d[i] = best;
            }
    /* backward: neighbours that follow (z, y, x) */
    for (int64_t z = gz - 1; z >= 0; --z)
        for (int64_t y = gy - 1; y >= 0; --y)
            for (int64_t x = gx - 1; x >= 0; --x) {
                int64_t i = (z * gy + y) * gx + x;
                int32_t best = d[i];
                for (int dz = 0; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int after = dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));
                            if (!after) continue;
                            int64_t nz = z + dz, ny = y + dy, nx = x + dx;
                            if (nz >= gz || ny < 0 || ny >= gy || nx < 0 || nx >= gx) continue;
                            int32_t c = d[(nz * gy + ny) * gx + nx];
                            if (c < OR_INF && c + 1 < best) best = c + 1;
                        }
                d[i] = best;
            }
    for (int64_t i = 0; i < G; ++i) out[i] = (uint8_t)(d[i] > 255 ? 255 : d[i]);
    free(d);
    return 0;
}

/*
 * Chessboard distance at one block by searching Chebyshev shells of growing radius r
 * around it (r = 0, 1, ..., 254) for an occupied block; 255 if none is found.  Used to
 * check single outputs of grids too large for the full transform in a test.
 */
int oracle_dt_at(const uint8_t *occ, const int32_t grid[3], int32_t x, int32_t y, int32_t z)
{
    const int64_t gx = grid[0], gy = grid[1], gz = grid[2];
    if (x < 0 || y < 0 || z < 0 || x >= gx || y >= gy || z >= gz) return -1;
    for (int64_t r = 0; r < 255; ++r) {
        for (int64_t dz = -r; dz <= r; ++dz) {
            int64_t nz = z + dz;
            if (nz < 0 || nz >= gz) continue;
            for (int64_t dy = -r; dy <= r; ++dy) {
                int64_t ny = y + dy;
                if (ny < 0 || ny >= gy) continue;
                int on_shell = (dz == -r || dz == r || dy == -r || dy == r);
                int64_t step = on_shell ? 1 : 2 * r;   /* interior rows: only x = +-r */
                for (int64_t dx = -r; dx <= r; dx += (step ? step : 1)) {
                    int64_t nx = x + dx;
                    if (nx < 0 || nx >= gx) continue;
                    if (occ[(nz * gy + ny) * gx + nx]) return (int)r;
                }
            }
        }
    }
    return 255;
}

/* Occupancy plane of partition p taken from the POM bit masks. */
static void pom_plane(const uint64_t *mask, int64_t G, int32_t W, int32_t p, uint8_t *occ)
{
    for (int64_t i = 0; i < G; ++i)
        occ[i] = (uint8_t)((mask[i * W + p / 64] >> (p % 64)) & 1u);
}

/*
 * One-time precompute (§3.1): partition table, POMs, then PDM_p = DT(POM_p) for every p.
 * mask [G*W], pdm [K*G]; vmin / vmax [G] may be NULL.
 */
int oracle_build_partitions(const void *vol, int32_t bytes_per_voxel, const int32_t dims[3],
                            int32_t b, int32_t a, int32_t N, int32_t K, const int32_t *borders,
                            uint64_t *mask, uint8_t *pdm, uint16_t *vmin, uint16_t *vmax)
{
    int64_t g[3];
    if (grid_of(dims, b, g) || !pdm || !mask) return -1;
    uint8_t *lut = (uint8_t *)malloc((size_t)N);
    if (!lut) return -1;
    if (oracle_partition_lut(N, K, borders, lut)) { free(lut); return -1; }
    int rc = oracle_pom(vol, bytes_per_voxel, dims, b, a, N, K, lut, mask, vmin, vmax);
    free(lut);
    if (rc) return rc;
    const int64_t G = g[0] * g[1] * g[2];
    const int32_t W = (K + 63) / 64;
    int32_t grid[3] = {(int32_t)g[0], (int32_t)g[1], (int32_t)g[2]};
    uint8_t *occ = (uint8_t *)malloc((size_t)G);
    if (!occ) return -1;
    for (int32_t p = 0; p < K; ++p) {
        pom_plane(mask, G, W, p, occ);
        if (oracle_chamfer_dt(occ, grid, pdm + (int64_t)p * G)) { free(occ); return -1; }
    }
    free(occ);
    return 0;
}

/* §3.1 step 1: S as a bit set of ceil(K/64) words. */
int oracle_active_set(const float *tf_rgba, int32_t N, int32_t K, const int32_t *borders,
                      uint64_t *smask)
{
    if (!tf_rgba || !smask) return -1;
    uint8_t *lut = (uint8_t *)malloc((size_t)N);
    if (!lut) return -1;
    if (oracle_partition_lut(N, K, borders, lut)) { free(lut); return -1; }
    for (int32_t w = 0; w < (K + 63) / 64; ++w) smask[w] = 0;
    for (int32_t i = 0; i < N; ++i) {
        float alpha = tf_rgba[4 * i + 3];
        if (alpha > 0.0f) smask[lut[i] / 64] |= (uint64_t)1 << (lut[i] % 64);
    }
    free(lut);
    return 0;
}

/* §3.1 step 2, Eq. 1: D'(blk) = min over p in S of PDM_p(blk); 255 when S is empty. */
int oracle_combine(const uint8_t *pdm, int32_t K, int64_t G, const uint64_t *smask,
                   uint8_t *out)
{
    if (!pdm || !smask || !out || K < 1 || G < 0) return -1;
    for (int64_t i = 0; i < G; ++i) out[i] = 255;
    for (int32_t p = 0; p < K; ++p) {
        if (!((smask[p / 64] >> (p % 64)) & 1u)) continue;
        const uint8_t *plane = pdm + (int64_t)p * G;
        for (int64_t i = 0; i < G; ++i)
            if (plane[i] < out[i]) out[i] = plane[i];
    }
    return 0;
}

/* Per-TF update: step 1 then step 2.  smask_out ([ceil(K/64)]) may be NULL. */
int oracle_update_tf(const uint8_t *pdm, int32_t K, int64_t G, const float *tf_rgba,
                     int32_t N, const int32_t *borders, uint8_t *out, uint64_t *smask_out)
{
    uint64_t s[4];
    if (K < 1 || K > 256) return -1;
    if (oracle_active_set(tf_rgba, N, K, borders, s)) return -1;
    if (smask_out)
        for (int32_t w = 0; w < (K + 63) / 64; ++w) smask_out[w] = s[w];
    return oracle_combine(pdm, K, G, s, out);
}

/*
 * TF occupancy of the plain min/max recompute: a block is occupied when one intensity i in
 * [vmin(blk), vmax(blk)] has alpha(i) > 0.  occ [G] receives 0 / 1.
 */
int oracle_occ_minmax(const uint16_t *vmin, const uint16_t *vmax, int64_t G,
                      const float *tf_rgba, int32_t N, uint8_t *occ)
{
    if (!vmin || !vmax || !tf_rgba || !occ || G < 0) return -1;
    for (int64_t i = 0; i < G; ++i) {
        occ[i] = 0;
        for (int64_t v = vmin[i]; v <= vmax[i] && v < N; ++v)
            if (tf_rgba[4 * v + 3] > 0.0f) { occ[i] = 1; break; }
    }
    return 0;
}

/* Plain full recompute with block min/max occupancy, then a fresh distance transform. */
int oracle_full_recompute_minmax(const uint16_t *vmin, const uint16_t *vmax,
                                 const int32_t grid[3], const float *tf_rgba, int32_t N,
                                 uint8_t *out)
{
    if (!vmin || !vmax || !tf_rgba || !out) return -1;
    const int64_t G = (int64_t)grid[0] * grid[1] * grid[2];
    uint8_t *occ = (uint8_t *)malloc((size_t)G);
    if (!occ) return -1;
    if (oracle_occ_minmax(vmin, vmax, G, tf_rgba, N, occ)) { free(occ); return -1; }
    int rc = oracle_chamfer_dt(occ, grid, out);
    free(occ);
    return rc;
}

/*
 * The exact distance map D of a TF: a block is occupied when one voxel of its footprint
 * has an intensity with alpha > 0; then the distance transform.
 */
int oracle_full_recompute_exact(const void *vol, int32_t bytes_per_voxel, const int32_t dims[3],
                                int32_t b, int32_t a, const float *tf_rgba, int32_t N,
                                uint8_t *out)
{
    int64_t g[3];
    if (!vol || !tf_rgba || !out || a < 0 || grid_of(dims, b, g)) return -1;
    if (bytes_per_voxel != 1 && bytes_per_voxel != 2) return -1;
    const int64_t X = dims[0], Y = dims[1];
    const int64_t G = g[0] * g[1] * g[2];
    uint8_t *occ = (uint8_t *)malloc((size_t)G);
    if (!occ) return -1;
    for (int64_t bz = 0; bz < g[2]; ++bz)
        for (int64_t by = 0; by < g[1]; ++by)
            for (int64_t bx = 0; bx < g[0]; ++bx) {
                int64_t x0, x1, y0, y1, z0, z1, blk = (bz * g[1] + by) * g[0] + bx;
                footprint(bx, b, a, X, &x0, &x1);
                footprint(by, b, a, Y, &y0, &y1);
                footprint(bz, b, a, dims[2], &z0, &z1);
                uint8_t o = 0;
                for (int64_t z = z0; z <= z1 && !o; ++z)
                    for (int64_t y = y0; y <= y1 && !o; ++y)
                        for (int64_t x = x0; x <= x1 && !o; ++x) {
                            int64_t i = voxel_at(vol, bytes_per_voxel, (z * Y + y) * X + x, N);
                            if (tf_rgba[4 * i + 3] > 0.0f) o = 1;
                        }
                occ[blk] = o;
            }
    int32_t grid[3] = {(int32_t)g[0], (int32_t)g[1], (int32_t)g[2]};
    int rc = oracle_chamfer_dt(occ, grid, out);
    free(occ);
    return rc;
}
