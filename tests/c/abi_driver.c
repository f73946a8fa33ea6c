/*
 * abi_driver.c -- drives libdm from plain C, with no Python in between: the caller
 * allocates every device buffer with cudaMalloc (sizes from dm_query_sizes), binds them,
 * builds the partitioned distance maps of a synthetic 12-bit volume and runs TF updates
 * (Eq. 1, through dm_update_tf and dm_update_tf_host) and plain full recomputes; then three
 * volumes of different size, voxel type and K through dm_build_partitions_batch and
 * dm_update_tf_batch.  Every PDM plane and every map is compared byte for byte with the
 * oracle's C functions, which are compiled into this test program.  Test infrastructure;
 * exit status 0 = all equal.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "dm.h"

int oracle_build_partitions(const void *vol, int32_t bytes_per_voxel, const int32_t dims[3],
                            int32_t b, int32_t a, int32_t N, int32_t K, const int32_t *borders,
                            uint64_t *mask, uint8_t *pdm, uint16_t *vmin, uint16_t *vmax);
int oracle_update_tf(const uint8_t *pdm, int32_t K, int64_t G, const float *tf_rgba,
                     int32_t N, const int32_t *borders, uint8_t *out, uint64_t *smask_out);
int oracle_full_recompute_minmax(const uint16_t *vmin, const uint16_t *vmax,
                                 const int32_t grid[3], const float *tf_rgba, int32_t N,
                                 uint8_t *out);

#define CK(x)                                                                          \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            fprintf(stderr, "CUDA error %s at line %d\n", cudaGetErrorString(e_), __LINE__); \
            return 2;                                                                  \
        }                                                                              \
    } while (0)
#define DK(ctx, x)                                                                     \
    do {                                                                               \
        dm_status s_ = (x);                                                            \
        if (s_ != DM_OK) {                                                             \
            fprintf(stderr, "libdm %s (%s) at line %d\n", dm_status_string(s_),       \
                    (ctx) ? dm_last_error_string(ctx) : "", __LINE__);                 \
            return 3;                                                                  \
        }                                                                              \
    } while (0)

static uint32_t rng_state = 12345u;
static uint32_t lcg(void)
{
    rng_state = rng_state * 1664525u + 1013904223u;
    return rng_state >> 8;
}

/* TF with one opacity ramp [c - w, c + w] (alpha 0 outside) */
static void ramp_tf(float *tf, int32_t N, int32_t c, int32_t w)
{
    memset(tf, 0, sizeof(float) * 4 * (size_t)N);
    for (int32_t i = c - w; i <= c + w; ++i)
        if (i >= 0 && i < N) {
            tf[4 * i + 0] = 1.0f;
            tf[4 * i + 3] = 0.2f + 0.5f * (float)(w - abs(i - c)) / (float)(w + 1);
        }
}

/* Three volumes of different size, voxel type and K built by one dm_build_partitions_batch
 * call, then updated by one dm_update_tf_batch call; planes and maps against the oracle. */
static int batch_check(int *bad_out, int *maps_out)
{
    enum { NV = 3 };
    const int32_t dims[NV][3] = {{45, 38, 29}, {64, 20, 33}, {17, 50, 41}};
    const int32_t bpv[NV] = {2, 1, 2}, Ks[NV] = {16, 32, 48}, Ns[NV] = {4096, 256, 4096};
    dm_ctx *ctx[NV] = {NULL, NULL, NULL};
    void *d_buf[NV][6];
    void *h_vol[NV];
    const void *d_vols[NV];
    dm_sizes sz[NV];
    dm_batch_item items[NV];
    int bad = 0;
    for (int i = 0; i < NV; ++i) {
        const int64_t V = (int64_t)dims[i][0] * dims[i][1] * dims[i][2];
        dm_config cfg;
        memset(&cfg, 0, sizeof cfg);
        memcpy(cfg.dims, dims[i], sizeof cfg.dims);
        cfg.dtype = bpv[i] == 1 ? DM_U8 : DM_U16; cfg.block = 4; cfg.apron = 1;
        cfg.num_partitions = Ks[i]; cfg.tf_size = Ns[i];
        cfg.occ_mode = DM_OCC_MINMAX; cfg.index_mode = DM_INDEX_NONE;
        DK(ctx[i], dm_create(&ctx[i], &cfg));
        DK(ctx[i], dm_query_sizes(ctx[i], &sz[i]));
        h_vol[i] = malloc((size_t)bpv[i] * (size_t)V);
        for (int64_t v = 0; v < V; ++v) {
            const uint32_t x = (uint32_t)(v % dims[i][0]), y = (uint32_t)(v / dims[i][0] % dims[i][1]);
            uint32_t val = ((x / 5) * 53u + (y / 4) * 29u + (uint32_t)(v / (dims[i][0] * dims[i][1])) / 3 * 17u) % (uint32_t)Ns[i];
            if (lcg() % 8 == 0) val = lcg() % (uint32_t)Ns[i];
            if (bpv[i] == 1) ((uint8_t *)h_vol[i])[v] = (uint8_t)val;
            else ((uint16_t *)h_vol[i])[v] = (uint16_t)val;
        }
        CK(cudaMalloc(&d_buf[i][0], sz[i].mask_bytes));
        CK(cudaMalloc(&d_buf[i][1], sz[i].pdm_bytes));
        CK(cudaMalloc(&d_buf[i][2], sz[i].minmax_bytes));
        CK(cudaMalloc(&d_buf[i][3], sz[i].scratch_bytes));
        CK(cudaMalloc(&d_buf[i][4], (size_t)bpv[i] * (size_t)V));
        CK(cudaMalloc(&d_buf[i][5], sz[i].out_bytes));
        CK(cudaMemcpy(d_buf[i][4], h_vol[i], (size_t)bpv[i] * (size_t)V, cudaMemcpyHostToDevice));
        DK(ctx[i], dm_bind(ctx[i], d_buf[i][0], d_buf[i][1], d_buf[i][2], d_buf[i][3]));
        d_vols[i] = d_buf[i][4];
    }
    DK(ctx[0], dm_build_partitions_batch(ctx, d_vols, NV, NULL));
    DK(ctx[0], dm_sync(ctx[0], NULL));
    float *tf[NV];
    void *d_tf[NV];
    uint8_t *pdm_o[NV];
    for (int i = 0; i < NV; ++i) {
        const int64_t G = (int64_t)sz[i].grid[0] * sz[i].grid[1] * sz[i].grid[2];
        const int32_t K = Ks[i];
        uint64_t *mask_o = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)G * ((K + 63) / 64));
        uint16_t *vmin = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)G);
        uint16_t *vmax = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)G);
        pdm_o[i] = (uint8_t *)malloc((size_t)K * (size_t)G);
        if (oracle_build_partitions(h_vol[i], bpv[i], dims[i], 4, 1, Ns[i], K, NULL, mask_o,
                                    pdm_o[i], vmin, vmax)) {
            fprintf(stderr, "oracle build failed (batch volume %d)\n", i);
            return 4;
        }
        uint8_t *plane = (uint8_t *)malloc((size_t)G);
        for (int32_t p = 0; p < K; ++p) {
            CK(cudaMemcpy(plane, (uint8_t *)d_buf[i][1] + (size_t)p * sz[i].plane_stride,
                          (size_t)G, cudaMemcpyDeviceToHost));
            if (memcmp(plane, pdm_o[i] + (size_t)p * G, (size_t)G)) {
                fprintf(stderr, "batch volume %d: PDM plane %d differs\n", i, p);
                ++bad;
            }
        }
        free(plane); free(mask_o); free(vmin); free(vmax);
        tf[i] = (float *)malloc(sizeof(float) * 4 * (size_t)Ns[i]);
        ramp_tf(tf[i], Ns[i], (int32_t)(lcg() % (uint32_t)Ns[i]), 8 + (int32_t)(lcg() % (uint32_t)(Ns[i] / 8)));
        CK(cudaMalloc(&d_tf[i], sizeof(float) * 4 * (size_t)Ns[i]));
        CK(cudaMemcpy(d_tf[i], tf[i], sizeof(float) * 4 * (size_t)Ns[i], cudaMemcpyHostToDevice));
        items[i].ctx = ctx[i];
        items[i].d_tf_rgba = (const float *)d_tf[i];
        items[i].d_out = (uint8_t *)d_buf[i][5];
    }
    DK(ctx[0], dm_update_tf_batch(items, NV, NULL, NULL));
    DK(ctx[0], dm_sync(ctx[0], NULL));
    for (int i = 0; i < NV; ++i) {
        const int64_t G = (int64_t)sz[i].grid[0] * sz[i].grid[1] * sz[i].grid[2];
        uint8_t *got = (uint8_t *)malloc((size_t)G), *want = (uint8_t *)malloc((size_t)G);
        oracle_update_tf(pdm_o[i], Ks[i], G, tf[i], Ns[i], NULL, want, NULL);
        CK(cudaMemcpy(got, d_buf[i][5], (size_t)G, cudaMemcpyDeviceToHost));
        if (memcmp(got, want, (size_t)G)) { fprintf(stderr, "batch volume %d: D' differs\n", i); ++bad; }
        free(got); free(want); free(pdm_o[i]); free(tf[i]); free(h_vol[i]);
        for (int k = 0; k < 6; ++k) CK(cudaFree(d_buf[i][k]));
        CK(cudaFree(d_tf[i]));
        dm_destroy(ctx[i]);
    }
    *bad_out += bad;
    *maps_out += NV;
    return 0;
}

int main(void)
{
    const int32_t X = 45, Y = 38, Z = 29, b = 4, a = 1, K = 16, N = 4096;
    const int64_t V = (int64_t)X * Y * Z;
    uint16_t *vol = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)V);
    for (int32_t z = 0; z < Z; ++z)
        for (int32_t y = 0; y < Y; ++y)
            for (int32_t x = 0; x < X; ++x) {
                const uint32_t blob = (uint32_t)((x / 9) * 131 + (y / 7) * 71 + (z / 6) * 37);
                uint32_t v = (blob * 97u) % (uint32_t)N;
                if (lcg() % 10 == 0) v = lcg() % (uint32_t)N;
                vol[((int64_t)z * Y + y) * X + x] = (uint16_t)v;
            }
    dm_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.dims[0] = X; cfg.dims[1] = Y; cfg.dims[2] = Z;
    cfg.dtype = DM_U16; cfg.block = b; cfg.apron = a; cfg.num_partitions = K;
    cfg.borders = NULL; cfg.tf_size = N; cfg.occ_mode = DM_OCC_MINMAX;
    cfg.index_mode = DM_INDEX_NONE;
    dm_ctx *ctx = NULL;
    DK(ctx, dm_create(&ctx, &cfg));
    dm_sizes sz;
    DK(ctx, dm_query_sizes(ctx, &sz));
    const int64_t G = (int64_t)sz.grid[0] * sz.grid[1] * sz.grid[2];

    void *d_mask, *d_pdm, *d_minmax, *d_scratch, *d_vol, *d_tf, *d_out, *d_full;
    CK(cudaMalloc(&d_mask, sz.mask_bytes));
    CK(cudaMalloc(&d_pdm, sz.pdm_bytes));
    CK(cudaMalloc(&d_minmax, sz.minmax_bytes));
    CK(cudaMalloc(&d_scratch, sz.scratch_bytes));
    CK(cudaMalloc(&d_vol, sizeof(uint16_t) * (size_t)V));
    CK(cudaMalloc(&d_tf, sizeof(float) * 4 * (size_t)N));
    CK(cudaMalloc(&d_out, (size_t)G));
    CK(cudaMalloc(&d_full, (size_t)G));
    CK(cudaMemcpy(d_vol, vol, sizeof(uint16_t) * (size_t)V, cudaMemcpyHostToDevice));
    DK(ctx, dm_bind(ctx, d_mask, d_pdm, d_minmax, d_scratch));
    DK(ctx, dm_build_partitions(ctx, d_vol, NULL));
    DK(ctx, dm_sync(ctx, NULL));

    /* the oracle's maps */
    uint64_t *mask_o = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)G * ((K + 63) / 64));
    uint8_t *pdm_o = (uint8_t *)malloc((size_t)K * (size_t)G);
    uint16_t *vmin = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)G);
    uint16_t *vmax = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)G);
    const int32_t dims[3] = {X, Y, Z};
    if (oracle_build_partitions(vol, 2, dims, b, a, N, K, NULL, mask_o, pdm_o, vmin, vmax)) {
        fprintf(stderr, "oracle build failed\n");
        return 4;
    }
    uint8_t *plane = (uint8_t *)malloc((size_t)G);
    int bad = 0;
    for (int32_t p = 0; p < K; ++p) {
        CK(cudaMemcpy(plane, (uint8_t *)d_pdm + (size_t)p * sz.plane_stride, (size_t)G,
                      cudaMemcpyDeviceToHost));
        if (memcmp(plane, pdm_o + (size_t)p * G, (size_t)G)) {
            fprintf(stderr, "PDM plane %d differs\n", p);
            ++bad;
        }
    }

    float *tf = (float *)malloc(sizeof(float) * 4 * (size_t)N);
    uint8_t *got = (uint8_t *)malloc((size_t)G), *want = (uint8_t *)malloc((size_t)G);
    const int32_t grid[3] = {sz.grid[0], sz.grid[1], sz.grid[2]};
    int checks = 0;
    for (int t = 0; t < 8; ++t) {
        if (t == 0) memset(tf, 0, sizeof(float) * 4 * (size_t)N);       /* S empty: all 255 */
        else ramp_tf(tf, N, (int32_t)(lcg() % (uint32_t)N), 20 + (int32_t)(lcg() % 600u));
        CK(cudaMemcpy(d_tf, tf, sizeof(float) * 4 * (size_t)N, cudaMemcpyHostToDevice));
        DK(ctx, dm_update_tf(ctx, (const float *)d_tf, (uint8_t *)d_out, NULL, NULL));
        DK(ctx, dm_full_recompute(ctx, NULL, (const float *)d_tf, (uint8_t *)d_full, NULL));
        DK(ctx, dm_sync(ctx, NULL));
        oracle_update_tf(pdm_o, K, G, tf, N, NULL, want, NULL);
        CK(cudaMemcpy(got, d_out, (size_t)G, cudaMemcpyDeviceToHost));
        if (memcmp(got, want, (size_t)G)) { fprintf(stderr, "D' differs on TF %d\n", t); ++bad; }
        /* the same update with host buffers in and out (pageable memory) */
        memset(got, 7, (size_t)G);
        DK(ctx, dm_update_tf_host(ctx, tf, got, NULL));
        if (memcmp(got, want, (size_t)G)) { fprintf(stderr, "host D' differs on TF %d\n", t); ++bad; }
        oracle_full_recompute_minmax(vmin, vmax, grid, tf, N, want);
        CK(cudaMemcpy(got, d_full, (size_t)G, cudaMemcpyDeviceToHost));
        if (memcmp(got, want, (size_t)G)) { fprintf(stderr, "D_mm differs on TF %d\n", t); ++bad; }
        checks += 3;
    }
    dm_destroy(ctx);
    const int rc = batch_check(&bad, &checks);
    if (rc) return rc;
    CK(cudaFree(d_mask)); CK(cudaFree(d_pdm)); CK(cudaFree(d_minmax)); CK(cudaFree(d_scratch));
    CK(cudaFree(d_vol)); CK(cudaFree(d_tf)); CK(cudaFree(d_out)); CK(cudaFree(d_full));
    free(vol); free(mask_o); free(pdm_o); free(vmin); free(vmax); free(plane); free(tf);
    free(got); free(want);
    if (bad) {
        printf("abi driver: %d mismatches\n", bad);
        return 1;
    }
    printf("abi driver: OK (%d planes, %d maps, grid %dx%dx%d)\n", K, checks, grid[0], grid[1],
           grid[2]);
    return 0;
}
