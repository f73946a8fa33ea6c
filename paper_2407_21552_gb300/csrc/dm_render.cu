// dm_render.cu -- a headless ray caster that consumes a distance map for empty-space
// skipping (the renderer of §1 / §3.2 that the distance map serves; not on the update path).
//
// Orthographic rays, one thread per pixel, samples on a fixed lattice t_k = t_in + k * dt
// inside the volume box.  Samples use pre-classified trilinear interpolation: the RGBA of
// the 8 corner voxels (TF lookups) are blended, so a sample whose corner voxels all map to
// alpha 0 has alpha 0.  Front-to-back compositing, early ray termination once the
// accumulated alpha reaches `ert` (§4.1 uses 0.98).
//
// Empty-space skipping with a Chebyshev distance map in block units: a sample's block is
// floor(floor(p) / b); if the map holds d > 0 there, every block within Chebyshev distance
// d - 1 is unoccupied, so all samples whose lower corner voxel lies in that cube of blocks
// have alpha 0.  With an apron of at least one voxel the 8 corners of such a sample lie in
// the block's footprint, which is why occupancy includes the apron.  The ray jumps to the
// last lattice point before it leaves that cube (never past it), so the samples it takes
// are a subset of the plain march and the skipped ones contribute exactly nothing: the
// image equals the one without skipping.
#include "../../include/dm.h"
#include "dm_internal.cuh"

namespace dmk {
namespace {

struct RParams {
    int X, Y, Z, gx, gy, gz, b, N, W, H;
    float o[3], dx[3], dy[3], dir[3];          // pixel (i, j) ray: o + i*dx + j*dy + t*dir
    float dt, ert;
    int ess;
};

template <typename T>
__device__ __forceinline__ float4 classify(const T* __restrict__ vol, const float4* __restrict__ tf,
                                           const RParams& P, int x, int y, int z)
{
    unsigned v = vol[(int64_t(z) * P.Y + y) * P.X + x];
    if (v > unsigned(P.N - 1)) v = unsigned(P.N - 1);
    return __ldg(tf + v);
}

template <typename T>
__global__ void __launch_bounds__(128)
k_raymarch(const T* __restrict__ vol, const uint8_t* __restrict__ dmap,
           const float4* __restrict__ tf, RParams P, float4* __restrict__ img,
           uint32_t* __restrict__ nsamp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= P.W || j >= P.H) return;
    float o[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) o[a] = P.o[a] + i * P.dx[a] + j * P.dy[a];
    // entry / exit of the box of voxel centres [0, dim - 1]
    const float hi[3] = {float(P.X - 1), float(P.Y - 1), float(P.Z - 1)};
    float tin = -1e30f, tout = 1e30f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (fabsf(P.dir[a]) < 1e-12f) {
            if (o[a] < 0.f || o[a] > hi[a]) tout = -1e30f;
        } else {
            const float t0 = (0.f - o[a]) / P.dir[a], t1 = (hi[a] - o[a]) / P.dir[a];
            tin = fmaxf(tin, fminf(t0, t1));
            tout = fminf(tout, fmaxf(t0, t1));
        }
    }
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t taken = 0;
    if (tin <= tout) {
        const int nk = int(floorf((tout - tin) / P.dt)) + 1;
        for (int k = 0; k < nk;) {
            const float t = tin + k * P.dt;
            float p[3];
            int c[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                p[a] = fminf(fmaxf(o[a] + t * P.dir[a], 0.f), hi[a]);
                c[a] = min(int(floorf(p[a])), int(hi[a]));
            }
            if (P.ess) {
                const int bx = c[0] / P.b, by = c[1] / P.b, bz = c[2] / P.b;
                const int d = dmap[(int64_t(bz) * P.gy + by) * P.gx + bx];
                if (d > 0) {
                    // leave the cube of blocks within distance d - 1 of (bx, by, bz)
                    const int bl[3] = {bx, by, bz};
                    float texit = 1e30f;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (fabsf(P.dir[a]) < 1e-12f) continue;
                        const float lo = float((bl[a] - d + 1) * P.b), up = float((bl[a] + d) * P.b);
                        const float bound = P.dir[a] > 0.f ? up : lo;
                        texit = fminf(texit, (bound - o[a]) / P.dir[a]);
                    }
                    // last lattice point strictly before the exit (minus a guard)
                    const int kn = int(floorf((texit - tin) / P.dt - 1e-3f));
                    k = max(k + 1, kn);
                    continue;
                }
            }
            ++taken;
            // pre-classified trilinear sample
            const int x0 = c[0], y0 = c[1], z0 = c[2];
            const int x1 = min(x0 + 1, P.X - 1), y1 = min(y0 + 1, P.Y - 1), z1 = min(z0 + 1, P.Z - 1);
            const float fx = p[0] - x0, fy = p[1] - y0, fz = p[2] - z0;
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            const int xs[2] = {x0, x1}, ys[2] = {y0, y1}, zs[2] = {z0, z1};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float w = ((q & 1) ? fx : 1.f - fx) * ((q & 2) ? fy : 1.f - fy) *
                                ((q & 4) ? fz : 1.f - fz);
                const float4 v = classify<T>(vol, tf, P, xs[q & 1], ys[(q >> 1) & 1], zs[(q >> 2) & 1]);
                s.x += w * v.x;
                s.y += w * v.y;
                s.z += w * v.z;
                s.w += w * v.w;
            }
            if (s.w > 0.f) {
                const float wgt = (1.f - acc.w) * s.w;
                acc.x += wgt * s.x;
                acc.y += wgt * s.y;
                acc.z += wgt * s.z;
                acc.w += wgt;
                if (acc.w >= P.ert) break;
            }
            ++k;
        }
    }
    img[int64_t(j) * P.W + i] = acc;
    if (nsamp) nsamp[int64_t(j) * P.W + i] = taken;
}

}  // namespace
}  // namespace dmk

extern "C" dm_status dm_render(const void* d_volume, int32_t dtype, const int32_t dims[3],
                               int32_t block, const uint8_t* d_dmap, const float* d_tf_rgba,
                               int32_t tf_size, const dm_camera* cam, float* d_image_rgba,
                               uint32_t* d_samples, void* stream)
{
    if (!d_volume || !dims || !d_tf_rgba || !cam || !d_image_rgba) return DM_ERR_INVALID_ARG;
    if ((dtype != DM_U8 && dtype != DM_U16) || block < 1 || tf_size < 2) return DM_ERR_INVALID_ARG;
    if (cam->width < 1 || cam->height < 1 || cam->height > 65535 || !(cam->step > 0.f))
        return DM_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_tf_rgba) & 15) || (reinterpret_cast<uintptr_t>(d_image_rgba) & 15))
        return DM_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1) return DM_ERR_INVALID_ARG;
    dmk::RParams P;
    P.X = dims[0]; P.Y = dims[1]; P.Z = dims[2];
    P.b = block;
    P.gx = (P.X + block - 1) / block;
    P.gy = (P.Y + block - 1) / block;
    P.gz = (P.Z + block - 1) / block;
    P.N = tf_size;
    P.W = cam->width;
    P.H = cam->height;
    for (int a = 0; a < 3; ++a) {
        P.o[a] = cam->origin[a];
        P.dx[a] = cam->pixel_dx[a];
        P.dy[a] = cam->pixel_dy[a];
        P.dir[a] = cam->direction[a];
    }
    P.dt = cam->step;
    P.ert = cam->ert;
    P.ess = d_dmap != nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    dim3 grid((P.W + 127) / 128, P.H);
    const float4* tf = reinterpret_cast<const float4*>(d_tf_rgba);
    float4* img = reinterpret_cast<float4*>(d_image_rgba);
    if (dtype == DM_U8)
        dmk::k_raymarch<uint8_t><<<grid, 128, 0, s>>>(static_cast<const uint8_t*>(d_volume), d_dmap,
                                                      tf, P, img, d_samples);
    else
        dmk::k_raymarch<uint16_t><<<grid, 128, 0, s>>>(static_cast<const uint16_t*>(d_volume),
                                                       d_dmap, tf, P, img, d_samples);
    return cudaGetLastError() == cudaSuccess ? DM_OK : DM_ERR_CUDA;
}
