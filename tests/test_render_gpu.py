"""Empty-space skipping with the distance maps never skips a visible sample.

The ray caster (dm_render) marches a fixed sample lattice with pre-classified trilinear
samples; with a distance map it jumps over cubes of blocks the map proves empty.  Images
with skipping driven by D' (partitioned update), by the exact D and by the min/max D must
equal the image without skipping bit for bit, while taking fewer samples.  A small numpy
ray caster written from the same definition checks the unskipped image itself.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import synth
from synth import tfs as T

pytestmark = pytest.mark.gpu


def _setup(kind, dims, K, N, seed):
    import __graft_entry__ as g
    g.build()
    from paper_2407_21552_gb300 import DM_U8, DM_U16, DM_OCC_EXACT
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    vol = synth.volume_of(kind, dims, seed).cuda()
    dt = DM_U8 if kind == "u8" else DM_U16
    eng = PartitionedDistanceMaps(dims, dt, 4, 1, K, N)
    eng.build_partitions(vol)
    ex = PartitionedDistanceMaps(dims, dt, 4, 1, K, N, occ_mode=DM_OCC_EXACT, with_minmax=False)
    return vol, dt, eng, ex


def _render(vol, dt, dims, dmap, tf, N, cam):
    from paper_2407_21552_gb300 import _abi as A
    img = torch.zeros((cam.height, cam.width, 4), dtype=torch.float32, device="cuda")
    ns = torch.zeros((cam.height, cam.width), dtype=torch.int32, device="cuda")
    A.dm_render(vol.data_ptr(), dt, dims, 4, dmap.data_ptr() if dmap is not None else None,
                tf.data_ptr(), N, cam, img.data_ptr(), ns.data_ptr(),
                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return img, ns


@pytest.mark.parametrize("kind,dims,K,N", [("u16", (72, 64, 80), 32, 4096),
                                           ("u8", (64, 70, 60), 16, 256)])
def test_skipping_is_exact_for_every_distance_map(kind, dims, K, N):
    from paper_2407_21552_gb300 import _abi as A
    vol, dt, eng, ex = _setup(kind, dims, K, N, 77)
    tfs = T.tf_edit_sequence(8, N, 6)[1::2] + [T.single_intensity_tf(N, N // 3)]
    saved = 0
    for ti, tf_np in enumerate(tfs):
        tf = torch.from_numpy(tf_np).cuda()
        maps = {"D'": eng.update_tf(tf), "D_mm": eng.full_recompute(tf),
                "D": ex.full_recompute(tf, volume=vol)}
        for angle in (0.3, 1.9):
            cam = A.orbit_camera(dims, angle, 48, 40, step=0.5, ert=0.98)
            ref, n_ref = _render(vol, dt, dims, None, tf, N, cam)
            for name, m in maps.items():
                img, n = _render(vol, dt, dims, m, tf, N, cam)
                assert torch.equal(img, ref), (name, ti, angle)
                assert bool((n <= n_ref).all()), (name, ti, angle)
                saved += int((n_ref - n).sum())
    assert saved > 0


def _numpy_render(vol, tf, cam, dims):
    X, Y, Z = dims
    N = tf.shape[0]
    cls = tf[np.minimum(vol.astype(np.int64), N - 1)]          # [Z, Y, X, 4]
    o0 = np.array(cam.origin[:], np.float64)
    dx, dy, d = (np.array(v[:], np.float64) for v in (cam.pixel_dx, cam.pixel_dy, cam.direction))
    hi = np.array([X - 1, Y - 1, Z - 1], np.float64)
    out = np.zeros((cam.height, cam.width, 4))
    for j in range(cam.height):
        for i in range(cam.width):
            o = o0 + i * dx + j * dy
            tin, tout = -1e30, 1e30
            for a in range(3):
                if abs(d[a]) < 1e-12:
                    if o[a] < 0 or o[a] > hi[a]:
                        tout = -1e30
                    continue
                t0, t1 = (0 - o[a]) / d[a], (hi[a] - o[a]) / d[a]
                tin, tout = max(tin, min(t0, t1)), min(tout, max(t0, t1))
            acc = np.zeros(4)
            if tin <= tout:
                for k in range(int(math.floor((tout - tin) / cam.step)) + 1):
                    p = np.clip(o + (tin + k * cam.step) * d, 0, hi)
                    c = np.minimum(np.floor(p).astype(int), hi.astype(int))
                    f = p - c
                    c1 = np.minimum(c + 1, hi.astype(int))
                    s = np.zeros(4)
                    for q in range(8):
                        xs = c1[0] if q & 1 else c[0]
                        ys = c1[1] if q & 2 else c[1]
                        zs = c1[2] if q & 4 else c[2]
                        w = ((f[0] if q & 1 else 1 - f[0]) * (f[1] if q & 2 else 1 - f[1])
                             * (f[2] if q & 4 else 1 - f[2]))
                        s += w * cls[zs, ys, xs]
                    if s[3] > 0:
                        wgt = (1 - acc[3]) * s[3]
                        acc[:3] += wgt * s[:3]
                        acc[3] += wgt
                        if acc[3] >= cam.ert:
                            break
            out[j, i] = acc
    return out


def test_unskipped_image_matches_numpy_ray_caster():
    from paper_2407_21552_gb300 import _abi as A
    dims = (20, 18, 22)
    vol, dt, eng, ex = _setup("u8", dims, 16, 256, 5)
    tf_np = T.tf_edit_sequence(3, 256, 2)[1]
    tf = torch.from_numpy(tf_np).cuda()
    cam = A.orbit_camera(dims, 0.7, 16, 14, step=0.5, ert=0.98)
    img, _ = _render(vol, dt, dims, None, tf, 256, cam)
    want = _numpy_render(synth.as_numpy(vol), tf_np.astype(np.float64), cam, dims)
    np.testing.assert_allclose(img.cpu().numpy(), want, atol=2e-4)
    img2, _ = _render(vol, dt, dims, eng.update_tf(tf), tf, 256, cam)
    assert torch.equal(img, img2)
