"""Seeded synthetic intensity volumes standing in for the paper's CT / micro-CT datasets.

The paper measures on manix (512x512x460), stag beetle (832x832x494) and kingsnake
(1024x1024x795), §4.1 and Table 1; none of them ships with it.  These generators make
volumes of the same order of size and bit depth with the structure that matters to the
method: a large near-empty background, a few materials with distinct intensity bands,
and smooth boundaries so that blocks on material edges hold mixed intensities.

This module only draws inputs.  It holds none of the method's arithmetic and is shared,
as plain input bytes, by the CPU oracle and the CUDA path.

All volumes are laid out [Z][Y][X] (x fastest).  8-bit volumes are torch.uint8; 12-bit
volumes are torch.int16 tensors whose values lie in [0, 4095], so their bytes are those of
the uint16 volume the library reads (torch has only partial uint16 support).
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as F


def _gauss_kernel(sigma: float, device) -> torch.Tensor:
    r = max(1, int(math.ceil(3.0 * sigma)))
    x = torch.arange(-r, r + 1, dtype=torch.float32, device=device)
    k = torch.exp(-(x * x) / (2.0 * sigma * sigma))
    return k / k.sum()


def _smooth_axis(v: torch.Tensor, k: torch.Tensor, axis: int) -> torch.Tensor:
    """1D convolution of a 3D float tensor along one axis, replicate padding."""
    r = (k.numel() - 1) // 2
    perm = [0, 1, 2]
    perm.remove(axis)
    perm.append(axis)
    inv = [perm.index(i) for i in range(3)]
    t = v.permute(*perm).contiguous()
    a, b, n = t.shape
    t = t.view(a * b, 1, n)
    t = F.pad(t, (r, r), mode="replicate")
    t = F.conv1d(t, k.view(1, 1, -1))
    return t.view(a, b, n).permute(*inv).contiguous()


def gaussian_smooth(v: torch.Tensor, sigma: float, slab: int = 64) -> torch.Tensor:
    """Separable Gaussian blur of a float32 [Z][Y][X] tensor (z processed in slabs)."""
    k = _gauss_kernel(sigma, v.device)
    r = (k.numel() - 1) // 2
    out = torch.empty_like(v)
    Z = v.shape[0]
    # x and y inside each z-slab, then z over y-slabs, to bound temporaries
    for z0 in range(0, Z, slab):
        s = v[z0:z0 + slab]
        s = _smooth_axis(s, k, 2)
        s = _smooth_axis(s, k, 1)
        out[z0:z0 + slab] = s
    Y = v.shape[1]
    res = torch.empty_like(v)
    for y0 in range(0, Y, slab):
        s = out[:, y0:y0 + slab, :]
        res[:, y0:y0 + slab, :] = _smooth_axis(s, k, 0)
    del out
    _ = r
    return res


def _ellipsoid_mask(shape, centre, radii, device) -> torch.Tensor:
    Z, Y, X = shape
    z = torch.arange(Z, device=device, dtype=torch.float32).view(-1, 1, 1)
    y = torch.arange(Y, device=device, dtype=torch.float32).view(1, -1, 1)
    x = torch.arange(X, device=device, dtype=torch.float32).view(1, 1, -1)
    cz, cy, cx = centre
    rz, ry, rx = radii
    return ((z - cz) / rz) ** 2 + ((y - cy) / ry) ** 2 + ((x - cx) / rx) ** 2 <= 1.0


def tiny_volume(seed: int = 0, size: int = 128, device="cpu") -> torch.Tensor:
    """128^3 uint8: smoothed uniform noise in [0, 40] plus 6 ellipsoids whose voxels are
    drawn from N(80|150|220, 10) (round-robin), clipped to [0, 255]."""
    rng = np.random.default_rng(seed)
    g = torch.Generator(device="cpu").manual_seed(seed)
    shape = (size, size, size)
    noise = torch.rand(shape, generator=g).to(device)
    s = gaussian_smooth(noise, 2.0)
    s = (s - s.min()) / (s.max() - s.min()) * 40.0
    means = (80.0, 150.0, 220.0)
    vol = s
    for e in range(6):
        centre = rng.uniform(0, size, size=3)
        radii = rng.uniform(6, 30, size=3) * (size / 128.0)
        m = _ellipsoid_mask(shape, centre, radii, device)
        vals = means[e % 3] + 10.0 * torch.randn(shape, generator=g).to(device)
        vol = torch.where(m, vals, vol)
    return vol.round().clamp(0, 255).to(torch.uint8)


def ct_volume(seed: int = 1, size: int = 512, device="cpu") -> torch.Tensor:
    """size^3 uint16 holding 12-bit CT-like data: air N(0, 20) (clipped at 0), a large
    soft-tissue ellipsoid N(1000, 50), bone as rods and shells with Gaussian bands in
    [1500, 3000]; smoothed with sigma 1.5 and clipped to [0, 4095]."""
    rng = np.random.default_rng(seed)
    g = torch.Generator(device=torch.device(device)).manual_seed(seed)
    shape = (size, size, size)
    f = size / 512.0
    vol = 20.0 * torch.randn(shape, generator=g, device=torch.device(device))
    body = _ellipsoid_mask(shape, (size / 2, size / 2, size / 2),
                           (0.45 * size, 0.38 * size, 0.42 * size), device)
    tissue = 1000.0 + 50.0 * torch.randn(shape, generator=g, device=torch.device(device))
    vol = torch.where(body, tissue, vol)
    del tissue
    Z, Y, X = shape
    zz = torch.arange(Z, device=device, dtype=torch.float32).view(-1, 1, 1)
    yy = torch.arange(Y, device=device, dtype=torch.float32).view(1, -1, 1)
    xx = torch.arange(X, device=device, dtype=torch.float32).view(1, 1, -1)
    # rods along z inside the body
    for _ in range(5):
        cy = size / 2 + rng.uniform(-0.2, 0.2) * size
        cx = size / 2 + rng.uniform(-0.25, 0.25) * size
        r = rng.uniform(10, 30) * f
        z0, z1 = sorted(rng.uniform(0.1, 0.9, size=2) * size)
        mu = rng.uniform(1500, 3000)
        m = (((yy - cy) ** 2 + (xx - cx) ** 2) <= r * r) & (zz >= z0) & (zz <= z1)
        vals = mu + 80.0 * torch.randn(shape, generator=g, device=torch.device(device))
        vol = torch.where(m, vals, vol)
    # ellipsoidal shells (a skull-like layer and an inner one)
    for k in range(2):
        rad = np.array([0.40, 0.33, 0.37]) * size * (1.0 - 0.25 * k)
        th = rng.uniform(6, 10) * f
        cz, cy, cx = size / 2, size / 2, size / 2
        rho = torch.sqrt(((zz - cz) / rad[0]) ** 2 + ((yy - cy) / rad[1]) ** 2
                         + ((xx - cx) / rad[2]) ** 2)
        m = (rho <= 1.0) & (rho >= 1.0 - th / float(rad.min()))
        del rho
        mu = rng.uniform(1500, 3000)
        vals = mu + 100.0 * torch.randn(shape, generator=g, device=torch.device(device))
        vol = torch.where(m, vals, vol)
    vol = gaussian_smooth(vol, 1.5)
    return vol.round().clamp(0, 4095).to(torch.int16)


def large_volume(seed: int = 2, dims=(1024, 1024, 1795), device="cuda",
                 empty_frac: float = 0.30) -> torch.Tensor:
    """X x Y x Z uint16 (12-bit) micro-CT-like volume: a blobby layered structure of three
    material bands plus an empty background covering about `empty_frac` of the voxels.

    A coarse random field is upsampled (trilinear) to make smooth blobs; the voxels below
    the `empty_frac` quantile of that field are background N(0, 15); the rest belong to one
    of three material bands picked by depth plus a second smooth field, with intensities
    N(700, 60), N(1800, 90) and N(3200, 120).  Built in z-slabs so that temporaries stay
    small next to the output (2 bytes per voxel)."""
    X, Y, Z = dims
    g = torch.Generator(device="cpu").manual_seed(seed)
    cz, cy, cx = max(4, Z // 32), max(4, Y // 32), max(4, X // 32)
    coarse_a = torch.rand((1, 1, cz, cy, cx), generator=g)
    coarse_b = torch.rand((1, 1, cz, cy, cx), generator=g)
    thr = float(torch.quantile(F.interpolate(coarse_a, scale_factor=2, mode="trilinear",
                                             align_corners=True).flatten(), empty_frac))
    coarse_a = coarse_a.to(device)
    coarse_b = coarse_b.to(device)
    out = torch.empty((Z, Y, X), dtype=torch.int16, device=device)
    gd = torch.Generator(device=device).manual_seed(seed)
    slab = 64
    means = torch.tensor([700.0, 1800.0, 3200.0], device=device)
    sds = torch.tensor([60.0, 90.0, 120.0], device=device)
    for z0 in range(0, Z, slab):
        z1 = min(Z, z0 + slab)
        # sample the coarse fields at this slab's voxel centres (align_corners grid)
        zs = torch.linspace(0, 1, Z, device=device)[z0:z1] * 2 - 1
        ys = torch.linspace(-1, 1, Y, device=device)
        xs = torch.linspace(-1, 1, X, device=device)
        gz, gy, gx = torch.meshgrid(zs, ys, xs, indexing="ij")
        grid = torch.stack((gx, gy, gz), dim=-1).unsqueeze(0)
        del gz, gy, gx
        fa = F.grid_sample(coarse_a, grid, mode="bilinear", align_corners=True)[0, 0]
        fb = F.grid_sample(coarse_b, grid, mode="bilinear", align_corners=True)[0, 0]
        del grid
        depth = (torch.arange(z0, z1, device=device, dtype=torch.float32) / Z).view(-1, 1, 1)
        band = ((depth + 0.35 * (fb - 0.5)) * 3.0).floor().clamp(0, 2).long()
        del fb
        noise = torch.randn((z1 - z0, Y, X), generator=gd, device=device)
        mat = means[band] + sds[band] * noise
        bg = (15.0 * noise.abs())
        v = torch.where(fa < thr, bg, mat)
        del fa, band, noise, mat, bg
        out[z0:z1] = v.round().clamp(0, 4095).to(torch.int16)
    return out


def as_numpy(vol: torch.Tensor) -> np.ndarray:
    """Host numpy copy with the unsigned dtype (uint8 / uint16)."""
    t = vol.detach().cpu()
    if t.dtype == torch.uint8:
        return t.numpy()
    if t.dtype == torch.int16:
        return t.numpy().view(np.uint16)
    raise TypeError(f"unsupported volume dtype {t.dtype}")


def volume_sha256(vol: torch.Tensor) -> str:
    import hashlib
    return hashlib.sha256(as_numpy(vol).tobytes()).hexdigest()


def volume_of(kind: str, dims, seed: int, device="cpu") -> torch.Tensor:
    """A volume of arbitrary dims (X, Y, Z) from one of the generators above: 'u8' uses the
    tiny recipe (noise + ellipsoids), 'u16' a CT-like recipe (air, soft tissue, bone), both
    with their structure scaled to the volume."""
    X, Y, Z = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    shape = (Z, Y, X)
    # noise is drawn where the volume is built (a CPU generator is slow for large volumes)
    gdev = torch.device(device)
    g = torch.Generator(device=gdev).manual_seed(seed)

    def rand(*shp):
        return torch.rand(shp, generator=g, device=gdev)

    def randn(*shp):
        return torch.randn(shp, generator=g, device=gdev)
    if kind == "u8":
        s = gaussian_smooth(rand(*shape), 2.0)
        s = (s - s.min()) / (s.max() - s.min() + 1e-12) * 40.0
        vol = s
        m0 = min(shape)
        for e in range(6):
            centre = rng.uniform(0, 1, size=3) * np.array(shape)
            radii = rng.uniform(0.05, 0.25, size=3) * m0
            m = _ellipsoid_mask(shape, centre, radii, device)
            vals = (80.0, 150.0, 220.0)[e % 3] + 10.0 * randn(*shape)
            vol = torch.where(m, vals, vol)
        return vol.round().clamp(0, 255).to(torch.uint8)
    vol = 20.0 * randn(*shape)
    body = _ellipsoid_mask(shape, (Z / 2, Y / 2, X / 2), (0.45 * Z, 0.38 * Y, 0.42 * X), device)
    vol = torch.where(body, 1000.0 + 50.0 * randn(*shape), vol)
    for _ in range(3):
        centre = (np.array(shape) * rng.uniform(0.3, 0.7, size=3))
        radii = np.array(shape) * rng.uniform(0.05, 0.15, size=3)
        m = _ellipsoid_mask(shape, centre, radii, device)
        vol = torch.where(m, rng.uniform(1500, 3000) + 80.0 * randn(*shape), vol)
    vol = gaussian_smooth(vol, 1.5)
    return vol.round().clamp(0, 4095).to(torch.int16)


def batch_specs(seed: int = 4, count: int = 64, lo: int = 64, hi: int = 384):
    """The batched-instances workload: `count` volumes with every side drawn uniformly in
    [lo, hi], alternating uint8 (N=256) and 12-bit (N=4096), K alternating 16 / 32."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        dims = tuple(int(v) for v in rng.integers(lo, hi + 1, size=3))
        kind = "u8" if i % 2 == 0 else "u16"
        out.append(dict(dims=dims, kind=kind, N=256 if kind == "u8" else 4096,
                        K=16 if (i // 2) % 2 == 0 else 32, seed=1000 + i))
    return out
