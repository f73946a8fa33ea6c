"""Pins for the CPU oracle: each test ties it to something other than itself.

* Fig. 2 caption (§3.1): the worked example's active set, from a golden fixture.
* scipy.ndimage.distance_transform_cdt(metric="chessboard"): a library chessboard DT.
* brute-force nearest-occupied search on tiny grids.
* scipy.ndimage maximum/minimum filters + block reduction for the POMs and min/max.
* invariants the paper states: D' <= D (§3.1), D' == D when no partition mixes zero and
  non-zero alpha (§3.1, Fig. 2 TF_A), Eq. 1 equals the DT of the union of the POMs.
* special cases: empty set, all visible, K = 1, K = N with b = 1, NaN / -0.0 alpha,
  clamping at 255 on a 600-long line, the memory formula of §5.
"""
import json
import os

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
from synth import tfs as T

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- independent references
def scipy_chessboard(occ):
    """Library chessboard DT to the nearest occupied cell, clamped to 255 (255 if none)."""
    occ = occ != 0
    if not occ.any():
        return np.full(occ.shape, 255, np.uint8)
    d = ndi.distance_transform_cdt(~occ, metric="chessboard")
    return np.minimum(d, 255).astype(np.uint8)


def brute_chessboard(occ):
    occ = occ != 0
    pts = np.argwhere(occ)
    out = np.full(occ.shape, 255, np.int64)
    if len(pts) == 0:
        return out.astype(np.uint8)
    allp = np.argwhere(np.ones_like(occ))
    d = np.abs(allp[:, None, :] - pts[None, :, :]).max(-1).min(1)
    out.reshape(-1)[:] = np.minimum(d, 255)
    return out.astype(np.uint8)


def part_index(vol, N, borders):
    v = np.minimum(vol.astype(np.int64), N - 1)
    return np.searchsorted(np.asarray(borders), v, side="right") - 1


def block_reduce(a, b, fn, fill):
    Z, Y, X = a.shape
    pz, py, px = (-Z) % b, (-Y) % b, (-X) % b
    a = np.pad(a, ((0, pz), (0, py), (0, px)), constant_values=fill)
    gz, gy, gx = a.shape[0] // b, a.shape[1] // b, a.shape[2] // b
    return fn(a.reshape(gz, b, gy, b, gx, b), axis=(1, 3, 5))


def scipy_pom(vol, b, a, N, borders):
    """POM bits and footprint min/max via dilation filters + block reduction."""
    K = len(borders) - 1
    pidx = part_index(vol, N, borders)
    size = 2 * a + 1
    planes = []
    for p in range(K):
        c = (pidx == p).astype(np.uint8)
        d = ndi.maximum_filter(c, size=size, mode="constant", cval=0)
        planes.append(block_reduce(d, b, np.max, 0))
    v = np.minimum(vol.astype(np.int64), N - 1)
    big = 1 << 20
    mn = ndi.minimum_filter(v, size=size, mode="constant", cval=big)
    mx = ndi.maximum_filter(v, size=size, mode="constant", cval=-1)
    return np.stack(planes), block_reduce(mn, b, np.min, big), block_reduce(mx, b, np.max, -1)


def rand_volume(rng, shape, N, dtype):
    """Piecewise-constant blobs plus noise: mixed blocks, empty regions, several classes."""
    v = rng.integers(0, N, size=(max(1, shape[0] // 3), max(1, shape[1] // 3),
                                 max(1, shape[2] // 3)))
    v = np.kron(v, np.ones((3, 3, 3), np.int64))[: shape[0], : shape[1], : shape[2]]
    v = np.pad(v, [(0, s - v.shape[i]) for i, s in enumerate(shape)], mode="edge")
    noise = rng.integers(-N // 16, N // 16 + 1, size=shape)
    v = np.clip(v + noise * (rng.uniform(size=shape) < 0.2), 0, N - 1)
    return v.astype(dtype)


# ------------------------------------------------------------------------------ Fig. 2
def test_fig2_active_set_golden():
    g = json.load(open(os.path.join(GOLD, "fig2_active_set.json")))
    N, K, borders = g["N"], g["K"], g["borders"]
    for name, nz in g["alpha_nonzero"].items():
        tf = T.zero_tf(N)
        tf[nz, 3] = 0.7
        S = oracle.active_set(tf, K, borders)
        assert [p + 1 for p in S] == g["expected_S_one_based"][name], name


def test_fig2_like_image_tf_a_exact_tf_b_lower():
    """Our own 2D intensity image (the figure's image is not available) under the two TFs
    of the caption, without block reduction: D'_A == D_A and D'_B <= D_B, D'_A == D'_B."""
    g = json.load(open(os.path.join(GOLD, "fig2_active_set.json")))
    N, K, borders = g["N"], g["K"], g["borders"]
    rng = np.random.default_rng(5)
    img = rng.integers(0, N, size=(1, 12, 12)).astype(np.uint8)
    mask, pdm, _, _ = oracle.build_partitions(img, 1, 0, N, K, borders)
    res = {}
    for name, nz in g["alpha_nonzero"].items():
        tf = T.zero_tf(N)
        tf[nz, 3] = 1.0
        dprime, _ = oracle.update_tf(pdm, tf, borders)
        d = oracle.full_recompute_exact(img, 1, 0, tf)
        res[name] = (dprime, d)
    assert np.array_equal(res["TF_A"][0], res["TF_A"][1])
    assert np.all(res["TF_B"][0] <= res["TF_B"][1])
    assert np.array_equal(res["TF_A"][0], res["TF_B"][0])
    assert np.any(res["TF_B"][0] < res["TF_B"][1])  # this image does show the gap


# ------------------------------------------------------------------ distance transform
@pytest.mark.parametrize("shape", [(7, 5, 9), (1, 13, 11), (12, 12, 12), (4, 1, 1), (3, 8, 2)])
@pytest.mark.parametrize("density", [0.0, 0.001, 0.05, 0.5, 1.0])
def test_chamfer_matches_scipy_and_brute_force(shape, density):
    rng = np.random.default_rng(hash((shape, density)) & 0xFFFF)
    occ = (rng.uniform(size=shape) < density).astype(np.uint8)
    if density == 0.001 and not occ.any():
        occ[tuple(rng.integers(0, s) for s in shape)] = 1
    got = oracle.chamfer_dt(occ)
    assert np.array_equal(got, scipy_chessboard(occ))
    assert np.array_equal(got, brute_chessboard(occ))


def test_chamfer_large_grid_matches_scipy():
    rng = np.random.default_rng(11)
    occ = (rng.uniform(size=(37, 61, 45)) < 0.0005).astype(np.uint8)
    occ[0, 0, 0] = 1
    assert np.array_equal(oracle.chamfer_dt(occ), scipy_chessboard(occ))


def test_chamfer_clamps_at_255_on_long_line():
    occ = np.zeros((600, 1, 1), np.uint8)
    occ[0, 0, 0] = 1
    d = oracle.chamfer_dt(occ)[:, 0, 0].astype(int)
    assert np.array_equal(d, np.minimum(np.arange(600), 255))
    occ2 = np.zeros((1, 1, 600), np.uint8)
    occ2[0, 0, 599] = 1
    d2 = oracle.chamfer_dt(occ2)[0, 0, :].astype(int)
    assert np.array_equal(d2, np.minimum(599 - np.arange(600), 255))


def test_dt_at_matches_library_dt():
    rng = np.random.default_rng(3)
    for shape, dens in [((9, 14, 11), 0.01), ((20, 3, 30), 0.002), ((5, 5, 5), 0.0)]:
        occ = (rng.uniform(size=shape) < dens).astype(np.uint8)
        ref = scipy_chessboard(occ)
        for _ in range(40):
            z, y, x = (int(rng.integers(0, s)) for s in shape)
            assert oracle.dt_at(occ, x, y, z) == ref[z, y, x]


def test_dt_at_clamps_at_255_on_long_line():
    # one occupied block at the end of a 600-block line: the shell search must reach
    # radius 254 and report 255 beyond it, like the full transform
    occ = np.zeros((1, 1, 600), np.uint8)
    occ[0, 0, 0] = 1
    for x, want in [(0, 0), (1, 1), (253, 253), (254, 254), (255, 255), (599, 255)]:
        assert oracle.dt_at(occ, x, 0, 0) == want, x
    occ_z = np.zeros((600, 1, 1), np.uint8)
    occ_z[599, 0, 0] = 1
    for z, want in [(599, 0), (345, 254), (344, 255)]:
        assert oracle.dt_at(occ_z, 0, 0, z) == want, z


def test_dt_lipschitz_and_zero_iff_occupied():
    rng = np.random.default_rng(4)
    occ = (rng.uniform(size=(10, 12, 14)) < 0.02).astype(np.uint8)
    d = oracle.chamfer_dt(occ).astype(int)
    assert np.array_equal(d == 0, occ == 1)
    for ax in range(3):
        assert np.abs(np.diff(d, axis=ax)).max() <= 1
    # diagonal neighbours differ by at most 1 too (Chebyshev)
    assert np.abs(d[1:, 1:, 1:] - d[:-1, :-1, :-1]).max() <= 1


# ----------------------------------------------------------------- partitions and POMs
@pytest.mark.parametrize("N,K", [(256, 16), (4096, 32), (10, 3), (8, 8), (4096, 256)])
def test_uniform_partition_lut(N, K):
    lut = oracle.partition_lut(N, K).astype(int)
    borders = T.uniform_borders(N, K)
    assert np.array_equal(lut, part_index(np.arange(N), N, borders))
    # each partition is non-empty, contiguous and ordered
    assert lut[0] == 0 and lut[-1] == K - 1 and np.all(np.diff(lut) >= 0)
    assert len(np.unique(lut)) == K


def test_explicit_borders_and_rejects():
    borders = [0, 1, 5, 200, 256]  # a separate partition for the minimum intensity
    lut = oracle.partition_lut(256, 4, borders)
    assert lut[0] == 0 and lut[1] == 1 and lut[4] == 1 and lut[5] == 2 and lut[255] == 3
    for bad in ([0, 5, 5, 200, 256], [1, 5, 9, 200, 256], [0, 5, 9, 200, 255]):
        with pytest.raises(ValueError):
            oracle.partition_lut(256, 4, bad)


@pytest.mark.parametrize("shape,b,a,N,K,dt", [
    ((9, 10, 11), 4, 1, 256, 16, np.uint8),
    ((5, 7, 9), 4, 0, 256, 7, np.uint8),
    ((8, 8, 8), 2, 2, 64, 64, np.uint8),
    ((6, 13, 7), 3, 1, 4096, 32, np.uint16),
    ((4, 4, 12), 1, 1, 300, 70, np.uint16),
    ((3, 5, 4), 8, 1, 256, 16, np.uint8),
])
def test_pom_and_minmax_match_filters(shape, b, a, N, K, dt):
    rng = np.random.default_rng(K + b)
    vol = rand_volume(rng, shape, N, dt)
    if dt == np.uint16:
        vol[0, 0, 0] = N + 17  # above the TF domain: clamps to N-1
    borders = T.uniform_borders(N, K)
    mask, vmin, vmax = oracle.pom(vol, b, a, N, K)
    planes, mn, mx = scipy_pom(vol, b, a, N, borders)
    for p in range(K):
        assert np.array_equal(oracle.mask_plane(mask, p), planes[p]), p
    assert np.array_equal(vmin.astype(np.int64), mn)
    assert np.array_equal(vmax.astype(np.int64), mx)


def test_memory_formula_pdm_bytes():
    """§5: the PDMs take n x volumesize / b^3 bytes (block grid ceil'd at the edges)."""
    vol = np.zeros((460 // 20, 512 // 16, 512 // 16), np.uint8)
    _, pdm, _, _ = oracle.build_partitions(vol, 4, 1, 256, 16)
    gz, gy, gx = -(-vol.shape[0] // 4), -(-vol.shape[1] // 4), -(-vol.shape[2] // 4)
    assert pdm.nbytes == 16 * gz * gy * gx


# --------------------------------------------------------------- update-level invariants
@pytest.fixture(scope="module")
def small_case():
    rng = np.random.default_rng(21)
    N, K, b, a = 256, 16, 4, 1
    vol = rand_volume(rng, (30, 26, 35), N, np.uint8)
    mask, pdm, vmin, vmax = oracle.build_partitions(vol, b, a, N, K)
    return dict(vol=vol, N=N, K=K, b=b, a=a, mask=mask, pdm=pdm, vmin=vmin, vmax=vmax,
                borders=T.uniform_borders(N, K))


def test_pdm_planes_are_library_dt_of_pom(small_case):
    c = small_case
    for p in range(c["K"]):
        assert np.array_equal(c["pdm"][p], scipy_chessboard(oracle.mask_plane(c["mask"], p)))


def test_update_equals_dt_of_union(small_case):
    """Eq. 1 == DT(union of POM_p over S): the DT of a union is the min of the DTs, and min
    commutes with the clamp at 255."""
    c = small_case
    for tf in T.tf_edit_sequence(1, c["N"], 12) + T.special_tfs(c["N"], c["borders"]):
        dprime, s = oracle.update_tf(c["pdm"], tf)
        S = oracle.active_set(tf, c["K"])
        assert np.array_equal(dprime, scipy_chessboard(oracle.union_plane(c["mask"], S)))
        assert [p for p in range(c["K"]) if (int(s[0]) >> p) & 1] == S


def test_conservative_and_aligned(small_case):
    c = small_case
    for tf in T.tf_edit_sequence(2, c["N"], 12):
        dprime, _ = oracle.update_tf(c["pdm"], tf)
        d = oracle.full_recompute_exact(c["vol"], c["b"], c["a"], tf)
        dmm = oracle.full_recompute_minmax(c["vmin"], c["vmax"], tf)
        assert np.all(dprime <= d)       # §3.1: D' is an element-wise lower limit of D
        assert np.all(dmm <= d)          # min/max occupancy is a superset of the exact one
    for k in range(8):
        tf = T.aligned_tf(100 + k, c["N"], c["borders"])
        dprime, _ = oracle.update_tf(c["pdm"], tf)
        d = oracle.full_recompute_exact(c["vol"], c["b"], c["a"], tf)
        assert np.array_equal(dprime, d)  # §3.1: equal when no partition is mixed


def test_minmax_occupancy_matches_prefix_count(small_case):
    c = small_case
    for tf in T.tf_edit_sequence(3, c["N"], 6):
        vis = tf[:, 3] > 0
        cnt = np.concatenate([[0], np.cumsum(vis)])
        occ = (cnt[c["vmax"].astype(int) + 1] - cnt[c["vmin"].astype(int)]) > 0
        assert np.array_equal(oracle.occ_minmax(c["vmin"], c["vmax"], tf), occ)
        assert np.array_equal(oracle.full_recompute_minmax(c["vmin"], c["vmax"], tf),
                              scipy_chessboard(occ))


def test_minmax_occupancy_interval_is_closed():
    """Min/max occupancy (Krueger & Westermann blocks, §2) tests the closed range
    [min, max]: a TF visible at exactly one intensity occupies a block iff that intensity
    is the block's minimum, its maximum or lies between them."""
    vmin = np.array([[[3, 5, 0, 9]]], dtype=np.uint16)
    vmax = np.array([[[7, 5, 0, 12]]], dtype=np.uint16)
    N = 16
    for i in range(N):
        want = ((vmin <= i) & (i <= vmax)).astype(np.uint8)
        got = oracle.occ_minmax(vmin, vmax, T.single_intensity_tf(N, i))
        assert np.array_equal(got, want), i


def test_exact_occupancy_matches_filters(small_case):
    c = small_case
    for tf in T.tf_edit_sequence(4, c["N"], 4):
        vis = tf[:, 3] > 0
        v = vis[np.minimum(c["vol"].astype(int), c["N"] - 1)].astype(np.uint8)
        d = ndi.maximum_filter(v, size=2 * c["a"] + 1, mode="constant", cval=0)
        occ = block_reduce(d, c["b"], np.max, 0)
        assert np.array_equal(oracle.full_recompute_exact(c["vol"], c["b"], c["a"], tf),
                              scipy_chessboard(occ))


def test_special_tfs(small_case):
    c = small_case
    N, K = c["N"], c["K"]
    z = T.zero_tf(N)
    dprime, s = oracle.update_tf(c["pdm"], z)
    assert int(s[0]) == 0 and np.all(dprime == 255)
    assert np.all(oracle.full_recompute_exact(c["vol"], c["b"], c["a"], z) == 255)
    allv = T.all_visible_tf(N)
    assert np.all(oracle.full_recompute_exact(c["vol"], c["b"], c["a"], allv) == 0)
    dprime, s = oracle.update_tf(c["pdm"], allv)
    assert int(s[0]) == (1 << K) - 1 and np.all(dprime == 0)
    tf = T.single_intensity_tf(N, 77)
    assert oracle.active_set(tf, K) == [77 * K // N]
    nan_tf = T.zero_tf(N)
    nan_tf[5, 3] = np.nan
    nan_tf[6, 3] = -0.0
    nan_tf[7, 3] = -1.0
    assert oracle.active_set(nan_tf, K) == []


def test_one_partition_and_exact_classes():
    rng = np.random.default_rng(8)
    N = 16
    vol = rand_volume(rng, (6, 7, 9), N, np.uint8)
    # K = 1: S = {0} iff any alpha is non-zero; D' is then the DT of "block non-empty" = 0
    _, pdm, _, _ = oracle.build_partitions(vol, 2, 1, N, 1)
    assert np.all(pdm == 0)
    # K = N, b = 1, a = 0: every partition is one intensity, so D' == D for every TF
    _, pdm, _, _ = oracle.build_partitions(vol, 1, 0, N, N)
    for tf in T.tf_edit_sequence(9, N, 10):
        dprime, _ = oracle.update_tf(pdm, tf)
        assert np.array_equal(dprime, oracle.full_recompute_exact(vol, 1, 0, tf))
