"""GPU path vs the CPU oracle, bit-exact (integer work; §3.2 uint8 maps).

Every call goes through the C ABI (ctypes) of libdm; torch only allocates device memory.
Covered: the tiny workload (128^3 uint8, K=16, 100 TF edits + special TFs), the CT
workload (512^3 12-bit, K=32, N=4096), ragged volumes (dims not multiples of b), several
tiles and partial tiles in every kernel, b in {1,2,3,4,8}, apron 0..2, K up to 256 (four
mask words), explicit borders (a separate partition for the minimum intensity, §4.2),
voxels above the TF domain, lines longer than 255 blocks (clamping), degenerate volumes.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from synth import tfs as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _engine(vol_np, b, a, N, K, borders=None, exact=False):
    from paper_2407_21552_gb300 import DM_U8, DM_U16, DM_OCC_EXACT, DM_OCC_MINMAX
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    Z, Y, X = vol_np.shape
    dt = DM_U8 if vol_np.dtype == np.uint8 else DM_U16
    return PartitionedDistanceMaps((X, Y, Z), dt, b, a, K, N, borders=borders,
                                   occ_mode=DM_OCC_EXACT if exact else DM_OCC_MINMAX)


def _to_dev(vol_np):
    if vol_np.dtype == np.uint8:
        return torch.from_numpy(vol_np).cuda()
    return torch.from_numpy(vol_np.view(np.int16)).cuda()


def check_build(vol_np, b, a, N, K, borders=None):
    eng = _engine(vol_np, b, a, N, K, borders)
    vd = _to_dev(vol_np)
    eng.build_partitions(vd)
    eng.sync()
    mask_o, pdm_o, vmin_o, vmax_o = oracle.build_partitions(vol_np, b, a, N, K, borders)
    mask_g = eng.mask_words().cpu().numpy().view(np.uint64)
    assert np.array_equal(mask_g, mask_o), "POM bit masks differ"
    mm = eng.minmax_pairs().cpu().numpy()
    if vol_np.dtype == np.uint16:
        mm = mm.view(np.uint16)
    assert np.array_equal(mm[..., 0].astype(np.int64), vmin_o.astype(np.int64)), "block min"
    assert np.array_equal(mm[..., 1].astype(np.int64), vmax_o.astype(np.int64)), "block max"
    pdm_g = eng.pdm_planes().cpu().numpy()
    for p in range(K):
        assert np.array_equal(pdm_g[p], pdm_o[p]), f"PDM plane {p} differs"
    return eng, vd, (mask_o, pdm_o, vmin_o, vmax_o)


def check_updates(eng, vd, vol_np, ref, tfs, b, a, borders=None, full=True, exact_every=0):
    from paper_2407_21552_gb300 import DM_OCC_EXACT
    mask_o, pdm_o, vmin_o, vmax_o = ref
    K = pdm_o.shape[0]
    W = (K + 63) // 64
    am = torch.zeros(W, dtype=torch.int64, device="cuda")
    for k, tf in enumerate(tfs):
        tfd = torch.from_numpy(tf).cuda()
        out = eng.update_tf(tfd, active_mask=am)
        want, smask = oracle.update_tf(pdm_o, tf, borders)
        got = out.cpu().numpy().reshape(want.shape)
        assert np.array_equal(got, want), f"D' differs on TF {k}"
        assert np.array_equal(am.cpu().numpy().view(np.uint64), smask), f"S differs on TF {k}"
        if full:
            d = eng.full_recompute(tfd).cpu().numpy().reshape(want.shape)
            assert np.array_equal(d, oracle.full_recompute_minmax(vmin_o, vmax_o, tf)), \
                f"min/max full recompute differs on TF {k}"
        if exact_every and k % exact_every == 0:
            ex = _engine(vol_np, b, a, vol_tf_size(tf), K, borders, exact=True)
            ex._minmax = None
            ex._bind()
            d = ex.full_recompute(tfd, volume=vd).cpu().numpy().reshape(want.shape)
            assert np.array_equal(d, oracle.full_recompute_exact(vol_np, b, a, tf)), \
                f"exact full recompute differs on TF {k}"
            ex.close()
    eng.sync()


def vol_tf_size(tf):
    return tf.shape[0]


# ------------------------------------------------------------------------ tiny workload
@pytest.fixture(scope="module")
def tiny():
    w = synth.WORKLOADS["tiny"]
    vol = synth.as_numpy(synth.make_volume("tiny"))
    eng, vd, ref = check_build(vol, w["block"], w["apron"], w["N"], w["K"])
    return dict(w=w, vol=vol, eng=eng, vd=vd, ref=ref)


def test_tiny_build_parity(tiny):
    assert tiny["ref"][1].shape == (16, 32, 32, 32)


def test_tiny_100_edits_and_special_tfs(tiny):
    w = tiny["w"]
    tfs = T.tf_edit_sequence(w["seed"], w["N"], w["edits"])
    tfs += T.special_tfs(w["N"], T.uniform_borders(w["N"], w["K"]))
    check_updates(tiny["eng"], tiny["vd"], tiny["vol"], tiny["ref"], tfs, w["block"],
                  w["apron"], exact_every=10)


def test_host_buffer_update_matches(tiny):
    w = tiny["w"]
    eng = tiny["eng"]
    tf = T.tf_edit_sequence(77, w["N"], 1)[0]
    h_tf = torch.from_numpy(tf).pin_memory()
    h_out = torch.empty(eng.G, dtype=torch.uint8).pin_memory()
    eng.update_tf_host(h_tf, h_out)
    want, _ = oracle.update_tf(tiny["ref"][1], tf)
    assert np.array_equal(h_out.numpy().reshape(want.shape), want)
    # pageable host memory works too
    h_out2 = torch.empty(eng.G, dtype=torch.uint8)
    eng.update_tf_host(torch.from_numpy(tf.copy()), h_out2)
    assert np.array_equal(h_out2.numpy().reshape(want.shape), want)


def test_new_scratch_needs_mark_built(tiny):
    """The scratch buffer carries a per-context table (the partition of every intensity):
    after binding a fresh scratch buffer the updates refuse to run until dm_mark_built has
    rewritten it, and then give the oracle's D' again, single and batched (explicit, uneven
    borders: the kernels' non-uniform path)."""
    from paper_2407_21552_gb300 import _abi as A
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    w = tiny["w"]
    X, Y, Z = w["dims"]
    borders = [0, 7, 40, 41, 100, 130, 200, 255, 256]          # explicit, uneven, K = 8
    eng = PartitionedDistanceMaps((X, Y, Z), A.DM_U8, w["block"], w["apron"], 8, w["N"],
                                  borders=borders)
    eng.build_partitions(tiny["vd"])
    tf = T.tf_edit_sequence(31, w["N"], 1)[0]
    tfd = torch.from_numpy(tf).cuda()
    _, pdm_o, _, _ = oracle.build_partitions(tiny["vol"], w["block"], w["apron"], w["N"], 8,
                                             np.array(borders, dtype=np.int32))
    want, _ = oracle.update_tf(pdm_o, tf, np.array(borders, dtype=np.int32))
    assert np.array_equal(eng.update_tf(tfd).cpu().numpy().reshape(want.shape), want)
    eng._scratch = torch.full_like(eng._scratch, 0xAB)            # tables not written here
    eng._bind()
    with pytest.raises(A.DmError):
        eng.update_tf(tfd)
    A.dm_mark_built(eng.ctx, A.dm_config_hash(eng.ctx), True,
                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert np.array_equal(eng.update_tf(tfd).cpu().numpy().reshape(want.shape), want)
    out = torch.empty(eng.G, dtype=torch.uint8, device="cuda")
    A.dm_update_tf_batch([(eng.ctx, tfd.data_ptr(), out.data_ptr())], None,
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert np.array_equal(out.cpu().numpy().reshape(want.shape), want)
    eng.close()


def test_repeated_updates_on_other_stream(tiny):
    w = tiny["w"]
    eng = tiny["eng"]
    s = torch.cuda.Stream()
    tfs = T.tf_edit_sequence(5, w["N"], 8)
    outs = []
    with torch.cuda.stream(s):
        for tf in tfs:
            outs.append(eng.update_tf(torch.from_numpy(tf).cuda(), stream=s))
    s.synchronize()
    for tf, o in zip(tfs, outs):
        want, _ = oracle.update_tf(tiny["ref"][1], tf)
        assert np.array_equal(o.cpu().numpy().reshape(want.shape), want)


# --------------------------------------------------------------- ragged / odd configs
def rand_volume(rng, shape, N, dtype, blob=3):
    v = rng.integers(0, N, size=tuple(max(1, s // blob) for s in shape))
    v = np.kron(v, np.ones((blob, blob, blob), np.int64))
    v = np.pad(v, [(0, max(0, s - v.shape[i])) for i, s in enumerate(shape)], mode="edge")
    v = v[: shape[0], : shape[1], : shape[2]]
    noise = rng.integers(-N // 16, N // 16 + 1, size=shape)
    v = np.clip(v + noise * (rng.uniform(size=shape) < 0.2), 0, N - 1)
    return v.astype(dtype)


CASES = [
    # shape (Z, Y, X), b, a, N, K, dtype, borders
    ((23, 29, 37), 4, 1, 256, 7, np.uint8, None),
    ((23, 29, 37), 4, 0, 256, 16, np.uint8, None),
    ((9, 10, 11), 3, 2, 4096, 32, np.uint16, None),
    ((17, 33, 65), 2, 1, 300, 65, np.uint16, None),          # two mask words
    ((13, 21, 40), 4, 1, 4096, 256, np.uint16, None),        # four mask words
    ((12, 12, 12), 1, 0, 64, 64, np.uint8, None),            # b = 1: exact voxel classes
    ((12, 12, 12), 1, 1, 64, 5, np.uint8, None),
    ((40, 24, 72), 8, 3, 256, 16, np.uint8, None),
    ((1, 1, 1), 4, 1, 256, 16, np.uint8, None),
    ((1, 7, 130), 4, 1, 256, 3, np.uint8, None),
    ((66, 3, 2), 1, 1, 256, 1, np.uint8, None),              # K = 1
    ((16, 64, 256), 4, 1, 256, 4, np.uint8, [0, 1, 86, 171, 256]),  # rho_min partition
    ((20, 36, 128), 4, 1, 256, 16, np.uint8, None),          # aligned rows, 16-byte paths
    ((20, 36, 128), 4, 1, 4096, 32, np.uint16, None),
    ((12, 20, 264), 4, 1, 256, 16, np.uint8, None),          # 3 x tiles of 32 blocks, ragged
    ((9, 14, 392), 4, 1, 4096, 64, np.uint16, None),         # two 32-bit mask words per lane
    ((7, 9, 200), 4, 1, 4096, 200, np.uint16, None),         # eight 32-bit mask words
    ((13, 11, 132), 4, 1, 300, 33, np.uint16, None),         # K just above one word
    ((40, 33, 50), 16, 5, 256, 16, np.uint8, None),          # the largest block size
    ((10, 12, 40), 4, 1, 8192, 64, np.uint16, None),         # largest TF of the one-launch update
    ((10, 12, 40), 4, 1, 8193, 64, np.uint16, None),         # N > 8192: active set + combine
    ((11, 9, 36), 2, 1, 65536, 256, np.uint16, None),        # the largest TF and K
]


@pytest.mark.parametrize("shape,b,a,N,K,dt,borders", CASES)
def test_ragged_configs(shape, b, a, N, K, dt, borders):
    rng = np.random.default_rng(sum(shape) * 7 + b * 3 + K)
    vol = rand_volume(rng, shape, N, dt)
    if dt == np.uint16 and vol.size > 2 and N + 5 <= 0xFFFF:
        vol.reshape(-1)[::97] = N + 5        # above the TF domain: treated as N - 1
    eng, vd, ref = check_build(vol, b, a, N, K, borders)
    bd = np.asarray(borders) if borders is not None else T.uniform_borders(N, K)
    tfs = T.tf_edit_sequence(int(rng.integers(1 << 30)), N, 6) + T.special_tfs(N, bd)
    check_updates(eng, vd, vol, ref, tfs, b, a, borders, exact_every=3)
    eng.close()


# b = 4, apron 1 with rows of whole 16-byte vectors: the footprint kernel with 16-byte
# voxel loads (8 uint16 or 16 uint8 voxels, 2 or 4 blocks per lane).  Its edges: CTAs with
# few active lanes, block rows and z chunks that the grid ends inside, volumes ending 0, 1,
# 2 or 3 slices into their last block, one and two mask words, TF tables up to 64 KiB,
# voxels above the TF domain (clamped on both sides), explicit borders.
VEC_CASES = [
    # shape (Z, Y, X), N, K, dtype, borders
    ((23, 37, 72), 4096, 64, np.uint16, None),      # 9 lanes; 10 block rows; gz = 6
    ((36, 64, 264), 4096, 48, np.uint16, None),     # 33 lanes: 2 CTAs in x; 2 z chunks
    ((34, 30, 8), 1000, 20, np.uint16, None),       # one lane per CTA; Z ends at slice 1
    ((33, 70, 48), 256, 32, np.uint8, None),        # 3 lanes of 16 voxels; Z ends at slice 0
    ((17, 9, 32), 200, 16, np.uint8, None),         # N < 256: uint8 voxels clamped
    ((8, 8, 16), 16, 4, np.uint16, None),           # tiny N: most voxels clamped
    ((19, 41, 80), 8192, 64, np.uint16, None),      # the largest table (64 KiB)
    ((21, 26, 96), 4096, 41, np.uint16,
     [0, 1] + [int(v) for v in np.linspace(90, 4000, 39).astype(int)] + [4096]),
]


@pytest.mark.parametrize("shape,N,K,dt,borders", VEC_CASES)
def test_vector_footprint_edges(shape, N, K, dt, borders):
    rng = np.random.default_rng(sum(shape) * 11 + K)
    vol = rand_volume(rng, shape, N, dt)
    top = 0xFFFF if dt == np.uint16 else 0xFF
    if N - 1 < top:
        vol.reshape(-1)[::53] = min(top, N + 7)      # above the TF domain: treated as N - 1
        vol.reshape(-1)[::211] = top
    eng, vd, ref = check_build(vol, 4, 1, N, K, borders)
    bd = np.asarray(borders) if borders is not None else T.uniform_borders(N, K)
    tfs = T.tf_edit_sequence(int(rng.integers(1 << 30)), N, 4) + T.special_tfs(N, bd)[:6]
    check_updates(eng, vd, vol, ref, tfs, 4, 1, borders, exact_every=2)
    eng.close()


RAGGED_CASES = [
    # shape (Z, Y, X), N, K, dtype, borders, volume offset in voxels: rows that are not a
    # whole number of 16-byte vectors (every row starts at another offset within its
    # vector), partial blocks at the row end, an odd number of blocks per row, several
    # CTAs along x, and volumes that start off a 16-byte boundary
    ((23, 37, 70), 4096, 64, np.uint16, None, 0),     # 9 lanes, the last one 6 voxels
    ((20, 30, 267), 4096, 32, np.uint16, None, 0),    # 2 CTAs in x; gx = 67; 3-voxel block
    ((17, 21, 5), 4096, 16, np.uint16, None, 0),      # one partial lane
    ((19, 23, 531), 256, 32, np.uint8, None, 0),      # 2 CTAs in x; gx = 133
    ((15, 26, 37), 200, 16, np.uint8, None, 0),       # N < 256: voxels clamped
    ((21, 26, 99), 4096, 41, np.uint16,
     [0, 1] + [int(v) for v in np.linspace(90, 4000, 39).astype(int)] + [4096], 0),
    ((18, 22, 64), 4096, 32, np.uint16, None, 1),     # whole-vector rows, unaligned volume
    ((13, 19, 45), 256, 16, np.uint8, None, 3),       # ragged rows, unaligned volume
    ((16, 17, 130), 4096, 64, np.uint16, None, 5),
]


@pytest.mark.parametrize("shape,N,K,dt,borders,offset", RAGGED_CASES)
def test_vector_footprint_ragged_rows(shape, N, K, dt, borders, offset):
    rng = np.random.default_rng(sum(shape) * 13 + K + offset)
    vol = rand_volume(rng, shape, N, dt)
    top = 0xFFFF if dt == np.uint16 else 0xFF
    if N - 1 < top:
        vol.reshape(-1)[::47] = min(top, N + 7)      # above the TF domain: treated as N - 1
    eng = _engine(vol, 4, 1, N, K, borders)
    src = vol if dt == np.uint8 else vol.view(np.int16)
    flat = torch.from_numpy(np.ascontiguousarray(src).reshape(-1)).cuda()
    buf = torch.zeros(flat.numel() + offset + 8, dtype=flat.dtype, device="cuda")
    vd = buf[offset: offset + flat.numel()]
    vd.copy_(flat)
    eng.build_partitions(vd)
    eng.sync()
    ref = oracle.build_partitions(vol, 4, 1, N, K, borders)
    mask_o, pdm_o, vmin_o, vmax_o = ref
    assert np.array_equal(eng.mask_words().cpu().numpy().view(np.uint64), mask_o), "POM masks"
    mm = eng.minmax_pairs().cpu().numpy()
    if dt == np.uint16:
        mm = mm.view(np.uint16)
    assert np.array_equal(mm[..., 0].astype(np.int64), vmin_o.astype(np.int64)), "block min"
    assert np.array_equal(mm[..., 1].astype(np.int64), vmax_o.astype(np.int64)), "block max"
    assert np.array_equal(eng.pdm_planes().cpu().numpy(), pdm_o), "PDM planes"
    bd = np.asarray(borders) if borders is not None else T.uniform_borders(N, K)
    tfs = T.tf_edit_sequence(int(rng.integers(1 << 30)), N, 3) + T.special_tfs(N, bd)[:4]
    check_updates(eng, vd, vol, ref, tfs, 4, 1, borders, exact_every=2)
    eng.close()


@pytest.mark.parametrize("shape", [(4 * 600, 8, 8), (8, 4 * 300, 8), (8, 8, 4 * 700)])
def test_long_lines_clamp_at_255(shape):
    """One occupied corner; lines of 300-700 blocks need the 255 clamp on every axis."""
    N, K, b, a = 256, 2, 4, 0
    vol = np.zeros(shape, np.uint8)
    vol[0, 0, 0] = 200                     # partition 1 occupied in block (0, 0, 0) only
    eng, vd, ref = check_build(vol, b, a, N, K)
    pd = ref[1][1]
    assert pd.max() == 255 and pd.min() == 0
    tf = T.single_intensity_tf(N, 200)
    check_updates(eng, vd, vol, ref, [tf, T.zero_tf(N), T.all_visible_tf(N)], b, a,
                  exact_every=1)
    eng.close()


def test_sparse_and_dense_lines_mix():
    """Wide grid (several x tiles) with sparse occupancy: long searches in every pass."""
    rng = np.random.default_rng(99)
    N, K, b, a = 256, 8, 4, 1
    vol = np.zeros((64, 96, 640), np.uint8)
    pts = rng.integers(0, [64, 96, 640], size=(40, 3))
    for z, y, x in pts:
        vol[z, y, x] = rng.integers(1, 255)
    eng, vd, ref = check_build(vol, b, a, N, K)
    tfs = T.tf_edit_sequence(3, N, 5) + [T.single_intensity_tf(N, int(vol[tuple(pts[0])]))]
    check_updates(eng, vd, vol, ref, tfs, b, a, exact_every=2)
    eng.close()


# ---------------------------------------------------------------------- CT workload
@pytest.fixture(scope="module")
def ct():
    w = synth.WORKLOADS["ct"]
    vol_t = synth.make_volume("ct", device="cuda")
    vol = synth.as_numpy(vol_t)
    eng, vd, ref = check_build(vol, w["block"], w["apron"], w["N"], w["K"])
    return dict(w=w, vol=vol, eng=eng, vd=vd, ref=ref)


def test_ct_build_parity(ct):
    assert ct["ref"][1].shape == (32, 128, 128, 128)


def test_ct_edits(ct):
    w = ct["w"]
    tfs = T.tf_edit_sequence(w["seed"], w["N"], w["edits"])
    picked = tfs[::25] + T.special_tfs(w["N"], T.uniform_borders(w["N"], w["K"]))
    check_updates(ct["eng"], ct["vd"], ct["vol"], ct["ref"], picked, w["block"], w["apron"],
                  full=True, exact_every=20)


def test_ct_all_edits_combine(ct):
    """All 1000 edits of the workload through the combine, against the oracle."""
    w = ct["w"]
    pdm_o = ct["ref"][1]
    eng = ct["eng"]
    out = torch.empty(eng.G, dtype=torch.uint8, device="cuda")
    for k, tf in enumerate(T.tf_edit_sequence(w["seed"], w["N"], w["edits"])):
        if k % 4:
            continue
        eng.update_tf(torch.from_numpy(tf).cuda(), out=out)
        want, _ = oracle.update_tf(pdm_o, tf)
        assert np.array_equal(out.cpu().numpy().reshape(want.shape), want), k


def test_checkpoint_resume_without_recompute(tiny, tmp_path):
    """Maps saved from a built context and loaded into a fresh one serve the same updates
    and full recomputes; maps of another configuration are refused."""
    from paper_2407_21552_gb300 import DM_U8, DmError
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    w = tiny["w"]
    path = str(tmp_path / "maps.npz")
    tiny["eng"].save(path)
    X, Y, Z = w["dims"]
    fresh = PartitionedDistanceMaps((X, Y, Z), DM_U8, w["block"], w["apron"], w["K"], w["N"])
    fresh.load(path)
    for tf in T.tf_edit_sequence(41, w["N"], 3):
        tfd = torch.from_numpy(tf).cuda()
        assert torch.equal(fresh.update_tf(tfd), tiny["eng"].update_tf(tfd))
        assert torch.equal(fresh.full_recompute(tfd), tiny["eng"].full_recompute(tfd))
    other = PartitionedDistanceMaps((X, Y, Z), DM_U8, w["block"], 0, w["K"], w["N"])
    with pytest.raises(DmError):
        other.load(path)
    fresh.close()
    other.close()


# ------------------------------------------------------- seeded random configurations
def random_config(seed):
    """A random configuration: dims 1..70 (1..40 when b <= 2), b in 1..16, apron 0..b,
    uint8 / 12-bit / 16-bit, N from 2 to 65536, K from 1 to min(N, 256), and explicit
    random borders for about a third of them."""
    rng = np.random.default_rng(9000 + seed)
    b = int(rng.choice([1, 2, 3, 4, 4, 4, 5, 7, 8, 16]))
    a = int(rng.integers(0, b + 1)) if rng.random() < 0.2 else int(rng.integers(0, min(b, 2) + 1))
    u16 = rng.random() < 0.5
    N = int(rng.choice([256, 300, 1024, 4096, 4096, 65536])) if u16 else int(rng.choice([2, 16, 100, 256]))
    K = int(rng.integers(1, min(N, 16) + 1)) if rng.random() < 0.5 else int(rng.integers(1, min(N, 256) + 1))
    hi = 40 if b <= 2 else 70
    shape = tuple(int(rng.integers(1, hi + 1)) for _ in range(3))
    borders = None
    if K > 1 and rng.random() < 0.35:
        inner = np.sort(rng.choice(np.arange(1, N), K - 1, replace=False))
        borders = [0] + [int(v) for v in inner] + [N]
    return shape, b, a, N, K, (np.uint16 if u16 else np.uint8), borders, rng


@pytest.mark.parametrize("seed", range(24))
def test_random_configs(seed):
    shape, b, a, N, K, dt, borders, rng = random_config(seed)
    vol = rand_volume(rng, shape, N, dt, blob=int(rng.integers(1, 5)))
    eng, vd, ref = check_build(vol, b, a, N, K, borders)
    bd = np.asarray(borders) if borders is not None else T.uniform_borders(N, K)
    tfs = T.tf_edit_sequence(int(rng.integers(1 << 30)), N, 4) + T.special_tfs(N, bd)
    check_updates(eng, vd, vol, ref, tfs, b, a, borders, exact_every=5)
    eng.close()


@pytest.mark.parametrize("shape", [(271, 269, 277),     # 308 tiles: a grid multiple of them
                                   (303, 303, 303)])    # 424 tiles: all of them
def test_plane_major_tiles_of_large_maps(shape):
    """Maps of 20-28 M blocks (b = 1) take the update's plane-major tiles; whole tiles, the
    chunks past them and a ragged byte tail all match the oracle."""
    rng = np.random.default_rng(sum(shape))
    vol = rand_volume(rng, shape, 256, np.uint8, blob=9)
    N, K = 256, 4
    eng = _engine(vol, 1, 0, N, K)
    eng.build_partitions(_to_dev(vol))
    _, pdm, _, _ = oracle.build_partitions(vol, 1, 0, N, K)
    assert eng.G % 16 != 0 and eng.G // 16 // (512 * 8) >= 2 * 152
    bd = T.uniform_borders(N, K)
    for tf in T.tf_edit_sequence(int(rng.integers(1 << 30)), N, 3) + T.special_tfs(N, bd)[:3]:
        got = eng.update_tf(torch.from_numpy(tf).cuda()).cpu().numpy()
        want, _ = oracle.update_tf(pdm, tf)
        assert np.array_equal(got.reshape(want.shape), want)
    eng.close()


def random_large_config(seed):
    """Larger random shapes (sides up to 240 voxels, grids up to 300 K blocks) so that every
    kernel spans several CTAs and tiles per axis; K up to 64, N up to 65536."""
    rng = np.random.default_rng(50000 + seed)
    b = int(rng.choice([1, 2, 3, 4, 4, 4, 5, 8, 16]))
    a = int(rng.integers(0, min(b, 2) + 1)) if rng.random() < 0.8 else int(rng.integers(0, b + 1))
    u16 = rng.random() < 0.5
    N = int(rng.choice([256, 1000, 4096, 65536])) if u16 else int(rng.choice([64, 256]))
    K = int(rng.integers(1, min(N, 64) + 1))
    while True:
        shape = tuple(int(rng.integers(1, 241)) for _ in range(3))
        if (np.prod([-(-s // b) for s in shape]) <= 300_000
                and np.prod(shape) <= 8_000_000):
            break
    borders = None
    if K > 1 and rng.random() < 0.3:
        inner = np.sort(rng.choice(np.arange(1, N), K - 1, replace=False))
        borders = [0] + [int(v) for v in inner] + [N]
    return shape, b, a, N, K, (np.uint16 if u16 else np.uint8), borders, rng


@pytest.mark.parametrize("seed", range(12))
def test_random_large_configs(seed):
    shape, b, a, N, K, dt, borders, rng = random_large_config(seed)
    vol = rand_volume(rng, shape, N, dt, blob=int(rng.integers(1, 9)))
    eng, vd, ref = check_build(vol, b, a, N, K, borders)
    bd = np.asarray(borders) if borders is not None else T.uniform_borders(N, K)
    tfs = T.tf_edit_sequence(int(rng.integers(1 << 30)), N, 3) + T.special_tfs(N, bd)[:4]
    check_updates(eng, vd, vol, ref, tfs, b, a, borders, exact_every=4)
    eng.close()
