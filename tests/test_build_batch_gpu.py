"""The batched precompute (dm_build_partitions_batch) vs the CPU oracle, bit-exact.

One call builds many volumes of different size, voxel type, block, apron, K and N.  Every
kernel variant of the batched path is covered: the 16-byte vector POM kernel (uint8 /
uint16, one or two mask words, partitions by shift or by table), the general POM kernel
(volumes the vector kernel does not take: rows of a ragged width, an unaligned volume,
b != 4, apron != 1), the one-volume fallback (K > 64), x passes of one to four mask
words, 8-bit and 16-bit sweep tables (lines longer than 256 blocks), axes of a single
block, maps without min/max, the range index, and batches longer than one launch group.
The partition tables the batch writes are checked through batched TF updates.
"""
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


def _borders(N, K, kind):
    """None (uniform), or explicit ascending borders: 'skew' puts a partition of its own on
    intensity 0 (§4.2) and spreads the rest unevenly."""
    if kind is None:
        return None
    rng = np.random.default_rng(N * 1000 + K)
    inner = np.sort(rng.choice(np.arange(2, N), size=K - 2, replace=False))
    return [0, 1] + [int(v) for v in inner] + [N]


def _volume(kind, dims, seed):
    return synth.as_numpy(synth.volume_of(kind, dims, seed, device="cpu"))


def _to_dev(vol_np, offset_elems=0):
    """The volume on the device; offset_elems > 0 places it that many voxels into a larger
    buffer, so that its address is aligned to the voxel size only."""
    src = vol_np if vol_np.dtype == np.uint8 else vol_np.view(np.int16)
    flat = torch.from_numpy(np.ascontiguousarray(src).reshape(-1)).cuda()
    if offset_elems == 0:
        return flat
    buf = torch.zeros(flat.numel() + offset_elems + 8, dtype=flat.dtype, device="cuda")
    view = buf[offset_elems: offset_elems + flat.numel()]
    view.copy_(flat)
    return view


def _engine(vol_np, b, a, N, K, borders=None, with_minmax=True, index=False):
    from paper_2407_21552_gb300 import DM_U8, DM_U16, DM_INDEX_NONE, DM_INDEX_RANGES
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    Z, Y, X = vol_np.shape
    dt = DM_U8 if vol_np.dtype == np.uint8 else DM_U16
    return PartitionedDistanceMaps((X, Y, Z), dt, b, a, K, N, borders=borders,
                                   with_minmax=with_minmax,
                                   index_mode=DM_INDEX_RANGES if index else DM_INDEX_NONE)


def _check_maps(eng, vol_np, spec, ref):
    mask_o, pdm_o, vmin_o, vmax_o = ref
    K = spec["K"]
    mask_g = eng.mask_words().cpu().numpy().view(np.uint64)
    assert np.array_equal(mask_g, mask_o), f"{spec['name']}: POM bit masks differ"
    if spec.get("with_minmax", True):
        mm = eng.minmax_pairs().cpu().numpy()
        if vol_np.dtype == np.uint16:
            mm = mm.view(np.uint16)
        assert np.array_equal(mm[..., 0].astype(np.int64), vmin_o.astype(np.int64)), \
            f"{spec['name']}: block min"
        assert np.array_equal(mm[..., 1].astype(np.int64), vmax_o.astype(np.int64)), \
            f"{spec['name']}: block max"
    pdm_g = eng.pdm_planes().cpu().numpy()
    for p in range(K):
        assert np.array_equal(pdm_g[p], pdm_o[p]), f"{spec['name']}: PDM plane {p} differs"


# name, voxel kind, dims (X, Y, Z), b, apron, K, N, borders, options
MIXED = [
    ("u8 vector, shift", "u8", (64, 48, 40), 4, 1, 16, 256, None, {}),
    ("u8 vector, table", "u8", (80, 36, 52), 4, 1, 32, 256, "skew", {}),
    ("u16 vector, shift", "u16", (96, 72, 44), 4, 1, 32, 4096, None, {}),
    ("u16 vector, table", "u16", (64, 40, 60), 4, 1, 32, 4096, "skew", {}),
    ("u16 vector, 2 words, shift", "u16", (72, 64, 36), 4, 1, 64, 4096, None, {}),
    ("u16 vector, 2 words, table", "u16", (56, 44, 48), 4, 1, 48, 4096, None, {}),
    ("u8 general, ragged rows", "u8", (70, 33, 45), 4, 1, 16, 256, None, {}),
    ("u8 general, 2 words", "u8", (64, 40, 40), 4, 1, 40, 256, None, {}),
    ("u16 general, ragged rows", "u16", (70, 50, 30), 4, 1, 16, 4096, None, {}),
    ("u16 general, unaligned volume", "u16", (64, 32, 32), 4, 1, 32, 4096, None,
     {"offset": 1}),
    ("u16 general, 2 words", "u16", (66, 38, 42), 4, 1, 50, 4096, "skew", {}),
    ("u16 b=8 apron 2", "u16", (72, 64, 56), 8, 2, 16, 4096, None, {}),
    ("u8 b=2 apron 1", "u8", (40, 30, 20), 2, 1, 16, 256, None, {}),
    ("u8 b=1 apron 0", "u8", (24, 20, 16), 1, 0, 8, 256, None, {}),
    ("u16 K=100, own POM launch", "u16", (48, 40, 36), 4, 1, 100, 4096, None, {}),
    ("u8 K=200, own POM launch", "u8", (48, 32, 32), 4, 1, 200, 256, None, {}),
    ("u16 K=150, three mask words", "u16", (40, 36, 28), 4, 1, 150, 4096, "skew", {}),
    ("u8 z lines of 275 blocks", "u8", (16, 16, 1100), 4, 1, 16, 256, None, {}),
    ("u16 one block along y", "u16", (64, 3, 64), 4, 1, 32, 4096, None, {}),
    ("u8 without min/max", "u8", (48, 48, 48), 4, 1, 16, 256, None,
     {"with_minmax": False}),
    ("u16 range index", "u16", (64, 64, 64), 4, 1, 32, 4096, None, {"index": True}),
]


def _make(specs, seed0):
    out = []
    for i, (name, kind, dims, b, a, K, N, bk, opt) in enumerate(specs):
        vol_np = _volume(kind, dims, seed0 + i)
        borders = _borders(N, K, bk)
        spec = dict(name=name, b=b, a=a, K=K, N=N, borders=borders,
                    with_minmax=opt.get("with_minmax", True))
        eng = _engine(vol_np, b, a, N, K, borders, spec["with_minmax"], opt.get("index", False))
        out.append((spec, vol_np, _to_dev(vol_np, opt.get("offset", 0)), eng))
    return out


def _oracle(spec, vol_np):
    return oracle.build_partitions(vol_np, spec["b"], spec["a"], spec["N"], spec["K"],
                                   spec["borders"])


def _check_batch_updates(items, refs, seed):
    """One TF per volume through dm_update_tf_batch, which classifies intensities with the
    partition tables the batched precompute wrote; D' against the oracle's Eq. 1."""
    from paper_2407_21552_gb300 import _abi as A
    tfs, outs, batch = [], [], []
    for k, ((spec, vol_np, vd, eng), ref) in enumerate(zip(items, refs)):
        tf = T.tf_edit_sequence(seed + k, spec["N"], 1)[0]
        tfd = torch.from_numpy(tf).cuda()
        out = torch.empty(eng.G, dtype=torch.uint8, device="cuda")
        tfs.append((tf, tfd))
        outs.append(out)
        batch.append((eng.ctx, tfd.data_ptr(), out.data_ptr()))
    A.dm_update_tf_batch(batch, None, None)
    torch.cuda.synchronize()
    for (spec, vol_np, vd, eng), ref, (tf, _), out in zip(items, refs, tfs, outs):
        want, _ = oracle.update_tf(ref[1], tf, spec["borders"])
        got = out.cpu().numpy().reshape(want.shape)
        assert np.array_equal(got, want), f"{spec['name']}: D' after the batched build differs"


def test_batched_precompute_covers_every_variant():
    from paper_2407_21552_gb300.maps import build_partitions_batch
    items = _make(MIXED, 9100)
    build_partitions_batch([e for _, _, _, e in items], [v for _, _, v, _ in items])
    torch.cuda.synchronize()
    refs = []
    for spec, vol_np, vd, eng in items:
        ref = _oracle(spec, vol_np)
        _check_maps(eng, vol_np, spec, ref)
        refs.append(ref)
    _check_batch_updates(items, refs, 300)
    for _, _, _, eng in items:
        eng.close()


def test_batched_precompute_longer_than_one_launch_group():
    """70 small volumes: two launch groups of at most 64; every volume against the oracle,
    then rebuilt in place from other volumes (the maps of the first build are replaced)."""
    from paper_2407_21552_gb300.maps import build_partitions_batch
    rng = np.random.default_rng(77)
    specs = []
    for i in range(70):
        kind = "u8" if i % 2 == 0 else "u16"
        dims = tuple(int(v) for v in rng.integers(8, 41, size=3))
        if i % 5 == 0:                                   # some rows of whole vectors
            dims = (32 if kind == "u8" else 24,) + dims[1:]
        K = (8, 16, 32)[i % 3]
        specs.append((f"item {i}", kind, dims, 4, 1, K, 256 if kind == "u8" else 4096,
                      None, {}))
    items = _make(specs, 20000)
    engs = [e for _, _, _, e in items]
    build_partitions_batch(engs, [v for _, _, v, _ in items])
    torch.cuda.synchronize()
    for spec, vol_np, vd, eng in items:
        _check_maps(eng, vol_np, spec, _oracle(spec, vol_np))
    # the same contexts from new volumes of the same shapes
    second = []
    for k, (spec, vol_np, vd, eng) in enumerate(items):
        kind = "u8" if vol_np.dtype == np.uint8 else "u16"
        Z, Y, X = vol_np.shape
        v2 = _volume(kind, (X, Y, Z), 30000 + k)
        second.append((spec, v2, _to_dev(v2), eng))
    build_partitions_batch(engs, [v for _, _, v, _ in second])
    torch.cuda.synchronize()
    refs = []
    for spec, vol_np, vd, eng in second:
        ref = _oracle(spec, vol_np)
        _check_maps(eng, vol_np, spec, ref)
        refs.append(ref)
    _check_batch_updates(second[:64], refs[:64], 500)
    for eng in engs:
        eng.close()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_batched_precompute_random_configurations(seed):
    """One batch of 16 random configurations (sides 1-70, b in 1..8 with any apron up to b,
    K 1-100, N from 2 to 4096, uniform or skewed borders, uint8 or uint16, with or without
    min/max, with or without the range index) against the oracle."""
    from paper_2407_21552_gb300.maps import build_partitions_batch
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(16):
        kind = "u8" if rng.random() < 0.5 else "u16"
        dims = tuple(int(v) for v in rng.integers(1, 71, size=3))
        b = int(rng.choice([1, 2, 3, 4, 4, 4, 8]))
        a = int(rng.integers(0, b + 1)) if b > 1 else int(rng.integers(0, 2))
        a = min(a, b)
        N = int(rng.choice([2, 200, 256, 1000, 4096] if kind == "u16" else [2, 100, 256]))
        K = int(rng.integers(1, min(N, 100) + 1))
        bk = "skew" if (K >= 3 and rng.random() < 0.4) else None
        opt = {"with_minmax": bool(rng.random() < 0.7), "index": bool(rng.random() < 0.2),
               "offset": int(rng.integers(0, 3))}
        specs.append((f"random {seed}.{i}", kind, dims, b, a, K, N, bk, opt))
    items = _make(specs, 40000 + 100 * seed)
    build_partitions_batch([e for _, _, _, e in items], [v for _, _, v, _ in items])
    torch.cuda.synchronize()
    refs = []
    for spec, vol_np, vd, eng in items:
        ref = _oracle(spec, vol_np)
        _check_maps(eng, vol_np, spec, ref)
        refs.append(ref)
    _check_batch_updates(items, refs, 700 + seed)
    for _, _, _, eng in items:
        eng.close()


def test_batched_precompute_splits_the_partition_tables_by_border_count():
    """48 volumes of K = 100 carry 48 x 101 borders, more than one launch of the partition
    tables holds: the tables are built in two launches, every one still exact."""
    from paper_2407_21552_gb300.maps import build_partitions_batch
    specs = []
    for i in range(48):
        kind = "u16" if i % 3 else "u8"
        N = 4096 if kind == "u16" else 256
        dims = (8 + i % 5, 9 + i % 7, 7 + i % 4)
        specs.append((f"K=100 item {i}", kind, dims, 4, 1, 100, N, "skew" if i % 2 else None, {}))
    items = _make(specs, 60000)
    build_partitions_batch([e for _, _, _, e in items], [v for _, _, v, _ in items])
    torch.cuda.synchronize()
    refs = []
    for spec, vol_np, vd, eng in items:
        ref = _oracle(spec, vol_np)
        _check_maps(eng, vol_np, spec, ref)
        refs.append(ref)
    _check_batch_updates(items, refs, 900)
    for _, _, _, eng in items:
        eng.close()
