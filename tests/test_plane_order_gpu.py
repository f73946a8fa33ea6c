"""The update's reading schedule (Eq. 1 without the range index), through the C ABI.

Maps of about 5 M blocks or more are read region by region (4096 blocks): the active
planes in ascending order of their minimum over the region (ties in the plane order, most
zero bytes first), a 16-byte chunk whose minimum is 0 in every byte loading no further
plane, and the region stopping once the next plane's regional minimum is at least the
largest minimum of the region.  Smaller maps are read chunk by chunk, 8 planes per batch
in the plane order, with the same stop at 0.

D' must not change: every case is compared with the oracle or with the value the
definition fixes.  The plane bytes the combine loads (dm_set_profile_counter) are pinned
where the schedule fixes them:
  * one active partition present near every block: each chunk of its plane once, G bytes;
  * every block in the LAST partition (that plane 0 everywhere, the others 255), all K = 64
    partitions active: the per-chunk path loads the two batches in flight before the first
    is folded, 16 G; the region path loads that plane and stops, G (every active plane
    would be 64 G);
  * two halves of different material, both visible: each region reads its own material's
    plane and stops, G, where one order for the whole map would read about 1.5 G;
  * after dm_mark_built (bounds taken from the planes rather than the z pass): the same.
Everywhere else the count is bounded by |S| G.
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


def _engine(dims, dtype, b, a, K, N):
    from paper_2407_21552_gb300 import DM_U8, DM_U16
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    return PartitionedDistanceMaps(dims, DM_U8 if dtype == np.uint8 else DM_U16, b, a, K, N)


def _dev(vol_np):
    if vol_np.dtype == np.uint8:
        return torch.from_numpy(vol_np).cuda()
    return torch.from_numpy(vol_np.view(np.int16)).cuda()


def _counted_update(eng, tf_np):
    """(D', plane bytes loaded) of one update."""
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = torch.empty(eng.G, dtype=torch.uint8, device="cuda")
    eng.set_profile_counter(cnt)
    try:
        eng.update_tf(torch.from_numpy(tf_np).cuda(), out=out)
        eng.sync()
    finally:
        eng.set_profile_counter(None)
    return out.cpu().numpy(), int(cnt.item())


def _active(tf_np, K):
    return len(oracle.active_set(tf_np, K))


@pytest.mark.parametrize("dims", [(128, 128, 128), (130, 67, 45)])
def test_one_active_partition_loads_its_plane_once(dims):
    X, Y, Z = dims
    vol = synth.as_numpy(synth.volume_of("u8", (X, Y, Z), 3))
    N, K = 256, 16
    eng = _engine(dims, np.uint8, 4, 1, K, N)
    eng.build_partitions(_dev(vol))
    _, pdm, _, _ = oracle.build_partitions(vol, 4, 1, N, K)
    i = int(np.median(vol))                          # an intensity the volume holds
    tf = T.single_intensity_tf(N, i)
    assert _active(tf, K) == 1
    d, loaded = _counted_update(eng, tf)
    assert np.array_equal(d, oracle.update_tf(pdm, tf)[0].reshape(-1))
    assert loaded == eng.G


def test_covering_plane_is_read_first():
    N, K = 256, 64
    vol = np.full((128, 128, 128), 255, dtype=np.uint8)      # partition 63 everywhere
    eng = _engine((128, 128, 128), np.uint8, 4, 1, K, N)
    eng.build_partitions(_dev(vol))
    tf = T.all_visible_tf(N)
    assert _active(tf, K) == K
    d, loaded = _counted_update(eng, tf)
    assert not d.any()                               # Eq. 1: plane 63 is 0 everywhere
    assert eng.G % 16 == 0
    assert loaded == 16 * eng.G                      # every active plane: 64 G


def test_large_map_reads_the_covering_plane_only():
    # b = 1: 21 M blocks, 5120 regions over every warp of the grid
    N, K = 256, 8
    X, Y, Z = 512, 256, 160
    vol = np.full((Z, Y, X), 250, dtype=np.uint8)            # partition 7 everywhere
    eng = _engine((X, Y, Z), np.uint8, 1, 0, K, N)
    eng.build_partitions(_dev(vol))
    tf = T.all_visible_tf(N)
    d, loaded = _counted_update(eng, tf)
    assert not d.any()
    assert loaded == eng.G                           # all K planes: 8 G


def test_random_edits_same_maps_counted_or_not():
    N, K = 256, 16
    vol = synth.as_numpy(synth.tiny_volume(0))
    eng = _engine((128, 128, 128), np.uint8, 4, 1, K, N)
    eng.build_partitions(_dev(vol))
    _, pdm, _, _ = oracle.build_partitions(vol, 4, 1, N, K)
    out = torch.empty(eng.G, dtype=torch.uint8, device="cuda")
    for tf in synth.tf_edit_sequence(0, N, 20):
        want = oracle.update_tf(pdm, tf)[0].reshape(-1)
        eng.update_tf(torch.from_numpy(tf).cuda(), out=out)
        eng.sync()
        assert np.array_equal(out.cpu().numpy(), want)
        d1, c1 = _counted_update(eng, tf)
        d2, c2 = _counted_update(eng, tf)
        assert np.array_equal(d1, want) and np.array_equal(d2, want)
        assert c1 == c2 <= _active(tf, K) * eng.G


def test_mark_built_ranks_the_loaded_planes(tmp_path):
    N, K = 256, 64
    vol = np.full((128, 128, 128), 255, dtype=np.uint8)
    a = _engine((128, 128, 128), np.uint8, 4, 1, K, N)
    a.build_partitions(_dev(vol))
    a.sync()
    path = str(tmp_path / "maps.npz")
    a.save(path)
    b = _engine((128, 128, 128), np.uint8, 4, 1, K, N)     # fresh scratch: no order yet
    b.load(path)
    tf = T.all_visible_tf(N)
    d, loaded = _counted_update(b, tf)
    assert not d.any()
    assert loaded == 16 * b.G


def test_regions_read_their_own_material_first():
    # b = 1, apron 0: 8.4 M blocks, 2048 regions, each inside one half
    N, K = 256, 16
    X, Y, Z = 512, 256, 64
    vol = np.full((Z, Y, X), 40, dtype=np.uint8)            # partition 2 ...
    vol[Z // 2:] = 200                                       # ... and 12 (upper half)
    eng = _engine((X, Y, Z), np.uint8, 1, 0, K, N)
    eng.build_partitions(_dev(vol))
    tf = T.zero_tf(N)
    tf[40, 3] = tf[200, 3] = 1.0
    assert oracle.active_set(tf, K) == [2, 12]
    d, loaded = _counted_update(eng, tf)
    assert not d.any()                               # every block holds a visible material
    assert loaded == eng.G


def test_region_bounds_after_mark_built():
    N, K = 256, 8
    X, Y, Z = 512, 256, 64
    vol = np.full((Z, Y, X), 250, dtype=np.uint8)            # partition 7 everywhere
    eng = _engine((X, Y, Z), np.uint8, 1, 0, K, N)
    eng.build_partitions(_dev(vol))
    eng.offload()                                    # planes to host, scratch released
    eng.reload()                                     # dm_mark_built: bounds from the planes
    d, loaded = _counted_update(eng, T.all_visible_tf(N))
    assert not d.any()
    assert loaded == eng.G


def test_region_path_matches_the_oracle():
    # b = 1: 6.3 M blocks of a noise-and-ellipsoids volume, read region by region
    N, K = 256, 16
    X, Y, Z = 512, 256, 48
    vol = synth.as_numpy(synth.volume_of("u8", (X, Y, Z), 9))
    eng = _engine((X, Y, Z), np.uint8, 1, 0, K, N)
    eng.build_partitions(_dev(vol))
    _, pdm, _, _ = oracle.build_partitions(vol, 1, 0, N, K)
    for tf in synth.tf_edit_sequence(9, N, 6):
        want = oracle.update_tf(pdm, tf)[0].reshape(-1)
        d, loaded = _counted_update(eng, tf)
        assert np.array_equal(d, want)
        assert loaded <= _active(tf, K) * eng.G


@pytest.mark.parametrize("dims", [(512, 256, 48), (64, 512, 160)])
def test_row_bounds_equal_plane_bounds(dims):
    # gx (512, or 64) divides 4096: dm_build_partitions takes the region bounds from the
    # masks' rows (ORed by the x pass itself for 512-block rows, by a separate kernel for
    # 64-block rows, which the x pass takes one warp per row); dm_mark_built (offload +
    # reload) takes them from the planes.  Both are the exact regional minima, so the
    # update (region by region at these 5-6 M blocks) reads the same bytes after either.
    N, K = 256, 16
    X, Y, Z = dims
    vol = synth.as_numpy(synth.volume_of("u8", (X, Y, Z), 11))
    eng = _engine((X, Y, Z), np.uint8, 1, 0, K, N)
    eng.build_partitions(_dev(vol))
    tfs = synth.tf_edit_sequence(11, N, 5)
    first = [_counted_update(eng, tf) for tf in tfs]
    eng.offload()
    eng.reload()
    for tf, (d1, c1) in zip(tfs, first):
        d2, c2 = _counted_update(eng, tf)
        assert np.array_equal(d1, d2)
        assert c1 == c2
