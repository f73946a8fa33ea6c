"""The update's plane order and its stop at 0 (Eq. 1 read most-covered plane first; a
16-byte chunk whose minimum is 0 in every byte loads no further plane), through the C ABI.

D' must not change: every case is compared with the oracle or with the value the
definition fixes.  The plane bytes the combine loads (dm_set_profile_counter) are pinned
where the schedule fixes them:
  * one active partition: every chunk of its plane is loaded once, so exactly G bytes;
  * a volume whose every block lies in the LAST partition, all partitions active: that
    plane is all 0 and is ranked first, so the per-chunk path loads only the batches of 8
    planes that are in flight before the first batch is folded (two or three, by the
    pipeline depth) and no more: at most 24 G bytes for K = 64, where ascending order
    would load all 64 G;
  * the same on a map large enough for the plane-major tiles: the planes in flight before
    the first is folded (at most three) per tile, so well under K G bytes;
and bounded by |S| G everywhere else.
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
    assert loaded % (8 * eng.G) == 0                 # whole batches of 8 planes
    assert 8 * eng.G <= loaded <= 24 * eng.G         # ascending order: 64 G


def test_plane_major_tiles_stop_at_zero():
    # b = 1: 21 M blocks, enough for the plane-major tiles of the update kernel
    N, K = 256, 8
    X, Y, Z = 512, 256, 160
    vol = np.full((Z, Y, X), 250, dtype=np.uint8)            # partition 7 everywhere
    eng = _engine((X, Y, Z), np.uint8, 1, 0, K, N)
    eng.build_partitions(_dev(vol))
    tf = T.all_visible_tf(N)
    d, loaded = _counted_update(eng, tf)
    assert not d.any()
    assert eng.G <= loaded <= 4 * eng.G              # all K planes: 8 G


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
    assert loaded % (8 * b.G) == 0 and 8 * b.G <= loaded <= 24 * b.G
