"""Full-size parity for the large workload (1024x1024x1795 12-bit, 256x256x449 grid, K=64),
in the configuration the benchmark runs (PartitionedDistanceMaps, default stream).

The oracle computes every POM bit mask and block min/max of the whole volume (plain C,
about 6e9 voxel visits) and these are compared in full.  Distance values are compared in
full too, every one of the 29.4 M blocks: the oracle's chamfer transform of an occupancy
grid built from the oracle's own masks gives a PDM plane (§3.1), D' for a TF (the union of
the POMs over S, whose transform equals Eq. 1's min of the PDMs) and the min/max full
recompute's D (the TF's min/max occupancy).  A few blocks are also checked against the
oracle's shell search, a third way to the same distances.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from synth import tfs as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def large():
    import __graft_entry__ as g
    g.build()
    from paper_2407_21552_gb300 import DM_U16
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    w = synth.WORKLOADS["large"]
    X, Y, Z = w["dims"]
    vol = synth.make_volume("large", device="cuda")
    eng = PartitionedDistanceMaps((X, Y, Z), DM_U16, w["block"], w["apron"], w["K"], w["N"])
    eng.build_partitions(vol)
    eng.sync()
    vol_np = synth.as_numpy(vol)
    del vol
    torch.cuda.empty_cache()
    mask_o, vmin_o, vmax_o = oracle.pom(vol_np, w["block"], w["apron"], w["N"], w["K"])
    return dict(w=w, eng=eng, mask=mask_o, vmin=vmin_o, vmax=vmax_o)


def _points(rng, grid, n):
    gz, gy, gx = grid
    pts = np.stack([rng.integers(0, gx, n), rng.integers(0, gy, n), rng.integers(0, gz, n)], 1)
    # include the grid corners and edge blocks
    corners = np.array([[0, 0, 0], [gx - 1, gy - 1, gz - 1], [gx - 1, 0, gz - 1],
                        [0, gy - 1, 0]])
    return np.concatenate([corners, pts])


def test_large_masks_and_minmax_in_full(large):
    g_mask = large["eng"].mask_words().cpu().numpy().view(np.uint64)
    assert np.array_equal(g_mask, large["mask"])
    mm = large["eng"].minmax_pairs().cpu().numpy().view(np.uint16)
    assert np.array_equal(mm[..., 0], large["vmin"])
    assert np.array_equal(mm[..., 1], large["vmax"])


def test_large_pdm_planes_in_full(large):
    """Every block of a sparse, a middling and a dense PDM plane, and of an empty one if
    the volume has one, against the oracle's chamfer transform of the oracle's POM."""
    rng = np.random.default_rng(2024)
    mask = large["mask"]
    K = large["w"]["K"]
    pd = large["eng"].pdm_planes()
    occupied = [p for p in range(K) if mask[..., p // 64].any()]
    counts = {p: int(oracle.mask_plane(mask, p).sum()) for p in occupied}
    by = sorted(counts, key=counts.get)
    planes = [by[0], by[len(by) // 4], by[len(by) // 2], by[-1]]
    empty = [p for p in range(K) if p not in counts]
    if empty:
        planes.append(empty[0])
    for p in planes:
        occ = oracle.mask_plane(mask, p)
        want = oracle.chamfer_dt(occ)
        got = pd[p].cpu().numpy()
        assert np.array_equal(got, want), p
        pts = _points(rng, occ.shape, 6)
        for (x, y, z), wv in zip(pts, oracle.dt_at_many(occ, pts)):
            assert got[z, y, x] == wv, (p, x, y, z)
    if empty:
        assert (pd[empty[0]] == 255).all()


def test_large_update_and_full_recompute_in_full(large):
    """D' (§3.1 step 1 + Eq. 1) and the min/max full recompute's D for four TFs, every
    block: three edits of the workload's sequence and a TF aligned with the partitions."""
    w = large["w"]
    eng = large["eng"]
    mask = large["mask"]
    tfs = T.tf_edit_sequence(w["seed"], w["N"], w["edits"])[::400] + \
        [T.aligned_tf(5, w["N"], T.uniform_borders(w["N"], w["K"]))]
    assert len(tfs) == 4
    for k, tf in enumerate(tfs):
        tfd = torch.from_numpy(tf).cuda()
        am = torch.zeros(1, dtype=torch.int64, device="cuda")
        dprime = eng.update_tf(tfd, active_mask=am).cpu().numpy().reshape(mask.shape[:3])
        S = oracle.active_set(tf, w["K"])
        got_S = int(am.cpu().numpy().view(np.uint64)[0])
        assert [p for p in range(w["K"]) if (got_S >> p) & 1] == S, k
        want = oracle.chamfer_dt(oracle.union_plane(mask, S))
        assert np.array_equal(dprime, want), ("D'", k)
        full = eng.full_recompute(tfd).cpu().numpy().reshape(mask.shape[:3])
        want_f = oracle.chamfer_dt(oracle.occ_minmax(large["vmin"], large["vmax"], tf))
        assert np.array_equal(full, want_f), ("D", k)
