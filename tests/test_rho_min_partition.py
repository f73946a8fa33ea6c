"""A separate partition for the volume's minimum intensity rho_min (§3.1, §4.2).

With uniform partitions, a TF that hides rho_min but shows other intensities of the first
partition makes that partition "mixed": D' < D wherever rho_min voxels are, and empty
space that D would skip is no longer skipped (the 32-partition case of §4.2).  Giving
rho_min its own partition makes every partition uniformly visible or invisible for such
TFs, so D' == D.  Checked with the oracle on the CPU and through libdm on the GPU.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2407_21552_gb300.partitions import rho_min_borders, uniform_borders
from synth import tfs as T


def _volume():
    """Mostly rho_min = 0 background with objects at 3..12 and 120..200 (uint8)."""
    rng = np.random.default_rng(31)
    v = np.zeros((40, 48, 56), np.uint8)
    for _ in range(12):
        z, y, x = rng.integers(0, [36, 44, 52])
        v[z:z + 4, y:y + 4, x:x + 4] = rng.integers(3, 13)
    for _ in range(6):
        z, y, x = rng.integers(0, [34, 42, 50])
        v[z:z + 6, y:y + 6, x:x + 6] = rng.integers(120, 201)
    return v


def _tf_hiding_rho_min(N):
    tf = T.zero_tf(N)
    tf[1:16, 3] = 0.6      # the rest of uniform partition 0 is visible ...
    tf[100:, 3] = 0.3      # ... and every intensity of the bright objects
    return tf              # alpha(rho_min = 0) stays 0


def test_borders_helpers():
    assert list(uniform_borders(256, 4)) == [0, 64, 128, 192, 256]
    b = rho_min_borders(256, 4, 0)
    assert list(b) == [0, 1, 86, 171, 256]
    assert list(rho_min_borders(4096, 3, 10)) == [0, 11, 2053, 4096]
    with pytest.raises(ValueError):
        rho_min_borders(256, 1, 0)
    with pytest.raises(ValueError):
        rho_min_borders(8, 8, 4)


def test_rho_min_partition_removes_mixed_partition_gap_oracle():
    N, K, b, a = 256, 16, 4, 1
    vol = _volume()
    tf = _tf_hiding_rho_min(N)
    d = oracle.full_recompute_exact(vol, b, a, tf)
    _, pdm_u, _, _ = oracle.build_partitions(vol, b, a, N, K)
    d_u, _ = oracle.update_tf(pdm_u, tf)
    assert np.all(d_u <= d) and np.any(d_u < d)          # uniform: mixed partition 0
    br = rho_min_borders(N, K, int(vol.min()))
    _, pdm_r, _, _ = oracle.build_partitions(vol, b, a, N, K, br)
    d_r, _ = oracle.update_tf(pdm_r, tf, br)
    assert np.array_equal(d_r, d)                         # rho_min partition: exact


@pytest.mark.gpu
def test_rho_min_partition_gpu_matches_oracle():
    import __graft_entry__ as g
    g.build()
    from paper_2407_21552_gb300 import DM_U8
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    N, K, b, a = 256, 16, 4, 1
    vol = _volume()
    tf = _tf_hiding_rho_min(N)
    br = rho_min_borders(N, K, int(vol.min()))
    Z, Y, X = vol.shape
    eng = PartitionedDistanceMaps((X, Y, Z), DM_U8, b, a, K, N, borders=br)
    eng.build_partitions(torch.from_numpy(vol).cuda())
    got = eng.update_tf(torch.from_numpy(tf).cuda()).cpu().numpy().reshape(
        eng.grid[2], eng.grid[1], eng.grid[0])
    assert np.array_equal(got, oracle.full_recompute_exact(vol, b, a, tf))
    eng.close()
