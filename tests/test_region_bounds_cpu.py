"""The identity behind the region bounds taken from the masks' rows (no GPU).

Where a region of the combine is whole rows of blocks (4096 a multiple of gx), the minimum
of a partition's distance map over the region equals the minimum, over the region's rows
(y, z), of D2: the 2D chessboard distance transform of the partition's occupancy ORed along
x.  (A block of a row can sit straight above the nearest occupied block in x, so x adds
nothing to the distance; clamping at 255 commutes with the minimum.)  The library builds
D2 with its x pass and line pass over the rows and reduces it per region; this test checks
the identity itself with the oracle's maps, including grids whose last region is partial,
and the 2D step against scipy's chessboard transform.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
import synth

REGION = 4096


def _cdt2(occ):
    occ = occ != 0
    if not occ.any():
        return np.full(occ.shape, 255, np.uint8)
    d = ndi.distance_transform_cdt(~occ, metric="chessboard")
    return np.minimum(d, 255).astype(np.uint8)


@pytest.mark.parametrize("dims,b,K", [((128, 128, 128), 4, 16),    # gx 32, 8 regions
                                      ((256, 96, 40), 4, 8),       # gx 64, partial last
                                      ((128, 64, 200), 2, 16),     # gx 64, 50 regions
                                      ((64, 16, 40), 1, 12)])      # gx 64, b = 1
def test_region_minimum_from_projected_rows(dims, b, K):
    N = 256
    vol = synth.as_numpy(synth.volume_of("u8", dims, 21))
    mask, pdm, _, _ = oracle.build_partitions(vol, b, 1 if b > 1 else 0, N, K)
    gz, gy, gx = pdm.shape[1:]
    assert REGION % gx == 0
    G = gx * gy * gz
    nreg = -(-G // REGION)
    rows_per_region = REGION // gx
    flat = pdm.reshape(K, -1)
    for p in range(K):
        want = np.array([flat[p, r * REGION:(r + 1) * REGION].min() for r in range(nreg)])
        occ = oracle.mask_plane(mask, p).reshape(gz, gy, gx)
        proj = occ.any(axis=2)                                 # [gz][gy]: OR along x
        d2 = _cdt2(proj)
        assert np.array_equal(d2, oracle.chamfer_dt(proj.reshape(gz, gy, 1))[:, :, 0])
        rows = d2.reshape(-1)                                  # row index z * gy + y
        got = np.array([rows[r * rows_per_region:(r + 1) * rows_per_region].min()
                        for r in range(nreg)])
        assert np.array_equal(got, want), (p, got[:6], want[:6])
