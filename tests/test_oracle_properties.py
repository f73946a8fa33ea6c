"""Property tests of the oracle on random tiny inputs (hypothesis): random dims that are not
multiples of b, random b, apron, N, K, volumes and TFs.  For every draw, the update is the
distance transform of the union of the active POMs (Eq. 1), never exceeds the exact map
D (§3.1), equals it when the TF is aligned with the partitions, and the distance
transform matches scipy's chessboard transform."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
import scipy.ndimage as ndi  # noqa: E402


def _cdt(occ):
    occ = occ != 0
    if not occ.any():
        return np.full(occ.shape, 255, np.uint8)
    return np.minimum(ndi.distance_transform_cdt(~occ, metric="chessboard"), 255).astype(np.uint8)


@st.composite
def cases(draw):
    dims = tuple(draw(st.integers(1, 11)) for _ in range(3))
    b = draw(st.integers(1, 4))
    a = draw(st.integers(0, b))
    N = draw(st.sampled_from([8, 16, 40, 256]))
    K = draw(st.integers(1, min(N, 12)))
    seed = draw(st.integers(0, 2**31 - 1))
    rng = np.random.default_rng(seed)
    vol = rng.integers(0, N + 3, size=(dims[2], dims[1], dims[0])).astype(np.uint8 if N <= 253 else np.uint16)
    alpha = np.where(rng.uniform(size=N) < draw(st.floats(0.0, 1.0)), rng.uniform(0.01, 1, size=N), 0)
    tf = np.zeros((N, 4), np.float32)
    tf[:, 3] = alpha
    return vol, b, a, N, K, tf


@settings(max_examples=60, deadline=None)
@given(cases())
def test_update_properties(case):
    vol, b, a, N, K, tf = case
    mask, pdm, vmin, vmax = oracle.build_partitions(vol, b, a, N, K)
    dprime, _ = oracle.update_tf(pdm, tf)
    S = oracle.active_set(tf, K)
    assert np.array_equal(dprime, _cdt(oracle.union_plane(mask, S)))
    d = oracle.full_recompute_exact(vol, b, a, tf)
    assert np.all(dprime <= d)
    assert np.all(oracle.full_recompute_minmax(vmin, vmax, tf) <= d)
    # the same TF made aligned: every partition that has a visible intensity made fully
    # visible, so no partition is mixed and D' equals D
    lut = oracle.partition_lut(N, K)
    tfa = tf.copy()
    tfa[:, 3] = np.where(np.isin(lut, S), 0.5, 0.0)
    da, _ = oracle.update_tf(pdm, tfa)
    assert np.array_equal(da, oracle.full_recompute_exact(vol, b, a, tfa))
    assert np.array_equal(da, dprime)                 # same S, same D'


@settings(max_examples=80, deadline=None)
@given(st.tuples(st.integers(1, 13), st.integers(1, 13), st.integers(1, 13)),
       st.floats(0.0, 1.0), st.integers(0, 2**31 - 1))
def test_chamfer_is_the_chessboard_transform(shape, density, seed):
    occ = (np.random.default_rng(seed).uniform(size=shape) < density).astype(np.uint8)
    assert np.array_equal(oracle.chamfer_dt(occ), _cdt(occ))
