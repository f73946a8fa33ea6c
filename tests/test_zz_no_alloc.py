"""dm_update_tf_noalloc: the TF update for callers that may not allocate device memory
(plug-ins handed their buffers by a host renderer, render loops that must not allocate
between frames).  It keeps its working memory in a fixed array inside the library instead
of a caller-bound scratch buffer, so its results must be those of dm_update_tf, bit for
bit, also when one call follows another and the array still holds the earlier call's
contents.  Collected last so that a failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2407_21552_gb300 import _abi as A
    return A


def _engine(vol, K, N, borders=None):
    from paper_2407_21552_gb300 import DM_U8, DM_U16
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    Z, Y, X = vol.shape
    dt = DM_U8 if vol.dtype == torch.uint8 else DM_U16
    eng = PartitionedDistanceMaps((X, Y, Z), dt, 4, 1, K, N, borders=borders)
    eng.build_partitions(vol.cuda())
    return eng


def _run_both(A, eng, tf_np, borders=None):
    tf = torch.from_numpy(tf_np).cuda()
    want = eng.update_tf(tf)
    got = torch.full((eng.G,), 7, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    A.dm_update_tf_noalloc(eng._pdm.data_ptr(), eng.plane_stride, eng.G, eng.K, borders, eng.N,
                           tf.data_ptr(), got.data_ptr(), stream)
    torch.cuda.synchronize()
    return want.cpu().numpy(), got.cpu().numpy()


def test_noalloc_matches_bound_scratch_update_two_calls_in_a_row(lib):
    import synth
    from synth import tfs as T
    vol = synth.tiny_volume(0, size=96)
    eng = _engine(vol, 16, 256)
    # many partitions active first, then few: stale list entries would show in call two
    calls = [T.all_visible_tf(256), T.single_intensity_tf(256, 150)]
    calls += T.tf_edit_sequence(11, 256, 2)
    for tf in calls:
        want, got = _run_both(lib, eng, tf)
        assert np.array_equal(got, want)
    eng.close()


def test_noalloc_12bit_explicit_borders(lib):
    import synth
    from synth import tfs as T
    vol = synth.ct_volume(1, size=96)
    borders = [0, 1] + [int(v) for v in np.linspace(64, 4096, 40).astype(int)[1:]]
    K = len(borders) - 1
    eng = _engine(vol, K, 4096, borders)
    for tf in T.tf_edit_sequence(12, 4096, 2):
        want, got = _run_both(lib, eng, tf, borders)
        assert np.array_equal(got, want)
    eng.close()


def test_noalloc_rejects_sizes_beyond_its_fixed_array(lib):
    A = lib
    raw = A.load()
    fake = ctypes.c_void_p(1 << 20)   # refused on the host before anything is enqueued
    big = A.DM_NOALLOC_MAX_TF_SIZE + 1
    assert raw.dm_update_tf_noalloc(fake, 64, 64, 16, None, big, fake, fake, None) == \
        A.DM_ERR_UNSUPPORTED
    assert raw.dm_update_tf_noalloc(fake, 64, 64, 257, None, 4096, fake, fake, None) == \
        A.DM_ERR_UNSUPPORTED
    assert raw.dm_update_tf_noalloc(fake, 32, 64, 16, None, 256, fake, fake, None) == \
        A.DM_ERR_INVALID_ARG
    assert raw.dm_update_tf_noalloc(None, 64, 64, 16, None, 256, fake, fake, None) == \
        A.DM_ERR_INVALID_ARG
