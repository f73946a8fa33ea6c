"""dm_update_tf_noalloc: the TF update for callers that may not allocate device memory
(plug-ins handed their buffers by a host renderer, render loops that must not allocate
between frames).  It keeps its working memory in a fixed array inside the library instead
of a caller-bound scratch buffer, so its results must be the oracle's D' (Eq. 1 over the
oracle's own maps) and those of dm_update_tf, bit for bit, also when one call follows
another and the array still holds the earlier call's contents.  The cases reach the top of
the array: TF sizes up to its limit of 16384 entries (visibility words up to byte 3072)
and K = 256 (all eight ballot words of the active list).  Collected last so that a
failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest
import torch

import oracle

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


def _oracle_maps(vol, K, N, borders=None):
    import synth
    return oracle.build_partitions(synth.as_numpy(vol), 4, 1, N, K, borders)[1]


def _run_both(A, eng, tf_np, borders=None):
    tf = torch.from_numpy(tf_np).cuda()
    want = eng.update_tf(tf)
    got = torch.full((eng.G,), 7, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    A.dm_update_tf_noalloc(eng._pdm.data_ptr(), eng.plane_stride, eng.G, eng.K, borders, eng.N,
                           tf.data_ptr(), got.data_ptr(), stream)
    torch.cuda.synchronize()
    return want.cpu().numpy(), got.cpu().numpy()


def _check_calls(A, eng, pdm_o, tfs, borders=None):
    """Every call in a row: the oracle's D' == the no-allocation call == dm_update_tf."""
    for k, tf in enumerate(tfs):
        want, got = _run_both(A, eng, tf, borders)
        ref, _ = oracle.update_tf(pdm_o, tf, borders)
        assert np.array_equal(got, ref.reshape(-1)), k
        assert np.array_equal(got, want), k


def test_noalloc_matches_oracle_and_bound_scratch_update_two_calls_in_a_row(lib):
    import synth
    from synth import tfs as T
    vol = synth.tiny_volume(0, size=96)
    eng = _engine(vol, 16, 256)
    pdm_o = _oracle_maps(vol, 16, 256)
    # many partitions active first, then few: stale list entries would show in call two
    calls = [T.all_visible_tf(256), T.single_intensity_tf(256, 150)]
    calls += T.tf_edit_sequence(11, 256, 2)
    _check_calls(lib, eng, pdm_o, calls)
    eng.close()


def test_noalloc_12bit_explicit_borders(lib):
    import synth
    from synth import tfs as T
    vol = synth.ct_volume(1, size=96)
    borders = [0, 1] + [int(v) for v in np.linspace(64, 4096, 40).astype(int)[1:]]
    K = len(borders) - 1
    eng = _engine(vol, K, 4096, borders)
    pdm_o = _oracle_maps(vol, K, 4096, borders)
    _check_calls(lib, eng, pdm_o, T.tf_edit_sequence(12, 4096, 2), borders)
    eng.close()


def _wide_volume(N, seed=31):
    """A 16-bit volume whose intensities span [0, N): the 12-bit CT-like recipe scaled."""
    import synth
    v = synth.volume_of("u16", (72, 56, 44), seed).to(torch.int32) * (N // 4096)
    return v.clamp(0, N - 1).to(torch.int16)


def _wide_tfs(N, seed):
    from synth import tfs as T
    return T.tf_edit_sequence(seed, N, 2) + [T.all_visible_tf(N), T.zero_tf(N)]


@pytest.mark.parametrize("N,K", [(12288, 64), (16384, 256)])
def test_noalloc_large_tf_sizes_and_all_partition_words(lib, N, K):
    """N above the fused update's 8192 entries (the library's two-launch path) up to the
    array's limit, and K = 256: the visibility words reach the top of the array and all
    eight 32-partition ballot words of the active list are used.  An all-visible TF is
    followed directly by an all-zero one, whose D' must be 255 everywhere."""
    vol = _wide_volume(N)
    eng = _engine(vol, K, N)
    pdm_o = _oracle_maps(vol, K, N)
    _check_calls(lib, eng, pdm_o, _wide_tfs(N, 40 + K))
    _, got = _run_both(lib, eng, _wide_tfs(N, 0)[-1])
    assert (got == 255).all()
    eng.close()


def test_noalloc_uneven_borders_at_the_limit(lib):
    """K = 256 uneven explicit borders over N = 16384: narrow partitions at the low end,
    wide ones at the top."""
    N, K = 16384, 256
    rng = np.random.default_rng(77)
    inner = np.sort(rng.choice(np.arange(1, N), size=K - 1, replace=False) ** 2 // N)
    inner = np.unique(np.clip(inner, 1, N - 1))
    while len(inner) < K - 1:                      # squaring may merge a few borders
        extra = rng.choice(np.setdiff1d(np.arange(1, N), inner), size=K - 1 - len(inner),
                           replace=False)
        inner = np.unique(np.concatenate([inner, extra]))
    borders = [0] + [int(v) for v in inner] + [N]
    assert len(borders) == K + 1 and all(b < c for b, c in zip(borders, borders[1:]))
    vol = _wide_volume(N, seed=32)
    eng = _engine(vol, K, N, borders)
    pdm_o = _oracle_maps(vol, K, N, borders)
    _check_calls(lib, eng, pdm_o, _wide_tfs(N, 91), borders)
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
