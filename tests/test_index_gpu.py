"""The optional partition-range index (dm_config.index_mode = DM_INDEX_RANGES): the update
reads two index planes per run of consecutive active partitions instead of one plane per
active partition, and must give the same D' -- the oracle's -- bit for bit, on the fused
path (N <= 8192), the two-kernel path (N > 8192) and the batched path."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from synth import tfs as T

pytestmark = pytest.mark.gpu


def _pair(vol_np, b, a, N, K):
    import __graft_entry__ as g
    g.build()
    from paper_2407_21552_gb300 import DM_U8, DM_U16, DM_INDEX_RANGES
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    Z, Y, X = vol_np.shape
    dt = DM_U8 if vol_np.dtype == np.uint8 else DM_U16
    vd = torch.from_numpy(vol_np if dt == DM_U8 else vol_np.view(np.int16)).cuda()
    plain = PartitionedDistanceMaps((X, Y, Z), dt, b, a, K, N)
    idx = PartitionedDistanceMaps((X, Y, Z), dt, b, a, K, N, index_mode=DM_INDEX_RANGES)
    plain.build_partitions(vd)
    idx.build_partitions(vd)
    return plain, idx


def _tfs(N, K, seed):
    bd = T.uniform_borders(N, K)
    out = T.tf_edit_sequence(seed, N, 8) + T.special_tfs(N, bd)
    alt = T.zero_tf(N)                       # every other partition visible: many runs
    for p in range(0, K, 2):
        alt[bd[p]:bd[p + 1], 3] = 0.5
    out.append(alt)
    return out


@pytest.mark.parametrize("shape,b,a,N,K,dt", [
    ((40, 36, 44), 4, 1, 256, 16, np.uint8),
    ((33, 29, 37), 4, 1, 4096, 32, np.uint16),
    ((20, 24, 28), 2, 1, 300, 7, np.uint16),
    ((16, 20, 64), 4, 1, 4096, 256, np.uint16),
    ((30, 30, 30), 3, 2, 65536, 64, np.uint16),      # N > 8192: two-kernel path
])
def test_index_matches_oracle(shape, b, a, N, K, dt):
    rng = np.random.default_rng(K + N)
    v = rng.integers(0, N, size=tuple(max(1, s // 3) for s in shape))
    v = np.kron(v, np.ones((3, 3, 3), np.int64))
    v = np.pad(v, [(0, max(0, s - v.shape[i])) for i, s in enumerate(shape)], mode="edge")
    vol = v[: shape[0], : shape[1], : shape[2]].astype(dt)
    plain, idx = _pair(vol, b, a, N, K)
    _, pdm_o, _, _ = oracle.build_partitions(vol, b, a, N, K)
    for tf in _tfs(N, K, 5):
        tfd = torch.from_numpy(tf).cuda()
        got = idx.update_tf(tfd)
        want, _ = oracle.update_tf(pdm_o, tf)
        assert np.array_equal(got.cpu().numpy().reshape(want.shape), want)
        assert torch.equal(got, plain.update_tf(tfd))


def test_index_in_batch_and_levels_are_range_minima():
    from paper_2407_21552_gb300 import _abi as A
    vol = synth.as_numpy(synth.tiny_volume(0, size=64))
    plain, idx = _pair(vol, 4, 1, 256, 16)
    # level planes are minima of consecutive PDMs
    K, G, st = 16, idx.G, idx.plane_stride
    raw = idx._pdm[: idx.sizes.pdm_planes * st].view(-1, st)[:, :G].cpu().numpy()
    base, k = 0, 0
    while (1 << k) <= K:
        for i in range(K - (1 << k) + 1):
            assert np.array_equal(raw[base + i], raw[i:i + (1 << k)].min(axis=0)), (k, i)
        base += K - (1 << k) + 1
        k += 1
    tfs = [torch.from_numpy(t).cuda() for t in T.tf_edit_sequence(9, 256, 2)]
    outs = [torch.empty(G, dtype=torch.uint8, device="cuda") for _ in range(2)]
    A.dm_update_tf_batch([(idx.ctx, tfs[0].data_ptr(), outs[0].data_ptr()),
                          (plain.ctx, tfs[1].data_ptr(), outs[1].data_ptr())], None,
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert torch.equal(outs[0], plain.update_tf(tfs[0]))
    assert torch.equal(outs[1], plain.update_tf(tfs[1]))
