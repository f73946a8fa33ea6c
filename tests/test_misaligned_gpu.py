"""Output buffers that are not 16-byte aligned take the byte-wise paths of the update, the
full recompute and the batched update; results still equal the oracle's.  Also: the
profiling events that dm_set_profile_events installs bracket exactly the update kernel."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from synth import tfs as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__ as g
    g.build()
    from paper_2407_21552_gb300 import DM_U16
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    vol = synth.volume_of("u16", (72, 40, 36), 21)           # grid 18 x 10 x 9
    vnp = synth.as_numpy(vol)
    eng = PartitionedDistanceMaps((72, 40, 36), DM_U16, 4, 1, 24, 4096)
    eng.build_partitions(vol.cuda())
    ref = oracle.build_partitions(vnp, 4, 1, 4096, 24)
    return eng, vnp, ref


def _misaligned(G, shift):
    buf = torch.empty(G + 64, dtype=torch.uint8, device="cuda")
    return buf[shift:shift + G]


@pytest.mark.parametrize("shift", [1, 3, 8])
def test_update_and_full_recompute_into_misaligned_outputs(setup, shift):
    eng, vnp, (mask, pdm, vmin, vmax) = setup
    tfs = T.tf_edit_sequence(30 + shift, 4096, 5) + [T.zero_tf(4096), T.all_visible_tf(4096)]
    for tf in tfs:
        tfd = torch.from_numpy(tf).cuda()
        out = _misaligned(eng.G, shift)
        assert out.data_ptr() % 16 != 0
        eng.update_tf(tfd, out=out)
        want, _ = oracle.update_tf(pdm, tf)
        assert np.array_equal(out.cpu().numpy().reshape(want.shape), want)
        full = _misaligned(eng.G, shift)
        eng.full_recompute(tfd, out=full)
        assert np.array_equal(full.cpu().numpy().reshape(want.shape),
                              oracle.full_recompute_minmax(vmin, vmax, tf))


def test_batch_with_misaligned_items(setup):
    from paper_2407_21552_gb300 import _abi as A
    eng, vnp, (mask, pdm, vmin, vmax) = setup
    tfs = T.tf_edit_sequence(77, 4096, 3)
    tfd = [torch.from_numpy(tf).cuda() for tf in tfs]
    # the same context may appear once per launch: three launches, aligned / not
    for k, shift in enumerate([0, 5, 13]):
        out = _misaligned(eng.G, shift)
        A.dm_update_tf_batch([(eng.ctx, tfd[k].data_ptr(), out.data_ptr())], None,
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        want, _ = oracle.update_tf(pdm, tfs[k])
        assert np.array_equal(out.cpu().numpy().reshape(want.shape), want)


def test_profile_events_bracket_the_update(setup):
    from paper_2407_21552_gb300 import dm_set_profile_events
    eng, vnp, (mask, pdm, vmin, vmax) = setup
    tf = torch.from_numpy(T.tf_edit_sequence(5, 4096, 1)[0]).cuda()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    b.record()                      # torch creates the events on their first record
    torch.cuda.synchronize()
    dm_set_profile_events(eng.ctx, a.cuda_event, b.cuda_event)
    out = eng.update_tf(tf)
    dm_set_profile_events(eng.ctx, None, None)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    assert 0.0 < ms < 50.0
    want, _ = oracle.update_tf(pdm, tf.cpu().numpy())
    assert np.array_equal(out.cpu().numpy().reshape(want.shape), want)
