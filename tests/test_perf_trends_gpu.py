"""Performance sanity checks with the trends that Table 1 reports, on the 512^3 12-bit
workload: the update takes longer the more partitions a TF makes active, the one-time
precompute grows with the number of partitions, and an all-visible TF makes the plain
full recompute fast (every block occupied: the distance passes have nothing to do).
Timings are CUDA-event means with the L2 flushed before every call; the bounds are loose
so that only a broken trend fails."""
import numpy as np
import pytest
import torch

import synth
from synth import tfs as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ct():
    import __graft_entry__ as g
    g.build()
    vol = synth.make_volume("ct", device="cuda")
    return vol


def _flush(buf):
    buf[0].zero_()
    buf[1].max()


def _mean_ms(fn, flush, reps=20):
    s = torch.cuda.current_stream()
    ts = []
    for _ in range(reps + 3):
        _flush(flush)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.mean(ts[3:]))


def _first_partitions_tf(N, K, m):
    """Alpha 0.5 on the intensities of partitions 0..m-1 (uniform borders), 0 elsewhere."""
    tf = np.zeros((N, 4), np.float32)
    tf[: (m * N) // K, 3] = 0.5
    return tf


def test_update_time_grows_with_active_partitions(ct):
    from paper_2407_21552_gb300 import DM_U16
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    flush = (torch.empty(256 << 20, dtype=torch.uint8, device="cuda"),
             torch.zeros(32 << 20, dtype=torch.int64, device="cuda"))
    eng = PartitionedDistanceMaps((512, 512, 512), DM_U16, 4, 1, 32, 4096)
    eng.build_partitions(ct)
    out = torch.empty(eng.G, dtype=torch.uint8, device="cuda")
    t = {}
    for m in (1, 8, 32):
        tf = torch.from_numpy(_first_partitions_tf(4096, 32, m)).cuda()
        t[m] = _mean_ms(lambda: eng.update_tf(tf, out=out), flush)
    assert t[32] > 1.3 * t[1], t
    assert t[32] > t[8] > 0.9 * t[1], t
    # an all-visible TF: every block occupied, the full recompute is fast (Table 1, TF2)
    tf_all = torch.from_numpy(T.all_visible_tf(4096)).cuda()
    sparse = np.zeros((4096, 4), np.float32)
    sparse[2000:2200, 3] = 0.5                  # a narrow bone band: scattered occupancy
    tf_sparse = torch.from_numpy(sparse).cuda()
    t_all = _mean_ms(lambda: eng.full_recompute(tf_all, out=out), flush)
    t_sparse = _mean_ms(lambda: eng.full_recompute(tf_sparse, out=out), flush)
    assert t_all < t_sparse, (t_all, t_sparse)
    eng.close()


def test_precompute_grows_with_partitions(ct):
    from paper_2407_21552_gb300 import DM_U16
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    flush = (torch.empty(256 << 20, dtype=torch.uint8, device="cuda"),
             torch.zeros(32 << 20, dtype=torch.int64, device="cuda"))
    t = {}
    for K in (4, 64):
        eng = PartitionedDistanceMaps((512, 512, 512), DM_U16, 4, 1, K, 4096)
        t[K] = _mean_ms(lambda: eng.build_partitions(ct), flush, reps=5)
        eng.close()
    assert t[64] > 1.3 * t[4], t
