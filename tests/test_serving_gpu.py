"""Serving loop on the GPU: edits from several sessions arrive while earlier batches are
still running, are batched (one edit per session per batch) on three streams, and every
result equals the same update computed alone -- for the partitioned server and for the
full-recompute server."""
import numpy as np
import pytest
import torch

import synth
from synth import tfs as T

pytestmark = pytest.mark.gpu


def _sessions(count=6, seed=21):
    import __graft_entry__ as g
    g.build()
    from paper_2407_21552_gb300 import DM_U8, DM_U16
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    out = []
    for sp in synth.batch_specs(seed=seed, count=count, lo=24, hi=96):
        X, Y, Z = sp["dims"]
        eng = PartitionedDistanceMaps((X, Y, Z), DM_U8 if sp["kind"] == "u8" else DM_U16, 4, 1,
                                      sp["K"], sp["N"])
        eng.build_partitions(synth.volume_of(sp["kind"], sp["dims"], sp["seed"]).cuda())
        out.append((sp, eng))
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("mode", ["partitioned", "full"])
def test_each_result_is_the_same_alone_and_in_the_mix(mode):
    from paper_2407_21552_gb300.serving import DeviceExecutor, Scheduler, SessionSpec
    sess = _sessions()
    ex = DeviceExecutor(slots=3, mode=mode)
    ex.keep_results = True
    sch = Scheduler(ex, budget_bytes=1 << 40, slots=3, max_batch=4)
    for sid, (sp, eng) in enumerate(sess):
        sch.open_session(SessionSpec(sid, eng.sizes.pdm_bytes, dict(engine=eng)))
    rng = np.random.default_rng(3)
    reqs = []
    for k in range(90):
        sid = int(rng.integers(0, len(sess)))
        tf = torch.from_numpy(T.tf_edit_sequence(100 + k, sess[sid][0]["N"], 1)[0]).pin_memory()
        reqs.append(sch.submit(sid, tf))
        if k % 3 == 0:
            sch.poll()                 # launches while earlier batches still run
    sch.drain()
    assert len(sch.completed) == len(reqs)
    assert max(sch.stats.batch_sizes) > 1 and sch.stats.batches < len(reqs)
    for r in sch.completed:
        eng = sess[r.session][1]
        tfd = r.tf.cuda()
        alone = eng.update_tf(tfd) if mode == "partitioned" else eng.full_recompute(tfd)
        assert torch.equal(ex.results[r.rid], alone), r.rid
