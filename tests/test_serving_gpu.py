"""Serving loop on the GPU: edits from several sessions arrive while earlier batches are
still running, are batched (one edit per session per batch) on three streams, and every
result equals the oracle's map for that edit (Eq. 1 over the oracle's PDMs for the
partitioned server, the min/max full recompute for the other) and the same update computed
alone -- also when idle sessions are evicted to host memory and readmitted."""
import numpy as np
import pytest
import torch

import oracle
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
        vol = synth.volume_of(sp["kind"], sp["dims"], sp["seed"])
        eng.build_partitions(vol.cuda())
        _, pdm_o, vmin_o, vmax_o = oracle.build_partitions(synth.as_numpy(vol), 4, 1, sp["N"],
                                                           sp["K"])
        sp = dict(sp, pdm=pdm_o, vmin=vmin_o, vmax=vmax_o)
        out.append((sp, eng))
    torch.cuda.synchronize()
    return out


def _oracle_map(sp, tf, mode):
    """The oracle's result for one edit of a session, flattened like the device map."""
    if mode == "partitioned":
        return oracle.update_tf(sp["pdm"], tf)[0].reshape(-1)
    return oracle.full_recompute_minmax(sp["vmin"], sp["vmax"], tf).reshape(-1)


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
        sp, eng = sess[r.session]
        tfd = r.tf.cuda()
        alone = eng.update_tf(tfd) if mode == "partitioned" else eng.full_recompute(tfd)
        assert torch.equal(ex.results[r.rid], alone), r.rid
        want = _oracle_map(sp, r.tf.numpy(), mode)
        assert np.array_equal(ex.results[r.rid].cpu().numpy(), want), r.rid


@pytest.mark.parametrize("mode", ["partitioned", "full"])
def test_eviction_and_readmission_keep_every_result(mode):
    """A budget that holds the largest session but not all of them, with eviction: idle
    sessions' maps move to host memory and come back for their next edit, many times over;
    every result still equals the same update computed before the loop, with all maps
    resident."""
    from paper_2407_21552_gb300.serving import DeviceExecutor, Scheduler, SessionSpec
    sess = _sessions(count=6, seed=23)
    rng = np.random.default_rng(4)
    plan = []
    for k in range(60):
        sid = int(rng.integers(0, len(sess)))
        tf = torch.from_numpy(T.tf_edit_sequence(300 + k, sess[sid][0]["N"], 1)[0]).pin_memory()
        eng = sess[sid][1]
        tfd = tf.cuda()
        want = eng.update_tf(tfd) if mode == "partitioned" else eng.full_recompute(tfd)
        plan.append((sid, tf, want.clone()))
    torch.cuda.synchronize()
    sizes = [eng.sizes.pdm_bytes + eng.sizes.minmax_bytes for _, eng in sess]
    ex = DeviceExecutor(slots=3, mode=mode)
    ex.keep_results = True
    budget = max(max(sizes), sum(sizes) // 2)            # the largest fits, not all
    assert budget < sum(sizes)
    sch = Scheduler(ex, budget_bytes=budget, slots=3, max_batch=4, evict_idle=True)
    for sid, (sp, eng) in enumerate(sess):
        sch.open_session(SessionSpec(sid, sizes[sid], dict(engine=eng)))
    reqs = []
    for k, (sid, tf, _) in enumerate(plan):
        reqs.append(sch.submit(sid, tf))
        if k % 2 == 0:
            sch.poll()
    sch.drain()
    assert len(sch.completed) == len(reqs)
    assert sch.stats.evictions > 0 and sch.stats.readmissions > 0
    assert sch.used <= sch.budget
    for r, (sid, tf, want) in zip(reqs, plan):
        assert torch.equal(ex.results[r.rid], want), r.rid
        ref = _oracle_map(sess[sid][0], tf.numpy(), mode)
        assert np.array_equal(ex.results[r.rid].cpu().numpy(), ref), r.rid
    # an evicted engine holds no device maps and refuses updates until reloaded
    off = [eng for _, eng in sess if eng.offloaded]
    assert off
    from paper_2407_21552_gb300 import _abi as A
    with pytest.raises(A.DmError):
        off[0].update_tf(torch.zeros((off[0].N, 4), device="cuda"))
    off[0].reload()
    assert not off[0].offloaded


def test_offload_copies_the_maps_again_after_a_rebuild():
    """The host copy is reused while the maps are unchanged and refreshed after a rebuild:
    offload, reload, rebuild from another volume, offload, reload; the update then equals
    a fresh engine's built from that other volume."""
    import __graft_entry__ as g
    g.build()
    from paper_2407_21552_gb300 import DM_U8
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    dims = (40, 33, 27)
    v1 = synth.volume_of("u8", dims, 11).cuda()
    v2 = synth.volume_of("u8", dims, 12).cuda()
    eng = PartitionedDistanceMaps(dims, DM_U8, 4, 1, 16, 256)
    ref = PartitionedDistanceMaps(dims, DM_U8, 4, 1, 16, 256)
    eng.build_partitions(v1)
    ref.build_partitions(v2)
    tf = torch.from_numpy(T.tf_edit_sequence(9, 256, 1)[0]).cuda()
    want1 = eng.update_tf(tf).clone()
    for _ in range(2):                                   # the second offload copies nothing
        eng.offload()
        eng.reload()
        assert torch.equal(eng.update_tf(tf), want1)
    eng.build_partitions(v2)
    eng.offload()
    eng.reload()
    assert torch.equal(eng.update_tf(tf), ref.update_tf(tf))
    assert not torch.equal(want1, ref.update_tf(tf))
