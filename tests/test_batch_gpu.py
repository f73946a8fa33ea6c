"""Batched update over volumes of uneven size, voxel type, K and N (one launch pair per
<= 64 items): every item's D' equals the oracle's, and equals dm_update_tf alone on that
item; batches longer than one launch pair and repeated-context errors are covered."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from synth import tfs as T

pytestmark = pytest.mark.gpu


def _engines(specs):
    import __graft_entry__ as g
    g.build()
    from paper_2407_21552_gb300 import DM_U8, DM_U16
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    out = []
    for sp in specs:
        vol = synth.volume_of(sp["kind"], sp["dims"], sp["seed"])
        X, Y, Z = sp["dims"]
        eng = PartitionedDistanceMaps((X, Y, Z), DM_U8 if sp["kind"] == "u8" else DM_U16,
                                      sp.get("b", 4), 1, sp["K"], sp["N"],
                                      index_mode=sp.get("index", 0))
        eng.build_partitions(vol.cuda())
        out.append((sp, vol, eng))
    torch.cuda.synchronize()
    return out


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _small_specs(count, seed):
    sp = synth.batch_specs(seed=seed, count=count, lo=9, hi=70)
    for i, s in enumerate(sp):
        if i % 5 == 4:
            s["b"] = 3                 # grids that are not multiples of 16: byte paths
    return sp


def test_batch_matches_oracle_and_single_updates():
    from paper_2407_21552_gb300 import _abi as A
    items = _engines(_small_specs(12, 9))
    tfs, outs = [], []
    for i, (sp, vol, eng) in enumerate(items):
        tf = T.tf_edit_sequence(50 + i, sp["N"], 3)[-1]
        tfs.append(torch.from_numpy(tf).cuda())
        outs.append(torch.full((eng.G,), 3, dtype=torch.uint8, device="cuda"))
    A.dm_update_tf_batch([(eng.ctx, tfs[i].data_ptr(), outs[i].data_ptr())
                          for i, (_, _, eng) in enumerate(items)], None, _stream())
    torch.cuda.synchronize()
    for i, (sp, vol, eng) in enumerate(items):
        vnp = synth.as_numpy(vol)
        _, pdm_o, _, _ = oracle.build_partitions(vnp, sp.get("b", 4), 1, sp["N"], sp["K"])
        want, _ = oracle.update_tf(pdm_o, tfs[i].cpu().numpy())
        assert np.array_equal(outs[i].cpu().numpy().reshape(want.shape), want), i
        single = eng.update_tf(tfs[i])
        assert torch.equal(single, outs[i]), i


@pytest.fixture(scope="module")
def long_batch():
    """71 small items (more than one launch pair holds), their TFs and the oracle's D'."""
    items = _engines(_small_specs(71, 10))
    tfs, wants = [], []
    for i, (sp, vol, _) in enumerate(items):
        tf = T.tf_edit_sequence(7 + i, sp["N"], 1)[0]
        pdm_o = oracle.build_partitions(synth.as_numpy(vol), sp.get("b", 4), 1, sp["N"],
                                        sp["K"])[1]
        tfs.append(torch.from_numpy(tf).cuda())
        wants.append(oracle.update_tf(pdm_o, tf)[0].reshape(-1))
    return items, tfs, wants


@pytest.mark.parametrize("per_sm", [1, 2, 8, 12, 24])
def test_batch_longer_than_one_launch_and_tuning(long_batch, per_sm):
    """A batch split over two launch pairs (> DM_BATCH_MAX_ITEMS) under five combine grid
    sizes: every item's D' is the oracle's and that of its own single update."""
    from paper_2407_21552_gb300 import _abi as A
    items, tfs, wants = long_batch
    outs = [torch.full((eng.G,), 5, dtype=torch.uint8, device="cuda") for _, _, eng in items]
    A.dm_update_tf_batch([(eng.ctx, tfs[i].data_ptr(), outs[i].data_ptr())
                          for i, (_, _, eng) in enumerate(items)], per_sm, _stream())
    torch.cuda.synchronize()
    for i, (_, _, eng) in enumerate(items):
        assert np.array_equal(outs[i].cpu().numpy(), wants[i]), i
        assert torch.equal(eng.update_tf(tfs[i]), outs[i]), i


@pytest.mark.parametrize("index", [False, True])
def test_batch_special_tfs_and_shrinking_active_sets(index):
    """The degenerate TFs in one batch (empty S, one partition, every partition, unions of
    whole partitions, NaN and -0.0 alpha), three calls in a row on the same items: the first
    makes every partition active, so the later, shorter active lists sit over longer stale
    ones in the items' scratch.  Each D' equals the oracle's."""
    from paper_2407_21552_gb300 import _abi as A, DM_INDEX_RANGES
    specs = _small_specs(16, 12)
    for sp in specs:
        sp["index"] = DM_INDEX_RANGES if index else 0
    items = _engines(specs)
    oracle_maps = [oracle.build_partitions(synth.as_numpy(vol), sp.get("b", 4), 1, sp["N"],
                                           sp["K"])[1] for sp, vol, _ in items]
    outs = [torch.empty(eng.G, dtype=torch.uint8, device="cuda") for _, _, eng in items]
    for call in range(3):
        tfs = []
        for i, (sp, _, _) in enumerate(items):
            special = T.special_tfs(sp["N"], T.uniform_borders(sp["N"], sp["K"]))
            tf = T.all_visible_tf(sp["N"]) if call == 0 else special[(i + 5 * call) % len(special)]
            tfs.append(torch.from_numpy(tf).cuda())
        A.dm_update_tf_batch([(eng.ctx, tfs[i].data_ptr(), outs[i].data_ptr())
                              for i, (_, _, eng) in enumerate(items)], None, _stream())
        torch.cuda.synchronize()
        for i, (sp, _, eng) in enumerate(items):
            want, _ = oracle.update_tf(oracle_maps[i], tfs[i].cpu().numpy())
            got = outs[i].cpu().numpy().reshape(want.shape)
            assert np.array_equal(got, want), (call, i)


@pytest.fixture(scope="module")
def bench_batch():
    """The benchmark's batch: 64 volumes, sides U[64, 384], b = 4 as tuned, one edit each;
    the oracle's POM masks of every volume."""
    from paper_2407_21552_gb300 import DM_U8, DM_U16
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    import __graft_entry__ as g
    g.build()
    items = []
    for sp in synth.batch_specs():
        vol = synth.volume_of(sp["kind"], sp["dims"], sp["seed"], device="cuda")
        X, Y, Z = sp["dims"]
        eng = PartitionedDistanceMaps((X, Y, Z), DM_U8 if sp["kind"] == "u8" else DM_U16, 4,
                                      1, sp["K"], sp["N"], with_minmax=False)
        eng.build_partitions(vol)
        eng.release_mask()
        mask = oracle.pom(synth.as_numpy(vol), 4, 1, sp["N"], sp["K"])[0]
        del vol
        tf = T.tf_edit_sequence(sp["seed"], sp["N"], 3)[-1]
        items.append((sp, eng, mask, tf, torch.from_numpy(tf).cuda(),
                      torch.empty(eng.G, dtype=torch.uint8, device="cuda")))
    torch.cuda.synchronize()
    return items


@pytest.mark.parametrize("per_sm", [None, 12])
def test_batch_at_bench_size_sampled(bench_batch, per_sm):
    """The benchmark's batch launched as the benchmark launches it (library default: one
    4 KiB unit per combine CTA) and with two units per CTA.  For every item: S is the
    oracle's, D' is 0 exactly on the union of the oracle's POMs over S, D' equals the item's
    own single update, and sampled blocks carry the oracle's exact Chebyshev distance."""
    from paper_2407_21552_gb300 import _abi as A
    rng = np.random.default_rng(404)
    for *_, out in bench_batch:
        out.fill_(7)
    A.dm_update_tf_batch([(e.ctx, tfd.data_ptr(), out.data_ptr())
                          for _, e, _, _, tfd, out in bench_batch], per_sm, _stream())
    torch.cuda.synchronize()
    for i, (sp, eng, mask, tf, tfd, out) in enumerate(bench_batch):
        am = torch.zeros(1, dtype=torch.int64, device="cuda")
        single = eng.update_tf(tfd, active_mask=am)
        assert torch.equal(single, out), i
        S = oracle.active_set(tf, sp["K"])
        got_S = int(am.cpu().numpy().view(np.uint64)[0])
        assert [p for p in range(sp["K"]) if (got_S >> p) & 1] == S, i
        union = oracle.union_plane(mask, S)
        dprime = out.cpu().numpy().reshape(union.shape)
        assert np.array_equal(dprime == 0, union == 1), i
        gz, gy, gx = union.shape
        pts = np.concatenate([np.array([[0, 0, 0], [gx - 1, gy - 1, gz - 1]]),
                              np.stack([rng.integers(0, gx, 6), rng.integers(0, gy, 6),
                                        rng.integers(0, gz, 6)], 1)])
        for (x, y, z), wv in zip(pts, oracle.dt_at_many(union, pts)):
            assert dprime[z, y, x] == wv, (i, x, y, z)


def test_batch_rejects_repeated_context():
    from paper_2407_21552_gb300 import _abi as A
    items = _engines(_small_specs(2, 11))
    eng = items[0][2]
    tf = torch.from_numpy(T.zero_tf(items[0][0]["N"])).cuda()
    out = torch.empty(eng.G, dtype=torch.uint8, device="cuda")
    with pytest.raises(A.DmError):
        A.dm_update_tf_batch([(eng.ctx, tf.data_ptr(), out.data_ptr())] * 2, None, _stream())
