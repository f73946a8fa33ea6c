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


def _ws(A, n):
    nbytes = A.dm_batch_workspace_bytes(n)
    return torch.empty(nbytes, dtype=torch.uint8, device="cuda"), nbytes


def _oracle_pdms(items):
    return [oracle.build_partitions(synth.as_numpy(vol), sp.get("b", 4), 1, sp["N"], sp["K"])[1]
            for sp, vol, _ in items]


@pytest.mark.parametrize("tuning", [None, (12, 8), (2, 4)])
def test_batch_ws_several_edits_per_volume(tuning):
    """dm_update_tf_batch_ws with repeated contexts: 6 volumes (one with the range index,
    one of b = 3 so its rows take the byte paths) with 1, 2, 3, 5, 8 and 11 TF edits (11:
    two groups of one context), interleaved in the item list, one output misaligned.  Every
    output is the oracle's D' for its own TF and that of dm_update_tf alone."""
    from paper_2407_21552_gb300 import _abi as A, DM_INDEX_RANGES
    specs = _small_specs(6, 31)
    specs[2]["index"] = DM_INDEX_RANGES
    specs[4]["b"] = 3
    items = _engines(specs)
    pdms = _oracle_pdms(items)
    counts = [1, 2, 3, 5, 8, 11]
    order = [(v, k) for k in range(max(counts)) for v in range(6) if k < counts[v]]
    tfs, outs, want = [], [], []
    for j, (v, k) in enumerate(order):
        sp, _, eng = items[v]
        tf = T.tf_edit_sequence(900 + 13 * v + k, sp["N"], 2)[-1] if k % 4 else \
            T.special_tfs(sp["N"], T.uniform_borders(sp["N"], sp["K"]))[k % 16]
        tfs.append(torch.from_numpy(tf).cuda())
        off = 1 if j == 7 else 0                          # one misaligned output
        buf = torch.full((eng.G + 16,), 9, dtype=torch.uint8, device="cuda")
        outs.append(buf[off: off + eng.G])
        want.append(oracle.update_tf(pdms[v], tf)[0].reshape(-1))
    ws, nbytes = _ws(A, len(order))
    A.dm_update_tf_batch_ws([(items[v][2].ctx, tfs[j].data_ptr(), outs[j].data_ptr())
                             for j, (v, _) in enumerate(order)], tuning, ws.data_ptr(), nbytes,
                            _stream())
    torch.cuda.synchronize()
    for j, (v, k) in enumerate(order):
        assert np.array_equal(outs[j].cpu().numpy(), want[j]), (v, k)
        assert torch.equal(items[v][2].update_tf(tfs[j]), outs[j]), (v, k)


def test_batch_graph_replay_with_new_tfs():
    """Both batched calls captured once in a CUDA graph over fixed TF buffers, then replayed
    with new TFs copied in: every replay gives the oracle's D' for the TFs of that replay."""
    from paper_2407_21552_gb300 import _abi as A
    items = _engines(_small_specs(9, 41))
    pdms = _oracle_pdms(items)
    NMAX = max(sp["N"] for sp, _, _ in items)
    n = len(items)
    tf_fixed = torch.zeros((n + 3, NMAX, 4), dtype=torch.float32, device="cuda")
    outs = [torch.empty(eng.G, dtype=torch.uint8, device="cuda") for _, _, eng in items]
    outs_ws = [torch.empty(items[i if i < n else i - n][2].G, dtype=torch.uint8, device="cuda")
               for i in range(n + 3)]
    single = [(eng.ctx, tf_fixed[i].data_ptr(), outs[i].data_ptr())
              for i, (_, _, eng) in enumerate(items)]
    multi = single[:] + [(items[i][2].ctx, tf_fixed[n + i].data_ptr(), 0) for i in range(3)]
    multi = [(c, t, outs_ws[i].data_ptr()) for i, (c, t, _) in enumerate(multi)]
    ws, nbytes = _ws(A, len(multi))
    pb1, pb2 = A.PreparedBatch(single), A.PreparedBatch(multi)
    A.dm_update_tf_batch(pb1, None, _stream())           # warm-up outside the capture
    A.dm_update_tf_batch_ws(pb2, None, ws.data_ptr(), nbytes, _stream())
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        A.dm_update_tf_batch(pb1, None, st)
        A.dm_update_tf_batch_ws(pb2, None, ws.data_ptr(), nbytes, st)
    for rep in range(3):
        cur = []
        for i in range(n + 3):
            sp = items[i % n if i < n else i - n][0]
            tf = T.tf_edit_sequence(5000 + 97 * rep + i, sp["N"], 1)[0]
            tf_fixed[i].zero_()
            tf_fixed[i, : sp["N"]] = torch.from_numpy(tf).cuda()
            cur.append(tf)
        graph.replay()
        torch.cuda.synchronize()
        for i in range(n):
            want = oracle.update_tf(pdms[i], cur[i])[0].reshape(-1)
            assert np.array_equal(outs[i].cpu().numpy(), want), (rep, i)
        for i in range(n + 3):
            v = i if i < n else i - n
            want = oracle.update_tf(pdms[v], cur[i])[0].reshape(-1)
            assert np.array_equal(outs_ws[i].cpu().numpy(), want), (rep, "ws", i)


def test_batch_of_block_8_volumes():
    """b = 8 (the autotuner's coarser choice) in a batch, against the oracle at b = 8."""
    from paper_2407_21552_gb300 import _abi as A
    specs = synth.batch_specs(seed=45, count=10, lo=20, hi=120)
    for sp in specs:
        sp["b"] = 8
    items = _engines(specs)
    pdms = _oracle_pdms(items)
    tfs = [torch.from_numpy(T.tf_edit_sequence(60 + i, sp["N"], 2)[-1]).cuda()
           for i, (sp, _, _) in enumerate(items)]
    outs = [torch.empty(eng.G, dtype=torch.uint8, device="cuda") for _, _, eng in items]
    A.dm_update_tf_batch([(eng.ctx, tfs[i].data_ptr(), outs[i].data_ptr())
                          for i, (_, _, eng) in enumerate(items)], (8, 8), _stream())
    torch.cuda.synchronize()
    for i in range(len(items)):
        want = oracle.update_tf(pdms[i], tfs[i].cpu().numpy())[0].reshape(-1)
        assert np.array_equal(outs[i].cpu().numpy(), want), i


def test_autotuner_search_and_choice():
    """The autotuner times every (block, CTAs per SM, loads per stage) of its search
    space, stops at the first block size whose best schedule meets the target (b = 4 for a
    target nothing misses), otherwise keeps the fastest schedule of all block sizes; the
    chosen schedule's batch gives the oracle's D' at the chosen block size."""
    from paper_2407_21552_gb300 import _abi as A
    from paper_2407_21552_gb300.autotune import tune
    base = synth.batch_specs(seed=47, count=6, lo=24, hi=80)
    built = {}

    def items_for(b):
        if b not in built:
            specs = [dict(sp, b=b) for sp in base]
            its = _engines(specs)
            tfs = [torch.from_numpy(T.tf_edit_sequence(70 + i, sp["N"], 1)[0]).cuda()
                   for i, (sp, _, _) in enumerate(its)]
            outs = [torch.empty(eng.G, dtype=torch.uint8, device="cuda") for _, _, eng in its]
            built[b] = (its, tfs, outs)
        its, tfs, outs = built[b]
        return [(eng.ctx, tfs[i].data_ptr(), outs[i].data_ptr()) for i, (_, _, eng) in enumerate(its)]

    cps, lps = (4, 24), (4, 8)
    easy = tune(items_for, 1e12, reps=3, ctas_per_sm=cps, loads_per_stage=lps)
    assert easy.block == 4 and set(easy.table) == {(4, c, k) for c in cps for k in lps}
    hard = tune(items_for, 0.0, reps=3, ctas_per_sm=cps, loads_per_stage=lps)
    assert set(hard.table) == {(b, c, k) for b in (4, 8) for c in cps for k in lps}
    assert hard.p50_us == min(hard.table.values())
    its, tfs, outs = built[hard.block]
    for o in outs:
        o.fill_(3)
    A.dm_update_tf_batch(items_for(hard.block), hard.tuning, _stream())
    torch.cuda.synchronize()
    for i, (sp, vol, _) in enumerate(its):
        pdm = oracle.build_partitions(synth.as_numpy(vol), hard.block, 1, sp["N"], sp["K"])[1]
        want = oracle.update_tf(pdm, tfs[i].cpu().numpy())[0].reshape(-1)
        assert np.array_equal(outs[i].cpu().numpy(), want), i
