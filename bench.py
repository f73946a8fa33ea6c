"""Benchmark: partitioned-distance-map TF update vs the plain full recompute on one GB300.

The headline workload is the large one (1024x1024x1795 12-bit, 256x256x449 blocks, K = 64,
1000 TF edits), whose maps stream from HBM.  A step is one session of it, one pass of the
whole hot path: the one-time precompute of the volume (partition table, POM masks, K
distance transforms; §3.1), then every TF edit of the workload through the partitioned
update (active set from the TF, then the Eq. 1 combine of the resident PDMs) and, on the
same edit, the plain full recompute it replaces (min/max occupancy + a fresh distance
transform).  `value` is the p50 latency of the timed updates (ms, lower is better).

Rules kept: inputs (volume, all TF edits) are resident in HBM before the timed region; the
L2 is flushed (a 256 MiB write, then a 256 MiB read, so no dirty lines remain) before every
timed call; kernels are timed with CUDA events on the stream they run on; clocks are
sampled with nvidia-smi during the timed region.  The line also carries the same edits
through the optional range index, an end-to-end figure through the host-buffer entry
point, the CPU oracle timed on the host cores, and the ct workload (512^3) as a sub-leg.
Other workloads: tiny, ct, mid, batch (64 uneven volumes, one batched launch pair),
serving (Poisson TF edits over 32 resident sessions), render (empty-space skipping) and
sweep (K = 4 .. 64).  `--impl reference` times the CPU oracle (plain C) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("TF-update latency (ms, p50/p99) & GB/s vs HBM peak: partitioned combine vs full "
          "recompute")
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20
# A device-side spin (about 100 us) issued before a timed call whose host-side issue is
# slow (the 64-item batch), so that the start event is reached only once the call is queued
# and the interval holds device time alone.
SPIN_CYCLES = 200_000
# DRAM bytes of the update kernel from one ncu capture (dram__bytes_read.sum and
# dram__bytes_write.sum over a few launches), keyed by workload, with the hash of the kernel
# code it was taken on; reported as null once that code has changed.  Reads are kept per
# byte of PDM planes that the same launches load (the kernel's own count), writes per
# block of the grid, so that the record scales to other edits and sizes.
NCU_TRAFFIC = {
    # k_update_fused, the first five edits of each workload's sequence (the bench's warm-up
    # session), DRAM read against the PDM bytes the same launches load: the combine loads
    # 16-byte chunks, DRAM moves larger atoms, so a chunk loaded next to finished ones costs
    # more than its 16 bytes (about 1.4x on the region-by-region maps, 1.01 on ct, where
    # nearly every chunk of every active plane is loaded)
    "ct": {"source_sha": "1376791f47d4a5d7", "read_per_loaded_byte": 1.009510,
           "write_per_block": 0.000000},
    "mid": {"source_sha": "1376791f47d4a5d7", "read_per_loaded_byte": 1.456792,
            "write_per_block": 0.072824},
    "large": {"source_sha": "1376791f47d4a5d7", "read_per_loaded_byte": 1.451583,
              "write_per_block": 0.556511},
}


# Warp instructions of the one-time precompute (its ten launches on these workloads:
# partition table, POM masks, x pass, y pass, z pass, plane cover, plane order, and the
# region bounds from the masks' rows: 2D x pass, 2D line pass, reduction) from one ncu
# capture (smsp__inst_executed.sum, one pass), keyed by workload, with the hash of the
# kernel code it was taken on; the precompute's ALU roofline is reported as null once that
# code has changed.
NCU_PRECOMPUTE_INST = {
    # mid (1024 x 1024 x 448, K = 64): 10,112 + 450,907,696 + 265,555,395 + 229,095,856 +
    # 442,675,200 + 957,440 + 1,158 + 1,026,181 + 1,701,416 + 508,928
    "mid": {"source_sha": "b8d26ebe65fb68c4", "warp_instructions": 1392439382.0},
    # large (1024 x 1024 x 1795, K = 64): 10,112 + 1,814,093,544 + 1,064,515,980 +
    # 918,354,416 (y, 256-block lines) + 1,701,677,056 (z, 449-block lines) +
    # 957,440 + 1,158 + 4,113,817 + 6,536,912 + 2,040,256
    "large": {"source_sha": "b8d26ebe65fb68c4", "warp_instructions": 5512300691.0},
}


def precompute_kernel_sources(csrc):
    """The precompute kernels' files (the plane order and region bounds are in the update's
    file) and the headers they include."""
    return [os.path.join(csrc, f) for f in ("dm_footprint.cu", "dm_dt.cu", "dm_update.cu",
                                            "dm_internal.cuh", "dm_build_batch.cuh")]


def precompute_alu(workload, pre_ms, clk, sms):
    """The precompute against the integer-ALU roofline: warp instructions (committed ncu
    capture) per second over the issue capacity, 4 warp instructions per cycle per SM at
    the median SM clock sampled under load; None without a capture of the current code."""
    tr = NCU_PRECOMPUTE_INST.get(workload)
    csrc = os.path.join(ROOT, "paper_2407_21552_gb300", "csrc")
    if not tr or tr.get("source_sha") != code_sha(*precompute_kernel_sources(csrc)):
        return None
    mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    peak = 4.0 * sms * mhz * 1e6
    achieved = tr["warp_instructions"] / (pre_ms * 1e-3)
    return {"bound": "alu", "warp_instructions": tr["warp_instructions"],
            "achieved": achieved, "peak": peak, "unit": "warp instructions/s",
            "frac": achieved / peak,
            "peak_source": f"4 warp instructions per cycle per SM x {sms} SMs x {mhz:.0f} MHz "
                           "(median SM clock sampled during the timed region)"}


def update_kernel_sources(csrc):
    """The update kernel's file and the header whose device helpers it inlines."""
    return [os.path.join(csrc, "dm_update.cu"), os.path.join(csrc, "dm_internal.cuh")]


def ncu_traffic(workload, G, mean_loaded):
    """DRAM bytes per update launch from the committed ncu capture, scaled to this grid and
    to the mean PDM bytes a launch loads; None once the kernel source has changed."""
    tr = NCU_TRAFFIC.get(workload)
    csrc = os.path.join(ROOT, "paper_2407_21552_gb300", "csrc")
    if not tr or tr.get("source_sha") != code_sha(*update_kernel_sources(csrc)):
        return None
    return float(tr["read_per_loaded_byte"] * mean_loaded + tr["write_per_block"] * G)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5,
                    help="timed steps; a step is one session of the workload (precompute "
                         "plus every TF edit)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload",
                    choices=["large", "ct", "tiny", "mid", "batch", "serving", "render",
                             "sweep"],
                    default="large")
    ap.add_argument("--edits", type=int, default=None,
                    help="TF edits per step (default: the workload's, 1000 for ct and large)")
    ap.add_argument("--serve-seconds", type=float, default=1.5,
                    help="serving workload: arrival window per rate and server")
    ap.add_argument("--batch-target-us", type=float, default=2000.0,
                    help="batch workload: latency target for the block-size choice")
    ap.add_argument("--cpu-edits", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ct-leg", action="store_true",
                    help="skip the ct sub-leg of the default large run")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
def pct(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def workload_name(name, w):
    X, Y, Z = w["dims"]
    return (f"{name}: {X}x{Y}x{Z} {'uint8' if w['dtype'] == 'u8' else 'uint16 (12-bit)'}, "
            f"b={w['block']} apron={w['apron']}, K={w['K']} partitions, N={w['N']} TF entries")


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (no MEASURED_PEAKS.json)"


def code_sha(*paths):
    """Hash of source files' code with comments and whitespace removed, so that the
    recorded ncu traffic stays tied to the kernel and not to its comments."""
    parts = []
    for path in paths:
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        parts.append(" ".join(text.split()))
    return hashlib.sha256("\n".join(parts).encode()).hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled in the background."""
    Q = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.gpu_id = gpu_id
        self.proc = None
        self.err = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            time.sleep(0.3)
        except Exception as e:   # no nvidia-smi
            self.err = str(e)

    def stop(self):
        if not self.proc:
            return {"unavailable": self.err or "nvidia-smi not started"}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 9]
        if not rows:
            return {"unavailable": "no samples"}
        sm = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[6:10]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max((float(r[4]) for r in rows
                                    if r[4].strip().replace(".", "").isdigit()), default=None)}


def smi_gpu_id(dev):
    """nvidia-smi -i selector (UUID) for a torch device, or None."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(dev).uuid).lower().replace("gpu-", "")
        out = subprocess.run(["nvidia-smi", "--query-gpu=uuid", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout.split()
        for line in out:
            if line.strip().lower().replace("gpu-", "") == u:
                return line.strip()
    except Exception:
        pass
    return None


def dist_setup():
    import torch
    import torch.distributed as dist
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1 and not dist.is_initialized():
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def reduce_max(values, ws):
    """Element-wise max of a list of floats over ranks (identity at world size 1)."""
    if ws <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(values, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.cpu().tolist()


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------------- CPU oracle
def oracle_slab(name, w):
    """The workload's volume cut to a z-slab of whole block-slices (about 1M blocks), as a
    host numpy array, with G / G_slab.  The volume is generated on the GPU when there is
    one (the CPU generator is slow at this size) and only the slab is copied to the host."""
    import torch
    import synth
    b = w["block"]
    X, Y, Z = w["dims"]
    gx, gy, gz = -(-X // b), -(-Y // b), -(-Z // b)
    slab_bz = max(1, min(gz, (1 << 20) // (gx * gy)))
    zs = min(Z, slab_bz * b)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    vol = synth.make_volume(name, device=dev)
    sub = np.ascontiguousarray(synth.as_numpy(vol[:zs]))
    del vol
    if dev == "cuda":
        torch.cuda.empty_cache()
    return sub, (gx * gy * gz) / (gx * gy * (-(-zs // b)))


def oracle_sample(name, w, edits, n_edits, n_full=3):
    """The CPU oracle, as it stands, on a bounded sample of the workload: a z-slab of the
    volume (whole block-slices, about 1M blocks), its one-time precompute timed once, then
    `n_edits` TF updates and `n_full` min/max full recomputes timed single-threaded; times
    scale to the whole volume by G / G_slab (all three are linear in G)."""
    import oracle
    b, a, N, K = w["block"], w["apron"], w["N"], w["K"]
    sub, scale = oracle_slab(name, w)
    zs, Y, X = sub.shape
    t0 = time.perf_counter()
    _, pdm, vmin, vmax = oracle.build_partitions(sub, b, a, N, K)
    pre_s = time.perf_counter() - t0
    upd = []
    for tf in edits[:n_edits]:
        t0 = time.perf_counter()
        oracle.update_tf(pdm, tf)
        upd.append((time.perf_counter() - t0) * 1e3 * scale)
    threads = os.cpu_count() or 1
    tput = oracle_throughput(pdm, edits[:max(1, n_edits)], scale, threads) if n_edits else None
    full = []
    for tf in edits[:n_full]:
        t0 = time.perf_counter()
        oracle.full_recompute_minmax(vmin, vmax, tf)
        full.append((time.perf_counter() - t0) * 1e3 * scale)
    return dict(pdm=pdm, scale=scale, slab=(X, Y, zs), pre_s=pre_s, upd=upd, full=full,
                tput=tput, threads=threads)


def oracle_throughput(pdm, edits, scale, threads):
    """Whole-volume edits per second of the oracle's update with one edit per host thread
    at a time (the C call releases the GIL): 2 x `threads` edits over the same slab, each
    slab edit counted as 1/scale of a whole-volume edit."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    n = 2 * threads
    batch = [edits[i % len(edits)] for i in range(n)]
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda tf: oracle.update_tf(pdm, tf), batch[:threads]))      # warm-up
        t0 = time.perf_counter()
        list(ex.map(lambda tf: oracle.update_tf(pdm, tf), batch))
        dt = time.perf_counter() - t0
    return n / (dt * scale)


def cpu_baseline_block(s, n_edits):
    X, Y, zs = s["slab"]
    return {"value": pct(s["upd"], 50), "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": (f"z-slab {X}x{Y}x{zs} of the same volume (its precompute took "
                       f"{s['pre_s']:.1f} s, outside the per-edit times), {n_edits} TF edits "
                       f"through the oracle's step 1 + "
                       f"Eq. 1, single-threaded C; per-edit times scaled by G/G_slab = "
                       f"{s['scale']:.3f}"),
            "full_recompute_p50_ms": pct(s["full"], 50),
            "precompute_ms": s["pre_s"] * 1e3 * s["scale"],
            "nproc": os.cpu_count(),
            "throughput_all_cores": {"edits_per_s": s["tput"], "threads": s["threads"],
                                     "sample": "one whole-volume-equivalent edit per thread "
                                               "at a time, same slab and scale"}}


# --------------------------------------------------------------------------- our arm
def session_leg(dev, name, steps, warmup, flush, peak, ws, edits=None, e2e=True, index=True):
    """One workload measured as sessions.  A step is one pass of the whole hot path over
    the workload: the one-time precompute of its volume (partition table, POM masks, K
    distance transforms; §3.1), then every TF edit of the workload (1000 for ct and large)
    through the partitioned update (step 1 + Eq. 1) and, on the same edit, the plain min/max
    full recompute it replaces.  The L2 is flushed before every timed call, and every call
    is timed with CUDA events on its stream.  After the timed steps: the same edits with the
    optional range index, and end to end through the host-buffer entry point."""
    import torch
    import synth
    from paper_2407_21552_gb300 import DM_U8, DM_U16, DM_INDEX_RANGES, dm_set_profile_events
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    w = synth.WORKLOADS[name]
    X, Y, Z = w["dims"]
    dtype = DM_U8 if w["dtype"] == "u8" else DM_U16
    stream = torch.cuda.current_stream(dev)
    vol = synth.make_volume(name, device=dev)
    vol_sha = synth.volume_sha256(vol) if vol.numel() <= (1 << 28) else None
    eng = PartitionedDistanceMaps((X, Y, Z), dtype, w["block"], w["apron"], w["K"], w["N"],
                                  device=dev)
    G, V = eng.G, X * Y * Z
    s_bytes = 1 if w["dtype"] == "u8" else 2
    E = int(edits or w["edits"])
    edit_list = synth.tf_edit_sequence(w["seed"], w["N"], E)
    tfs = torch.from_numpy(np.stack(edit_list)).to(dev)            # [E, N, 4], resident
    Wm = (w["K"] + 63) // 64
    am = torch.zeros((E, Wm), dtype=torch.int64, device=dev)
    out = torch.empty(G, dtype=torch.uint8, device=dev)
    out_full = torch.empty(G, dtype=torch.uint8, device=dev)

    def step(ev=None):
        """One session; `ev` = (pre0, pre1, ua, ub, fa, fb) events, or None (warm-up)."""
        flush()
        if ev:
            ev[0].record(stream)
        eng.build_partitions(vol)
        if ev:
            ev[1].record(stream)
        for e in range(E):
            flush()
            if ev:
                ev[2][e].record(stream)
            eng.update_tf(tfs[e], out=out, active_mask=am[e])
            if ev:
                ev[3][e].record(stream)
            flush()
            if ev:
                ev[4][e].record(stream)
            eng.full_recompute(tfs[e], out=out_full)
            if ev:
                ev[5][e].record(stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    mk = lambda n: [torch.cuda.Event(enable_timing=True) for _ in range(n)]  # noqa: E731
    evs = [(*mk(2), mk(E), mk(E), mk(E), mk(E)) for _ in range(steps)]
    for ev in evs:                   # torch creates each CUDA event on its first record
        for e in ev[:2]:
            e.record(stream)
        for lst in ev[2:]:
            for e in lst:
                e.record(stream)
    region0 = torch.cuda.Event(enable_timing=True)
    region1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(smi_gpu_id(dev))
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize(dev)
    region0.record(stream)
    for k in range(steps):
        step(evs[k])
    region1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    clk = clocks.stop()
    region_ms = region0.elapsed_time(region1)
    pre = [ev[0].elapsed_time(ev[1]) for ev in evs]
    upd = [ev[2][e].elapsed_time(ev[3][e]) for ev in evs for e in range(E)]
    full = [ev[4][e].elapsed_time(ev[5][e]) for ev in evs for e in range(E)]
    del evs
    masks = am.cpu().numpy().view(np.uint64)
    nact = np.array([sum(bin(int(x)).count("1") for x in row) for row in masks])
    # the PDM bytes each edit's combine loads (plane order, stop at 0), counted in the kernel
    # on an untimed replay of the same edits on the same maps: with the write of D', the
    # update's algorithmic bytes per launch, at most the method's (|S| + 1) G
    loaded = torch.zeros(E, dtype=torch.int64, device=dev)
    for e in range(E):
        eng.set_profile_counter(loaded[e:e + 1])
        eng.update_tf(tfs[e], out=out)
    eng.set_profile_counter(None)
    loaded = loaded.cpu().numpy().astype(np.float64)
    bytes_upd = np.tile(loaded + G, steps)                          # per launch, algorithmic
    bytes_plain = np.tile((nact + 1) * G, steps).astype(np.float64)  # every active plane read
    upd_a = np.asarray(upd)
    # the update of an N <= 8192 TF is one kernel (k_update_fused): its events bracket it
    fused = w["N"] <= 8192
    achieved = float(bytes_upd.sum() / (upd_a.sum() * 1e-3)) / 1e9 if fused else None

    # ---- the same edits with the optional partition-range index (DM_INDEX_RANGES)
    idx = None
    if index:
        idx_eng = PartitionedDistanceMaps((X, Y, Z), dtype, w["block"], w["apron"], w["K"],
                                          w["N"], device=dev, with_minmax=False,
                                          index_mode=DM_INDEX_RANGES)
        idx_eng.build_partitions(vol)
        idx_eng.release_mask()
        for e in range(min(warmup, E)):
            idx_eng.update_tf(tfs[e], out=out)
        ia, ib = mk(E), mk(E)
        torch.cuda.synchronize(dev)
        for e in range(E):
            flush()
            ia[e].record(stream)
            idx_eng.update_tf(tfs[e], out=out)
            ib[e].record(stream)
        torch.cuda.synchronize(dev)
        upd_idx = [ia[e].elapsed_time(ib[e]) for e in range(E)]
        idx = {"p50_ms": pct(upd_idx, 50), "p99_ms": pct(upd_idx, 99),
               "pdm_planes": int(idx_eng.sizes.pdm_planes), "edits": E}
        idx_eng.close()
        del idx_eng
        torch.cuda.empty_cache()

    # ---- end to end through the host-buffer entry point: pinned TF in, D' out to pinned
    #      host memory, stream sync; host wall clock per call.  The update kernel is timed
    #      inside the same calls (profile events) and the TF copy alone with events, which
    #      splits the wall time into its parts.
    e2e_res = None
    if e2e:
        h_tf = torch.empty((E, w["N"], 4), dtype=torch.float32).pin_memory()
        h_tf.copy_(tfs.cpu())
        h_out = torch.empty(G, dtype=torch.uint8).pin_memory()
        views = [h_tf[k] for k in range(E)]          # the per-edit host TFs, made up front
        for k in range(min(warmup, E)):
            eng.update_tf_host(views[k], h_out)
        ka, kb = mk(E), mk(E)
        for e in ka + kb:
            e.record(stream)
        torch.cuda.synchronize(dev)
        lat = []
        barrier(ws)
        for k in range(E):
            dm_set_profile_events(eng.ctx, ka[k].cuda_event, kb[k].cuda_event)
            t0 = time.perf_counter()
            eng.update_tf_host(views[k], h_out)
            lat.append((time.perf_counter() - t0) * 1e3)
        dm_set_profile_events(eng.ctx, None, None)
        barrier(ws)
        kern = [ka[k].elapsed_time(kb[k]) for k in range(E)]
        tf_dev = torch.empty((w["N"], 4), dtype=torch.float32, device=dev)
        ca, cb = mk(50), mk(50)
        for k in range(50):
            ca[k].record(stream)
            tf_dev.copy_(views[k % E], non_blocking=True)
            cb[k].record(stream)
        torch.cuda.synchronize(dev)
        copy_ms = pct([ca[k].elapsed_time(cb[k]) for k in range(50)], 50)
        p50 = pct(lat, 50)
        e2e_res = {"value": p50, "unit": "ms", "p99": pct(lat, 99), "edits": E,
                   "h2d_bytes_per_step": int(V * s_bytes + E * w["N"] * 16),
                   "d2h_bytes_per_step": int(E * G),
                   "per_edit": {"h2d_bytes": int(w["N"] * 16), "d2h_bytes": int(G)},
                   "breakdown_p50_ms": {
                       "tf_h2d_copy": copy_ms,
                       "update_kernel_writing_host_memory": pct(kern, 50),
                       "host_side_rest": p50 - pct(kern, 50) - copy_ms},
                   "how": "dm_update_tf_host per edit: pinned TF -> device, step 1 + Eq. 1 with "
                          "D' written into pinned host memory, stream sync; host wall clock "
                          "per call over the workload's edits.  Per step the volume is also "
                          "uploaded once (counted in h2d_bytes_per_step)"}
    eng.close()
    del eng, vol, tfs, out, out_full
    torch.cuda.empty_cache()
    p50u, p99u, p50f, p99f, region_max = reduce_max(
        [pct(upd, 50), pct(upd, 99), pct(full, 50), pct(full, 99), region_ms], ws)
    pre_ms = float(np.median(pre))
    pre_bytes = s_bytes * V + w["K"] * G
    traffic = ncu_traffic(name, G, float(loaded.mean()))
    res = {
        "workload": workload_name(name, w), "volume_xyz": [X, Y, Z], "grid_G": G,
        "edits_per_step": E, "volume_sha256": vol_sha, "region_ms": region_max,
        "update": {"p50_ms": p50u, "p99_ms": p99u, "mean_ms": float(upd_a.mean()),
                   "calls": len(upd),
                   "gbs_p50": float(np.median(bytes_upd / (upd_a * 1e-3)) / 1e9),
                   "voxels_per_s_p50": V / (p50u * 1e-3),
                   "loaded_fraction_of_active_planes": float(loaded.sum() / (nact.sum() * G))
                   if nact.sum() else None,
                   "plain_bytes_per_launch": float(bytes_plain.mean()),
                   "plain_gbs_mean": float(bytes_plain.sum() / (upd_a.sum() * 1e-3)) / 1e9,
                   "loaded_bytes_first_edits": [int(x) for x in loaded[:5]]},
        "full_recompute": {"p50_ms": p50f, "p99_ms": p99f, "mean_ms": float(np.mean(full)),
                           "mode": "min/max occupancy", "voxels_per_s_p50": V / (p50f * 1e-3)},
        "speedup_vs_full_recompute_p50": p50f / p50u,
        "active_partitions": {"mean": float(nact.mean()), "min": int(nact.min()),
                              "max": int(nact.max()), "K": w["K"]},
        "precompute": {"ms": pre_ms, "min_ms": float(np.min(pre)),
                       "algorithmic_gb": pre_bytes / 1e9,
                       "gbs": pre_bytes / (pre_ms * 1e-3) / 1e9,
                       "frac_of_hbm": pre_bytes / (pre_ms * 1e-3) / 1e9 / peak[0],
                       "alu_roofline": precompute_alu(
                           name, pre_ms, clk, torch.cuda.get_device_properties(dev).multi_processor_count)},
        "roofline": {"kernel": "k_update_fused (step 1 + Eq. 1)", "bound": "hbm",
                     "achieved": achieved, "peak": peak[0], "unit": "GB/s",
                     "frac": achieved / peak[0] if achieved else None,
                     "traffic": traffic,
                     # DRAM bytes moved (the traffic record) per second of the mean launch,
                     # against the same peak: the combine loads 16-byte chunks, DRAM moves
                     # larger atoms, so this runs above `frac` where chunks finish early
                     "dram_frac": (traffic / (upd_a.mean() * 1e-3) / 1e9 / peak[0]
                                   if traffic and fused else None),
                     "peak_source": peak[1],
                     "algorithmic_bytes_per_launch": float(bytes_upd.mean()),
                     "mean_launch_us": float(upd_a.mean() * 1e3)},
        "clocks": clk,
        "e2e": e2e_res,
        # the precompute: partition table, POM, x, y, z, plane cover and order, then the
        # region bounds from the masks' rows (2D x pass, 2D line pass, reduction) where
        # the grid's rows tile its regions (every bench workload), else one pass over planes
        "gpu_launches": steps * (10 + E * ((1 if fused else 2) + 4)),
    }
    if idx:
        idx["speedup_vs_full_recompute_p50"] = p50f / idx["p50_ms"]
        idx["note"] = ("optional DM_INDEX_RANGES: same D', two index planes per run of active "
                       f"partitions; memory {idx['pdm_planes']}/{w['K']} of the plain PDMs")
        res["update_range_index"] = idx
    return res, edit_list


def run_ours(args, ws, rank, local):
    import torch
    import synth
    from paper_2407_21552_gb300.build import build as build_lib

    build_lib()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = synth.WORKLOADS[args.workload]
    peak = measured_peak()
    flush_w = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    flush_r = torch.zeros(L2_FLUSH_BYTES // 8, dtype=torch.int64, device=dev)

    def flush():
        """Evict the L2: write 256 MiB, then read 256 MiB so that no dirty line is left
        to be written back inside the next timed call."""
        flush_w.zero_()
        flush_r.max()

    main, edits = session_leg(dev, args.workload, args.steps, args.warmup, flush, peak, ws,
                              edits=args.edits, e2e=not args.no_e2e)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        s = oracle_sample(args.workload, w, edits, args.cpu_edits)
        cpu = cpu_baseline_block(s, args.cpu_edits)
    sub = None
    if ws == 1 and args.workload == "large" and not args.no_ct_leg:
        sub, _ = session_leg(dev, "ct", 1, 1, flush, peak, ws, e2e=not args.no_e2e)
    if rank != 0:
        return
    X, Y, Z = w["dims"]
    K = args.steps
    res = {
        "metric": METRIC, "value": main["update"]["p50_ms"], "unit": "ms", "n_gpus": ws,
        "steps": K, "warmup": args.warmup, "ms_per_step": main["region_ms"] / K,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": main["workload"], "volume_xyz": [X, Y, Z],
                   "grid_G": main["grid_G"], "edits_per_step": main["edits_per_step"],
                   "l2": "flushed before every timed call (256 MiB device write, then a "
                         "256 MiB read)",
                   "volume_sha256": main["volume_sha256"],
                   "parallelism": f"replicas x{ws}"},
        "step": "one session of the workload: the one-time precompute of its volume, then "
                f"its {main['edits_per_step']} TF edits, each through the partitioned update "
                "(step 1 + Eq. 1) and the plain min/max full recompute; value = p50 of the "
                f"{main['update']['calls']} timed updates",
    }
    for key in ("update", "full_recompute", "speedup_vs_full_recompute_p50",
                "update_range_index", "active_partitions", "precompute", "roofline"):
        if key in main:
            res[key] = main[key]
    res["cpu_baseline"] = cpu
    res["e2e"] = main["e2e"]
    res["ct_workload"] = sub
    res["gpu_launches"] = main["gpu_launches"]
    res["clocks"] = main["clocks"]
    res["paper_context"] = ("paper: up to 30x faster DM update (RTX 4090, OpenGL/GLSL, "
                            "Table 1; kingsnake 1024x1024x795 at n = 64: 1.23-1.99 ms update, "
                            "7.28-21.40 ms DM recompute, 913.7 ms init); not re-run here (no "
                            "graphics stack)")
    print(json.dumps(res))


# ------------------------------------------------------------ batched instances workload
def run_batch(args, ws, rank, local):
    """64 volumes of uneven size (sides U[64, 384], uint8 / 12-bit, K 16 / 32), one TF edit
    each per step: 64 separate update launches vs one batched launch pair vs a CUDA-graph
    replay of the batched pair.  The autotuner picks the block size and combine grid."""
    import ctypes
    import torch
    import synth
    from paper_2407_21552_gb300 import DM_U8, DM_U16, _abi as A
    from paper_2407_21552_gb300.autotune import tune
    from paper_2407_21552_gb300.build import build as build_lib
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps

    build_lib()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    specs = synth.batch_specs()
    n = len(specs)
    vols = [synth.volume_of(sp["kind"], sp["dims"], sp["seed"], device=dev) for sp in specs]
    E = max(8, min(64, args.steps + args.warmup))
    NMAX = max(sp["N"] for sp in specs)
    edits = torch.zeros((E, n, NMAX, 4), dtype=torch.float32, device=dev)
    for i, sp in enumerate(specs):
        seq = synth.tf_edit_sequence(sp["seed"], sp["N"], E)
        edits[:, i, : sp["N"]] = torch.from_numpy(np.stack(seq)).to(dev)
    engines = {}

    def build(b):
        if b not in engines:
            engs = []
            for sp, v in zip(specs, vols):
                X, Y, Z = sp["dims"]
                e = PartitionedDistanceMaps((X, Y, Z), DM_U8 if sp["kind"] == "u8" else DM_U16,
                                            b, 1, sp["K"], sp["N"], device=dev, with_minmax=False)
                e.build_partitions(v)
                e.release_mask()
                engs.append(e)
            torch.cuda.synchronize(dev)
            outs = [torch.empty(e.G, dtype=torch.uint8, device=dev) for e in engs]
            engines[b] = (engs, outs)
        return engines[b]

    def items_for(b, k):
        engs, outs = build(b)
        return [(e.ctx, edits[k, i].data_ptr(), outs[i].data_ptr()) for i, e in enumerate(engs)]

    tr = tune(lambda b: items_for(b, 0), args.batch_target_us, device=dev)
    engs, outs = build(tr.block)
    stream = torch.cuda.current_stream(dev)
    sp_ = ctypes.c_void_p(stream.cuda_stream)
    # graph of the batched pair reading fixed TF buffers
    tf_fixed = torch.zeros((n, NMAX, 4), dtype=torch.float32, device=dev)
    fixed_items = [(e.ctx, tf_fixed[i].data_ptr(), outs[i].data_ptr()) for i, e in enumerate(engs)]
    A.dm_update_tf_batch(fixed_items, tr.tuning, sp_)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        A.dm_update_tf_batch(fixed_items, tr.tuning,
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    flush_w = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    flush_r = torch.zeros(L2_FLUSH_BYTES // 8, dtype=torch.int64, device=dev)

    def flush():
        flush_w.zero_()
        flush_r.max()
    for k in range(args.warmup):
        for i, e in enumerate(engs):
            e.update_tf(edits[k % E, i, : specs[i]["N"]], out=outs[i])
        A.dm_update_tf_batch(items_for(tr.block, k % E), tr.tuning, sp_)
        tf_fixed.copy_(edits[k % E])
        graph.replay()
    torch.cuda.synchronize(dev)
    K = args.steps
    prepared = [A.PreparedBatch(items_for(tr.block, kk)) for kk in range(E)]   # marshalled once
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(K)]
    am = torch.zeros((K, n, 4), dtype=torch.int64, device=dev)     # S of every item and step
    clocks = ClockSampler(smi_gpu_id(dev))
    clocks.start()
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    r0.record(stream)
    for k in range(K):
        kk = k % E
        flush()
        ev[k][0].record(stream)
        for i, e in enumerate(engs):
            e.update_tf(edits[kk, i, : specs[i]["N"]], out=outs[i], active_mask=am[k, i])
        ev[k][1].record(stream)
        flush()
        torch.cuda._sleep(SPIN_CYCLES)              # the device is busy while the host issues
        ev[k][2].record(stream)
        A.dm_update_tf_batch(prepared[kk], tr.tuning, sp_)
        ev[k][3].record(stream)
        flush()
        ev[k][4].record(stream)
        tf_fixed.copy_(edits[kk])
        graph.replay()
        ev[k][5].record(stream)
    r1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    sep = [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]
    bat = [ev[k][2].elapsed_time(ev[k][3]) for k in range(K)]
    gra = [ev[k][4].elapsed_time(ev[k][5]) for k in range(K)]
    vox = sum(int(np.prod(sp["dims"])) for sp in specs)
    # algorithmic bytes of a step: the PDM bytes the batched combine loads for the step's
    # edits (plane order, stop at 0), counted in the kernel on an untimed replay of the same
    # calls, plus the writes of the n maps D'; at most sum over items of (|S_i| + 1) G_i,
    # the bytes when every active plane is read (the same edits go through the separate and
    # the batched updates)
    Gs = np.array([e.G for e in engs], dtype=np.float64)
    masks = am.cpu().numpy().view(np.uint64)
    nact = np.array([[sum(bin(int(x)).count("1") for x in masks[k, i]) for i in range(n)]
                     for k in range(K)], dtype=np.float64)
    counted = torch.zeros(E, dtype=torch.int64, device=dev)
    for kk in sorted({k % E for k in range(K)}):       # the counter of items[0]'s context
        engs[0].set_profile_counter(counted[kk:kk + 1])
        A.dm_update_tf_batch(prepared[kk], tr.tuning, sp_)
    engs[0].set_profile_counter(None)
    counted = counted.cpu().numpy().astype(np.float64)
    step_loaded = np.array([counted[k % E] for k in range(K)])
    step_bytes = step_loaded + Gs.sum()
    plain_step_bytes = ((nact + 1) * Gs).sum(axis=1)
    bat_gbs = step_bytes / (np.array(bat) * 1e-3) / 1e9
    peak, peak_src = measured_peak()
    multi = multi_edit_leg(engs, edits, specs, tr, flush, stream, min(8, E), reps=max(5, K))
    pre = precompute_batch_leg(engs, vols, flush, stream, reps=max(5, K))
    if rank != 0:
        return
    res = {
        "metric": METRIC + " (batched instances)", "value": pct(bat, 50), "unit": "ms",
        "n_gpus": ws, "steps": K, "warmup": args.warmup, "ms_per_step": r0.elapsed_time(r1) / K,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": f"batch: {n} volumes, sides U[64,384], uint8/12-bit, K 16/32, "
                               f"one TF edit each", "voxels": vox,
                   "l2": "flushed before every timed call (256 MiB write, then 256 MiB read)"},
        "separate_launches": {"p50_ms": pct(sep, 50), "p99_ms": pct(sep, 99),
                              "launches": n},
        "batched": {"p50_ms": pct(bat, 50), "p99_ms": pct(bat, 99), "launches": 2},
        "batched_graph": {"p50_ms": pct(gra, 50), "p99_ms": pct(gra, 99),
                          "note": "includes the device copy of the 64 TFs into the "
                                  "graph's fixed buffers"},
        "speedup_batched_vs_separate_p50": pct(sep, 50) / pct(bat, 50),
        "roofline": {"kernel": "k_active_group + k_combine_group (launch pair)", "bound": "hbm",
                     "achieved": float(step_bytes.sum() / (np.sum(bat) * 1e-3) / 1e9),
                     "achieved_p50_step": float(np.median(bat_gbs)), "peak": peak,
                     "unit": "GB/s", "frac": float(step_bytes.sum() / (np.sum(bat) * 1e-3) / 1e9) / peak,
                     "traffic": None, "peak_source": peak_src,
                     "algorithmic_bytes_per_step": float(step_bytes.mean()),
                     "plain_bytes_per_step": float(plain_step_bytes.mean()),
                     "loaded_fraction_of_active_planes":
                         float(step_loaded.sum() / (nact * Gs).sum()) if nact.sum() else None,
                     "mean_active_partitions": float(nact.mean())},
        "autotune": {"block": tr.block, "combine_ctas_per_sm": tr.ctas_per_sm,
                     "loads_per_stage": tr.loads_per_stage,
                     "target_us": args.batch_target_us,
                     "table_us": {f"b{b}_c{c}_l{kb}": v for (b, c, kb), v in tr.table.items()}},
        "several_edits_per_volume": multi,
        "precompute_batched": pre,
        "gpu_launches": K * (n + 2 + 2),
        "clocks": clk,
    }
    print(json.dumps(res))


def multi_edit_leg(engs, edits, specs, tr, flush, stream, n_edits, reps):
    """Several TF edits per volume in one call: the batch's volumes with `n_edits` edits
    each through dm_update_tf_batch_ws (a volume's edits share their plane reads), against
    the same edits as `n_edits` single-edit batched calls.  CUDA events, L2 flushed first."""
    import ctypes
    import torch
    from paper_2407_21552_gb300 import _abi as A
    dev = edits.device
    n = len(engs)
    sp_ = ctypes.c_void_p(stream.cuda_stream)
    outs = [[torch.empty(e.G, dtype=torch.uint8, device=dev) for e in engs]
            for _ in range(n_edits)]
    per_call = [A.PreparedBatch([(e.ctx, edits[k, i].data_ptr(), outs[k][i].data_ptr())
                                 for i, e in enumerate(engs)]) for k in range(n_edits)]
    every = A.PreparedBatch([(e.ctx, edits[k, i].data_ptr(), outs[k][i].data_ptr())
                             for k in range(n_edits) for i, e in enumerate(engs)])
    nbytes = A.dm_batch_workspace_bytes(every.n)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    # the active sets, for the algorithmic bytes
    am = torch.zeros((n_edits, n, 4), dtype=torch.int64, device=dev)
    for k in range(n_edits):
        for i, e in enumerate(engs):
            e.update_tf(edits[k, i, : specs[i]["N"]], out=outs[k][i], active_mask=am[k, i])
    torch.cuda.synchronize(dev)
    m = am.cpu().numpy().view(np.uint64)
    Gs = np.array([e.G for e in engs], dtype=np.float64)
    cnt = lambda row: sum(bin(int(x)).count("1") for x in row)  # noqa: E731
    sep_plain = sum((cnt(m[k, i]) + 1) * Gs[i] for k in range(n_edits) for i in range(n))
    union = [np.bitwise_or.reduce(m[:, i], axis=0) for i in range(n)]
    ws_plain = sum((cnt(union[i]) + n_edits) * Gs[i] for i in range(n))
    # algorithmic bytes: the PDM bytes each variant's combines load (counted in the kernels
    # on an untimed replay, the counter of items[0]'s context) plus the writes of the maps
    loaded = torch.zeros(2, dtype=torch.int64, device=dev)
    engs[0].set_profile_counter(loaded[0:1])
    for k in range(n_edits):
        A.dm_update_tf_batch(per_call[k], tr.tuning, sp_)
    engs[0].set_profile_counter(loaded[1:2])
    A.dm_update_tf_batch_ws(every, tr.tuning, ws.data_ptr(), nbytes, sp_)
    engs[0].set_profile_counter(None)
    loaded = loaded.cpu().numpy().astype(np.float64)
    sep_bytes = float(loaded[0] + n_edits * Gs.sum())
    ws_bytes = float(loaded[1] + n_edits * Gs.sum())
    t_sep, t_ws = [], []
    for r in range(reps + 2):
        flush()
        torch.cuda._sleep(SPIN_CYCLES)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for k in range(n_edits):
            A.dm_update_tf_batch(per_call[k], tr.tuning, sp_)
        b.record(stream)
        flush()
        torch.cuda._sleep(SPIN_CYCLES)
        c, d = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c.record(stream)
        A.dm_update_tf_batch_ws(every, tr.tuning, ws.data_ptr(), nbytes, sp_)
        d.record(stream)
        torch.cuda.synchronize(dev)
        if r >= 2:
            t_sep.append(a.elapsed_time(b))
            t_ws.append(c.elapsed_time(d))
    peak, _ = measured_peak()
    p_ws = pct(t_ws, 50)
    return {"volumes": n, "edits_per_volume": n_edits,
            "separate_calls": {"p50_ms": pct(t_sep, 50), "calls": n_edits,
                               "algorithmic_bytes": sep_bytes, "plain_bytes": sep_plain},
            "one_call": {"p50_ms": p_ws, "algorithmic_bytes": ws_bytes, "plain_bytes": ws_plain,
                         "gbs": ws_bytes / (p_ws * 1e-3) / 1e9,
                         "frac": ws_bytes / (p_ws * 1e-3) / 1e9 / peak},
            "speedup": pct(t_sep, 50) / p_ws}


def precompute_batch_leg(engs, vols, flush, stream, reps):
    """The one-time precompute of the batch's volumes: one dm_build_partitions call per
    volume against one dm_build_partitions_batch call for all of them.  CUDA events, L2
    flushed first; a spin long enough for the host to queue every call precedes the start
    event, so that both intervals hold device time alone."""
    import torch
    from paper_2407_21552_gb300.maps import build_partitions_batch
    dev = vols[0].device
    # algorithmic bytes: every volume read once, every PDM plane written once
    nbytes = float(sum(v.numel() * v.element_size() + e.K * e.G for e, v in zip(engs, vols)))
    t_sep, t_bat = [], []
    for r in range(reps + 2):
        flush()
        torch.cuda._sleep(20 * SPIN_CYCLES)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for e, v in zip(engs, vols):
            e.build_partitions(v)
        b.record(stream)
        flush()
        torch.cuda._sleep(20 * SPIN_CYCLES)
        c, d = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c.record(stream)
        build_partitions_batch(engs, vols)
        d.record(stream)
        torch.cuda.synchronize(dev)
        if r >= 2:
            t_sep.append(a.elapsed_time(b))
            t_bat.append(c.elapsed_time(d))
    peak, _ = measured_peak()
    p_bat = pct(t_bat, 50)
    return {"volumes": len(engs), "algorithmic_bytes": nbytes,
            "separate_calls": {"p50_ms": pct(t_sep, 50), "calls": len(engs)},
            "one_call": {"p50_ms": p_bat, "gbs": nbytes / (p_bat * 1e-3) / 1e9,
                         "frac_of_hbm": nbytes / (p_bat * 1e-3) / 1e9 / peak},
            "speedup": pct(t_sep, 50) / p_bat}


# -------------------------------------------------------------------- serving workload
def _open_loop(sch, n_sess, rate, n_req, tfs, rng):
    """Poisson arrivals at `rate` edits/s over the sessions, uniformly chosen; returns the
    wall time until every edit completed."""
    arrive = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    sess = rng.integers(0, n_sess, size=n_req)
    t0 = time.perf_counter()
    k = 0
    while k < n_req or sch.has_work():
        now = time.perf_counter() - t0
        while k < n_req and arrive[k] <= now:
            sch.submit(int(sess[k]), tfs[k % len(tfs)], t_arrival=t0 + arrive[k])
            k += 1
        sch.poll()
    return time.perf_counter() - t0


def _serve_stats(sch, wall, rate):
    lat = np.array(sch.stats.latencies) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "edits": int(len(lat)), "sustained_edits_per_s": len(lat) / wall,
            "offered_edits_per_s": rate, "batches": sch.stats.batches,
            "mean_batch": float(np.mean(sch.stats.batch_sizes)),
            "max_batch": int(np.max(sch.stats.batch_sizes))}


def _knee(rows):
    """The highest offered rate the server sustains (within 5 %) with p99 at most 10x the
    p99 of the lowest rate: above it the queues grow and p99 leaves the low-load regime."""
    base = rows[0]["p99_ms"]
    knee = rows[0]
    for r in rows:
        if r["sustained_edits_per_s"] >= 0.95 * r["offered_edits_per_s"] and r["p99_ms"] <= 10 * base:
            knee = r
    return {"offered_edits_per_s": knee["offered_edits_per_s"], "p50_ms": knee["p50_ms"],
            "p99_ms": knee["p99_ms"], "sustained_edits_per_s": knee["sustained_edits_per_s"],
            "mean_batch": knee["mean_batch"]}


def run_serving(args, ws, rank, local):
    """32 sessions (12-bit volumes with sides U[256, 1024], K in {16, 32, 64}) admitted
    under a 150 GB HBM budget; TF edits arrive as a Poisson process over the sessions at
    200 .. 100000 edits/s.  Three servers in the same loop on 3 streams: the partitioned
    one batching one edit per session per batch, the partitioned one batching up to 4 edits
    per session (dm_update_tf_batch_ws: a session's edits share their plane reads), and a
    full recompute per edit.  The knee of each (the highest rate it sustains with a p99
    near its low-load p99) is reported.  Then: 1000 edits/s under a budget of 40 % of the
    sessions' bytes, evicting idle sessions to host memory and readmitting them; and a
    churn run where 48 sessions of b = 2 maps with K in {128, 256} (about 290 GB in all)
    open at 200 per second under the 150 GB budget, their maps built at admission, each
    sending 40 edits and leaving once they completed, so that sessions wait for admission."""
    import torch
    import synth
    from paper_2407_21552_gb300 import DM_U16
    from paper_2407_21552_gb300.build import build as build_lib
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    from paper_2407_21552_gb300.serving import DeviceExecutor, Scheduler, SessionSpec

    build_lib()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(5)
    n_sess, budget = 32, 150 * 10**9
    engines, specs = [], []
    for sid in range(n_sess):
        side = int(rng.integers(256, 1025))
        K = int(rng.choice([16, 32, 64]))
        vol = synth.volume_of("u16", (side, side, side), 2000 + sid, device=dev)
        eng = PartitionedDistanceMaps((side, side, side), DM_U16, 4, 1, K, 4096, device=dev)
        eng.build_partitions(vol)
        eng.release_mask()
        del vol
        engines.append(eng)
        s = eng.sizes
        specs.append(SessionSpec(sid, int(s.pdm_bytes + s.minmax_bytes + s.scratch_bytes
                                          + 3 * 4 * s.out_bytes), dict(engine=eng)))
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()
    tfs = [torch.from_numpy(t).pin_memory() for t in synth.tf_edit_sequence(6, 4096, 256)]
    rates = (200, 1000, 5000, 20000, 50000, 100000)
    servers = {"partitioned": ("partitioned", 1), "partitioned_4_per_session": ("partitioned", 4),
               "full_recompute": ("full", 1)}
    results, knees = {}, {}
    for name, (mode, E) in servers.items():
        rows = []
        for rate in rates:
            ex = DeviceExecutor(slots=3, mode=mode, device=dev, edits_per_session=E)
            sch = Scheduler(ex, budget, slots=3, edits_per_session=E)
            for sp in specs:
                sch.open_session(sp)
            n_req = int(min(max(50, rate * args.serve_seconds), 20000))
            wall = _open_loop(sch, n_sess, rate, n_req, tfs, rng)
            rows.append(_serve_stats(sch, wall, rate))
            for sp in specs:
                sch.close_session(sp.sid)
        results[name] = rows
        knees[name] = _knee(rows)
    # eviction: a budget of 40 % of the sessions' device bytes; idle sessions' maps move
    # to pinned host memory and come back (no recompute) for their next edit
    ev_budget = int(0.4 * sum(sp.device_bytes for sp in specs))
    rate = 1000
    ex = DeviceExecutor(slots=3, mode="partitioned", device=dev)
    sch = Scheduler(ex, ev_budget, slots=3, evict_idle=True)
    for sp in specs:
        sch.open_session(sp)
    ev0, re0 = sch.stats.evictions, sch.stats.readmissions
    wall = _open_loop(sch, n_sess, rate, max(50, int(rate * args.serve_seconds)), tfs, rng)
    evict = _serve_stats(sch, wall, rate)
    evict.update({"budget_gb": ev_budget / 1e9, "evictions": sch.stats.evictions - ev0,
                  "readmissions": sch.stats.readmissions - re0, "evictions_at_open": ev0})
    for e in engines:                             # every session resident again
        e.reload()
    churn = serving_churn(dev, budget, rng, tfs)
    if rank != 0:
        return
    sides = [e.grid[0] * 4 for e in engines]
    res = {"metric": "serving: TF-update latency p50/p99 (ms) and sustained edits/s",
           "value": knees["partitioned"]["p50_ms"], "unit": "ms", "n_gpus": ws,
           "higher_is_better": False, "data": "synthetic",
           "config": {"workload": f"serving: {n_sess} sessions, 12-bit volumes with sides "
                                  f"{min(sides)}..{max(sides)}, K in {{16,32,64}}, 150 GB "
                                  f"budget, Poisson arrivals, 3 streams",
                      "resident_gb": sum(sp.device_bytes for sp in specs) / 1e9},
           "knee": knees, "servers": results, "eviction_at_40pct_budget": evict,
           "churn_150gb_budget": churn}
    print(json.dumps(res))


def serving_churn(dev, budget, rng, tfs, n_sess=48, edits=40, session_rate=200.0,
                  edit_rate=200.0):
    """Sessions that come and go under the HBM budget: `n_sess` sessions open as a Poisson
    process (`session_rate` per s), each with b = 2 maps (K 128 or 256) of one of three
    12-bit volumes (sides 384, 576 and 768 voxels), built at admission on a side stream;
    each sends `edits` TF edits at `edit_rate` per s from its opening on (queued while it
    waits for admission) and leaves once they all completed.  Reports admission waits and
    edit latencies."""
    import torch
    import synth
    from paper_2407_21552_gb300 import DM_U16, _abi as A
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    from paper_2407_21552_gb300.serving import DeviceExecutor, Scheduler, SessionSpec
    sides = (384, 576, 768)

    def session_bytes(side, K):
        """Device bytes of a session as the library sizes them (no allocation)."""
        cfg, keep = A.make_config((side, side, side), DM_U16, 2, 1, K, 4096)
        ctx = A.dm_create(cfg)
        sz = A.dm_query_sizes(ctx)
        A.dm_destroy(ctx)
        return int(sz.pdm_bytes + sz.minmax_bytes + sz.scratch_bytes + 3 * sz.out_bytes)
    base = {s: synth.volume_of("u16", (s, s, s), 3000 + s, device=dev) for s in sides}
    torch.cuda.synchronize(dev)
    ex = DeviceExecutor(slots=3, mode="partitioned", device=dev)
    sch = Scheduler(ex, budget, slots=3)
    plan = []
    t_open = np.cumsum(rng.exponential(1.0 / session_rate, size=n_sess))
    for sid in range(n_sess):
        side = int(rng.choice(sides))
        K = int(rng.choice([128, 256]))
        nbytes = session_bytes(side, K)

        def build(stream, side=side, K=K):
            with torch.cuda.stream(stream):
                eng = PartitionedDistanceMaps((side, side, side), DM_U16, 2, 1, K, 4096,
                                              device=dev)
                eng.build_partitions(base[side], stream=stream)
                eng.release_mask()
            return eng, None
        spec = SessionSpec(100 + sid, int(nbytes), dict(build=build))
        times = t_open[sid] + np.arange(edits) / edit_rate
        plan.append((spec, times))
    events = sorted((t, i, k) for i, (_, times) in enumerate(plan) for k, t in enumerate(times))
    opened, finished = set(), 0
    fin = {}                                              # sid -> completed edits
    seen = 0
    t0 = time.perf_counter()
    e = 0
    while e < len(events) or sch.has_work() or finished < n_sess:
        now = time.perf_counter() - t0
        while e < len(events) and events[e][0] <= now:
            t, i, k = events[e]
            spec = plan[i][0]
            if i not in opened:
                sch.open_session(spec)
                opened.add(i)
            sch.submit(spec.sid, tfs[(7 * i + k) % len(tfs)], t_arrival=t0 + t)
            e += 1
        sch.poll()
        for r in sch.completed[seen:]:                    # sessions done with their edits
            fin[r.session] = fin.get(r.session, 0) + 1    # leave
            if fin[r.session] == edits:
                sch.close_session(r.session)
                finished += 1
        seen = len(sch.completed)
    wall = time.perf_counter() - t0
    del base
    torch.cuda.empty_cache()
    lat = np.array(sch.stats.latencies) * 1e3
    waits = np.array(sch.stats.admission_waits) * 1e3
    total = sum(sp.device_bytes for sp, _ in plan)
    return {"sessions": n_sess, "edits": int(len(lat)), "wall_s": wall,
            "budget_gb": budget / 1e9, "demand_gb": total / 1e9,
            "max_resident_gb": sch.stats.max_used / 1e9,
            "sessions_that_waited": int(sch.stats.rejected_waits),
            "admission_wait_ms": {"p50": float(np.percentile(waits, 50)),
                                  "p99": float(np.percentile(waits, 99)),
                                  "max": float(waits.max())},
            "edit_latency_ms": {"p50": float(np.percentile(lat, 50)),
                                "p99": float(np.percentile(lat, 99))},
            "sustained_edits_per_s": len(lat) / wall,
            "maps": "b = 2, K in {128, 256}, volumes 384^3 / 576^3 / 768^3 12-bit, built "
                    "at admission"}


# ---------------------------------------------------------------- partition-count sweep
def run_sweep(args, ws, rank, local):
    """The shape of the paper's Table 1 on the ct volume: for K = 4 .. 64 partitions, the
    one-time precompute, the partitioned update and the plain min/max full recompute over
    the same TF edits (CUDA events, L2 flushed before every call).  Update time grows with
    the number of maps combined; the full recompute does not depend on K."""
    import torch
    import synth
    from paper_2407_21552_gb300 import DM_U16
    from paper_2407_21552_gb300.build import build as build_lib
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps
    build_lib()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = synth.WORKLOADS["ct"]
    X, Y, Z = w["dims"]
    vol = synth.make_volume("ct", device=dev)
    stream = torch.cuda.current_stream(dev)
    flush_w = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    flush_r = torch.zeros(L2_FLUSH_BYTES // 8, dtype=torch.int64, device=dev)
    E = max(8, min(args.steps, 200))
    tfs = torch.from_numpy(np.stack(synth.tf_edit_sequence(w["seed"], w["N"], E))).to(dev)

    def timed(fn, reps):
        ts = []
        for k in range(reps + args.warmup):
            flush_w.zero_()
            flush_r.max()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn(k)
            b.record(stream)
            b.synchronize()
            if k >= args.warmup:
                ts.append(a.elapsed_time(b))
        return ts

    rows = []
    for K in (4, 8, 16, 32, 64):
        eng = PartitionedDistanceMaps((X, Y, Z), DM_U16, w["block"], w["apron"], K, w["N"],
                                      device=dev)
        out = torch.empty(eng.G, dtype=torch.uint8, device=dev)
        am = torch.zeros((E, 1), dtype=torch.int64, device=dev)
        pre = timed(lambda k: eng.build_partitions(vol), 3)
        upd = timed(lambda k: eng.update_tf(tfs[k % E], out=out,
                                            active_mask=am[k % E]), E)
        full = timed(lambda k: eng.full_recompute(tfs[k % E], out=out), E)
        nact = np.array([bin(int(x)).count("1") for x in am.cpu().numpy().view(np.uint64)[:, 0]])
        rows.append({"K": K, "precompute_ms": pct(pre, 50), "update_p50_ms": pct(upd, 50),
                     "update_p99_ms": pct(upd, 99), "full_recompute_p50_ms": pct(full, 50),
                     "speedup_p50": pct(full, 50) / pct(upd, 50),
                     "mean_active_partitions": float(nact.mean()),
                     "pdm_mib": K * eng.plane_stride / 2**20})
        eng.close()
        del eng, out
        torch.cuda.empty_cache()
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC + " (partition-count sweep)", "value": rows[3]["update_p50_ms"],
        "unit": "ms", "n_gpus": ws, "higher_is_better": False, "data": "synthetic",
        "config": {"workload": workload_name("ct", w) + "; K swept over 4..64",
                   "edits": E, "l2": "flushed before every timed call"},
        "rows": rows,
        "paper_context": "Table 1 reports, per dataset, the update time growing with the "
                         "number of partitions n and a roughly linear init time in n"}))


# --------------------------------------------------------------------- render workload
def run_render(args, ws, rank, local):
    """Frame times of the ray caster at 2160^2 (§4.1) on the CT volume, camera circling the
    vertical axis, early ray termination at 0.98: no skipping, and skipping with the exact
    distance map D, the min/max D and the partitioned D' (K = 32), as in Figs. 3-4."""
    import ctypes
    import torch
    import synth
    from paper_2407_21552_gb300 import DM_U16, DM_OCC_EXACT, _abi as A
    from paper_2407_21552_gb300.build import build as build_lib
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps

    build_lib()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = synth.WORKLOADS["ct"]
    dims = w["dims"]
    vol = synth.make_volume("ct", device=dev)
    eng = PartitionedDistanceMaps(dims, DM_U16, 4, 1, w["K"], w["N"], device=dev)
    eng.build_partitions(vol)
    ex = PartitionedDistanceMaps(dims, DM_U16, 4, 1, w["K"], w["N"], occ_mode=DM_OCC_EXACT,
                                 device=dev, with_minmax=False)
    tfs = synth.tf_edit_sequence(w["seed"], w["N"], 4)
    W = H = 2160
    img = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    ns = torch.empty((H, W), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp_ = ctypes.c_void_p(stream.cuda_stream)
    rows = {}
    for ti, tf_np in enumerate(tfs):
        tf = torch.from_numpy(tf_np).to(dev)
        maps = {"no_ess": None, "D_exact": ex.full_recompute(tf, volume=vol),
                "D_minmax": eng.full_recompute(tf), "D_partitioned": eng.update_tf(tf)}
        for name, m in maps.items():
            ts, smp = [], []
            for k in range(8):
                cam = A.orbit_camera(dims, 2 * np.pi * k / 8, W, H, step=0.5, ert=0.98)
                for _ in range(2 if k == 0 else 1):        # one warm-up frame
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    A.dm_render(vol.data_ptr(), DM_U16, dims, 4,
                                m.data_ptr() if m is not None else None, tf.data_ptr(), w["N"],
                                cam, img.data_ptr(), ns.data_ptr(), sp_)
                    b.record(stream)
                    b.synchronize()
                ts.append(a.elapsed_time(b))
                smp.append(float(ns.float().mean()))
            rows.setdefault(name, []).append((float(np.mean(ts)), float(np.mean(smp))))
    if rank != 0:
        return
    res = {"metric": "frame time (ms) at 2160^2 with and without empty-space skipping",
           "unit": "ms", "n_gpus": ws, "data": "synthetic", "higher_is_better": False,
           "config": {"workload": "ct volume 512^3 12-bit, b=4 apron=1, K=32; 4 TFs x 8 "
                                  "camera angles; ERT 0.98; step 0.5 voxel"},
           "value": float(np.mean([r[0] for r in rows["D_partitioned"]])),
           "frames": {k: {"mean_ms": float(np.mean([r[0] for r in v])),
                          "per_tf_ms": [r[0] for r in v],
                          "mean_samples_per_ray": float(np.mean([r[1] for r in v]))}
                      for k, v in rows.items()}}
    print(json.dumps(res))


# --------------------------------------------------------------------- reference arm
def run_reference(args, ws, rank):
    if rank != 0:
        return
    import synth
    import oracle
    oracle.build()
    if args.workload not in synth.WORKLOADS:      # batch / serving / render / sweep: ct
        args.workload = "ct"
    w = synth.WORKLOADS[args.workload]
    edits = synth.tf_edit_sequence(w["seed"], w["N"], w["edits"])
    sub, scale = oracle_slab(args.workload, w)
    zs, Y, X = sub.shape
    pdm = oracle.build_partitions(sub, w["block"], w["apron"], w["N"], w["K"])[1]
    del sub
    # the steps walk the workload's edit sequence with an even stride
    stride = max(1, len(edits) // max(1, args.steps))
    for k in range(args.warmup):
        oracle.update_tf(pdm, edits[(k * stride + stride // 2) % len(edits)])
    lat = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.update_tf(pdm, edits[(k * stride) % len(edits)])
        lat.append((time.perf_counter() - t0) * 1e3 * scale)
    v = pct(lat, 50)
    s = {"scale": scale}
    res = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(lat)),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
           "data": "synthetic",
           "config": {"workload": workload_name(args.workload, w)},
           "p99_ms": pct(lat, 99),
           "cpu_baseline": {"value": v, "unit": "ms", "cores": 1, "kind": "oracle",
                            "sample": f"z-slab {X}x{Y}x{zs} of the workload volume, one "
                                      f"oracle TF update per step, scaled by "
                                      f"G/G_slab = {s['scale']:.3f}"},
           "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "note": "the paper's own GLSL implementation needs a graphics stack, which is not "
                   "available here; the reference arm is the plain CPU oracle"}
    print(json.dumps(res))


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "batch":
        run_batch(args, ws, rank, local)
    elif args.workload == "serving":
        run_serving(args, ws, rank, local)
    elif args.workload == "render":
        run_render(args, ws, rank, local)
    elif args.workload == "sweep":
        run_sweep(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
