"""Benchmark: partitioned-distance-map TF update vs the plain full recompute on one GB300.

A step is one TF edit through the whole per-edit hot path: the partitioned update (active
set from the TF, then the Eq. 1 combine of the resident PDMs) and, on the same edit, the
plain full recompute it replaces (min/max occupancy + a fresh distance transform).  The
one-time precompute (partition table, POMs, K distance transforms) runs once per volume,
as in the paper (§3.1), and is timed separately.

Rules kept: inputs (volume, PDMs, all TF edits) are resident in HBM before the timed
region; the L2 is flushed (a 256 MiB write, then a 256 MiB read, so no dirty lines remain)
before every timed call; kernels are timed
with CUDA events on the stream they run on; clocks are sampled with nvidia-smi during the
timed region.  `value` is the p50 latency of the partitioned update (ms, lower is better).
`--impl reference` times the CPU oracle (plain C) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
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
# DRAM bytes per combine launch from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by workload, with the hash of the kernel source it was
# taken on; reported as null once the source has changed.
NCU_TRAFFIC = {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["ct", "tiny", "large"], default="ct")
    ap.add_argument("--cpu-edits", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
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


def file_sha(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


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
def oracle_sample(vol_np, w, edits, n_edits, n_full=3):
    """The CPU oracle, as it stands, on a bounded sample of the workload: a z-slab of the
    volume (whole block-slices, about 1M blocks), its one-time precompute untimed, then
    `n_edits` TF updates and `n_full` min/max full recomputes timed single-threaded; times
    scale to the whole volume by G / G_slab (both are linear in G)."""
    import oracle
    b, a, N, K = w["block"], w["apron"], w["N"], w["K"]
    Z, Y, X = vol_np.shape
    gx, gy, gz = -(-X // b), -(-Y // b), -(-Z // b)
    slab_bz = max(1, min(gz, (1 << 20) // (gx * gy)))
    zs = min(Z, slab_bz * b)
    sub = np.ascontiguousarray(vol_np[:zs])
    G = gx * gy * gz
    Gs = gx * gy * (-(-zs // b))
    scale = G / Gs
    t0 = time.perf_counter()
    _, pdm, vmin, vmax = oracle.build_partitions(sub, b, a, N, K)
    pre_s = time.perf_counter() - t0
    upd = []
    for tf in edits[:n_edits]:
        t0 = time.perf_counter()
        oracle.update_tf(pdm, tf)
        upd.append((time.perf_counter() - t0) * 1e3 * scale)
    full = []
    for tf in edits[:n_full]:
        t0 = time.perf_counter()
        oracle.full_recompute_minmax(vmin, vmax, tf)
        full.append((time.perf_counter() - t0) * 1e3 * scale)
    return dict(pdm=pdm, scale=scale, slab=(X, Y, zs), pre_s=pre_s, upd=upd, full=full)


def cpu_baseline_block(s, n_edits):
    X, Y, zs = s["slab"]
    return {"value": pct(s["upd"], 50), "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": (f"z-slab {X}x{Y}x{zs} of the same volume (precompute untimed, "
                       f"{s['pre_s']:.1f} s), {n_edits} TF edits through the oracle's step 1 + "
                       f"Eq. 1, single-threaded C; per-edit times scaled by G/G_slab = "
                       f"{s['scale']:.3f}"),
            "full_recompute_p50_ms": pct(s["full"], 50),
            "nproc": os.cpu_count()}


# --------------------------------------------------------------------------- our arm
def run_ours(args, ws, rank, local):
    import torch
    import synth
    from paper_2407_21552_gb300 import DM_U8, DM_U16, dm_set_profile_events
    from paper_2407_21552_gb300.build import build as build_lib
    from paper_2407_21552_gb300.maps import PartitionedDistanceMaps

    build_lib()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = synth.WORKLOADS[args.workload]
    X, Y, Z = w["dims"]
    vol = synth.make_volume(args.workload, device=dev)
    vol_sha = synth.volume_sha256(vol) if args.workload != "large" else None
    eng = PartitionedDistanceMaps((X, Y, Z), DM_U8 if w["dtype"] == "u8" else DM_U16,
                                  w["block"], w["apron"], w["K"], w["N"], device=dev)
    G = eng.G
    V = X * Y * Z
    s_bytes = 1 if w["dtype"] == "u8" else 2
    stream = torch.cuda.current_stream(dev)
    flush_w = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    flush_r = torch.zeros(L2_FLUSH_BYTES // 8, dtype=torch.int64, device=dev)

    def flush():
        """Evict the L2: write 256 MiB, then read 256 MiB so that no dirty line is left
        to be written back inside the next timed call."""
        flush_w.zero_()
        flush_r.max()

    # ---- one-time precompute, timed on its own (3 runs, median)
    pre = []
    for _ in range(3):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        eng.build_partitions(vol)
        e1.record(stream)
        e1.synchronize()
        pre.append(e0.elapsed_time(e1))
    eng.sync()

    edits = synth.tf_edit_sequence(w["seed"], w["N"], w["edits"])
    tfs = torch.from_numpy(np.stack(edits)).to(dev)                # [E, N, 4], resident
    E = tfs.shape[0]
    Wm = (w["K"] + 63) // 64
    am = torch.zeros((args.steps, Wm), dtype=torch.int64, device=dev)
    out = torch.empty(G, dtype=torch.uint8, device=dev)
    out_full = torch.empty(G, dtype=torch.uint8, device=dev)

    for k in range(args.warmup):
        tf = tfs[k % E]
        eng.update_tf(tf, out=out)
        eng.full_recompute(tf, out=out_full)
    torch.cuda.synchronize(dev)

    K = args.steps
    mk = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(K)]  # noqa: E731
    ua, ub, ca, cb, fa, fb = mk(), mk(), mk(), mk(), mk(), mk()
    region0 = torch.cuda.Event(enable_timing=True)
    region1 = torch.cuda.Event(enable_timing=True)
    for ev in ca + cb:            # torch creates the CUDA event on first record
        ev.record(stream)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(smi_gpu_id(dev))
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize(dev)
    region0.record(stream)
    for k in range(K):
        tf = tfs[k % E]
        flush()
        ua[k].record(stream)
        eng.update_tf(tf, out=out, active_mask=am[k])
        ub[k].record(stream)
        flush()
        fa[k].record(stream)
        eng.full_recompute(tf, out=out_full)
        fb[k].record(stream)
        # the same update once more with events around the combine kernel alone (kept
        # out of the timed update above: an event between its two kernels would stop the
        # combine from launching while the active-set kernel runs)
        flush()
        dm_set_profile_events(eng.ctx, ca[k].cuda_event, cb[k].cuda_event)
        eng.update_tf(tf, out=out)
        dm_set_profile_events(eng.ctx, None, None)
    region1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    clk = clocks.stop()
    region_ms = region0.elapsed_time(region1)
    upd = [ua[k].elapsed_time(ub[k]) for k in range(K)]
    comb = [ca[k].elapsed_time(cb[k]) for k in range(K)]
    full = [fa[k].elapsed_time(fb[k]) for k in range(K)]
    masks = am.cpu().numpy().view(np.uint64)
    nact = np.array([sum(bin(int(x)).count("1") for x in row) for row in masks])
    bytes_comb = (nact + 1) * G                                   # per launch, algorithmic
    achieved = float(bytes_comb.sum() / (np.sum(comb) * 1e-3)) / 1e9   # GB/s
    peak, peak_src = measured_peak()
    traffic = None
    tr = NCU_TRAFFIC.get(args.workload)
    src = os.path.join(ROOT, "paper_2407_21552_gb300", "csrc", "dm_update.cu")
    if tr and tr.get("source_sha") == file_sha(src):
        traffic = tr["bytes_per_launch"]

    # ---- end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        h_tf = torch.empty((E, w["N"], 4), dtype=torch.float32).pin_memory()
        h_tf.copy_(tfs.cpu())
        h_out = torch.empty(G, dtype=torch.uint8).pin_memory()
        for k in range(min(args.warmup, E)):
            eng.update_tf_host(h_tf[k], h_out)
        lat = []
        barrier(ws)
        for k in range(K):
            t0 = time.perf_counter()
            eng.update_tf_host(h_tf[k % E], h_out)
            lat.append((time.perf_counter() - t0) * 1e3)
        barrier(ws)
        e2e = {"value": pct(lat, 50), "unit": "ms", "p99": pct(lat, 99),
               "h2d_bytes_per_step": int(w["N"] * 16), "d2h_bytes_per_step": int(G),
               "how": "dm_update_tf_host: pinned TF -> device, step 1 + Eq. 1, D' -> pinned host, "
                      "stream sync; host wall clock per call"}

    p50u, p99u, p50f, p99f, p50c, region_max = reduce_max(
        [pct(upd, 50), pct(upd, 99), pct(full, 50), pct(full, 99), pct(comb, 50), region_ms], ws)
    if e2e is not None:
        e2e["value"] = reduce_max([e2e["value"]], ws)[0]

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        s = oracle_sample(synth.as_numpy(vol), w, edits, args.cpu_edits)
        cpu = cpu_baseline_block(s, args.cpu_edits)

    if rank != 0:
        return
    launches_per_step = 2 + 4 + 2
    res = {
        "metric": METRIC, "value": p50u, "unit": "ms", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": region_max / K, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": workload_name(args.workload, w), "volume_xyz": [X, Y, Z],
                   "grid_xyz": list(eng.grid), "G": G, "edits": E,
                   "l2": "flushed before every timed call (256 MiB device write, then a "
                         "256 MiB read)",
                   "volume_sha256": vol_sha, "parallelism": f"replicas x{ws}"},
        "step": "one TF edit: partitioned update (active set + combine) and, on the same "
                "edit, the plain min/max full recompute; then the update once more with "
                "events around the combine kernel for the roofline; ms_per_step includes "
                "all three and the three L2 flushes",
        "update": {"p50_ms": p50u, "p99_ms": p99u, "mean_ms": float(np.mean(upd)),
                   "gbs_p50": float(np.median((nact + 1) * G / (np.array(upd) * 1e-3)) / 1e9),
                   "voxels_per_s_p50": V / (p50u * 1e-3)},
        "full_recompute": {"p50_ms": p50f, "p99_ms": p99f, "mode": "min/max occupancy",
                           "voxels_per_s_p50": V / (p50f * 1e-3)},
        "speedup_vs_full_recompute_p50": p50f / p50u,
        "active_partitions": {"mean": float(nact.mean()), "min": int(nact.min()),
                              "max": int(nact.max()), "K": w["K"]},
        "precompute": {"ms": float(np.median(pre)),
                       "algorithmic_gb": (s_bytes * V + w["K"] * G) / 1e9,
                       "gbs": (s_bytes * V + w["K"] * G) / (np.median(pre) * 1e-3) / 1e9},
        "roofline": {"kernel": "k_combine (Eq. 1)", "bound": "hbm", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": float(bytes_comb.mean()),
                     "mean_launch_us": float(np.mean(comb) * 1e3)},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": K * launches_per_step,
        "clocks": clk,
        "paper_context": "paper: up to 30x faster DM update (RTX 4090, OpenGL/GLSL, Table 1); "
                         "not re-run here (no graphics stack)",
    }
    print(json.dumps(res))


# --------------------------------------------------------------------- reference arm
def run_reference(args, ws, rank):
    if rank != 0:
        return
    import torch
    import synth
    import oracle
    oracle.build()
    w = synth.WORKLOADS[args.workload]
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    vol_np = synth.as_numpy(synth.make_volume(args.workload, device=dev))
    edits = synth.tf_edit_sequence(w["seed"], w["N"], w["edits"])
    s = oracle_sample(vol_np, w, edits, 0, 0)
    for k in range(args.warmup):
        oracle.update_tf(s["pdm"], edits[k % len(edits)])
    lat = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.update_tf(s["pdm"], edits[k % len(edits)])
        lat.append((time.perf_counter() - t0) * 1e3 * s["scale"])
    X, Y, zs = s["slab"]
    v = pct(lat, 50)
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
           "note": "the paper's own GLSL implementation needs a graphics stack (unavailable on "
                   "this box); the reference arm is the plain CPU oracle"}
    print(json.dumps(res))


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
