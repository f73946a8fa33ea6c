"""Autotuner for the batched update: block size and combine schedule by measurement.

For a batch of volumes it times the batched update (CUDA events on the launching stream,
L2 flushed before every rep) for each combine grid size, and picks the block
size: b = 4 (the paper's choice, §3.1) when its best schedule meets the latency target,
else b = 8, whose maps are 8x smaller but coarser for empty-space skipping.  Every timed
call goes through libdm; this module only chooses parameters.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _abi as A

CTAS_PER_SM = (4, 8, 12, 16, 24, 32)


@dataclass
class TuneResult:
    block: int
    ctas_per_sm: int
    p50_us: float
    table: dict = field(default_factory=dict)     # (block, ctas_per_sm) -> p50 us


def _flusher(device):
    w = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    r = torch.zeros(32 << 20, dtype=torch.int64, device=device)

    def flush():
        w.zero_()
        r.max()
    return flush


def time_batch(items, ctas_per_sm, reps=20, warmup=3, device="cuda"):
    """p50 microseconds of dm_update_tf_batch over `items` [(ctx, tf_ptr, out_ptr)]."""
    stream = torch.cuda.current_stream(device)
    sp = ctypes.c_void_p(stream.cuda_stream)
    flush = _flusher(device)
    items = A.PreparedBatch(items) if not isinstance(items, A.PreparedBatch) else items
    for _ in range(warmup):
        A.dm_update_tf_batch(items, ctas_per_sm, sp)
    ts = []
    for _ in range(reps):
        flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        A.dm_update_tf_batch(items, ctas_per_sm, sp)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b) * 1e3)
    return float(np.percentile(ts, 50))


def tune(build_items, target_us: float, blocks=(4, 8), reps=20, device="cuda") -> TuneResult:
    """build_items(block) -> items [(ctx, tf_ptr, out_ptr)] for that block size (the caller
    builds or reuses the partitioned maps).  Block sizes are tried finest first; the first
    whose best schedule meets `target_us` is chosen, else the fastest one seen."""
    table = {}
    chosen = None
    for b in blocks:
        items = build_items(b)
        for c in CTAS_PER_SM:
            table[(b, c)] = time_batch(items, c, reps=reps, device=device)
        t, c = min((table[(b, c)], c) for c in CTAS_PER_SM)
        if t <= target_us:
            chosen = (b, c, t)
            break
        if chosen is None or t < chosen[2]:
            chosen = (b, c, t)
    return TuneResult(block=chosen[0], ctas_per_sm=chosen[1], p50_us=chosen[2], table=table)
