"""Autotuner for the batched update: block size and combine schedule by measurement.

For a batch of volumes it times the batched update (CUDA events on the launching stream,
L2 flushed before every rep) for every combine schedule -- CTAs per SM (with one 4 KiB
work unit per CTA at the largest grids, several consecutive units per CTA at the smaller
ones) and plane loads per pipeline stage (4 or 8) -- and picks the block size: b = 4 (the
paper's choice, §3.1) when its best schedule meets the latency target, else b = 8, whose
maps are 8x smaller but coarser for empty-space skipping.  Every timed call goes through
libdm; this module only chooses parameters.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _abi as A

CTAS_PER_SM = (4, 8, 12, 16, 24, 32)
LOADS_PER_STAGE = (4, 8)


@dataclass
class TuneResult:
    block: int
    ctas_per_sm: int
    loads_per_stage: int
    p50_us: float
    table: dict = field(default_factory=dict)     # (block, ctas_per_sm, loads) -> p50 us

    @property
    def tuning(self):
        """The schedule as dm_update_tf_batch's tuning argument."""
        return (self.ctas_per_sm, self.loads_per_stage)


def _flusher(device):
    w = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    r = torch.zeros(32 << 20, dtype=torch.int64, device=device)

    def flush():
        w.zero_()
        r.max()
    return flush


def time_batch(items, tuning, reps=20, warmup=3, device="cuda"):
    """p50 microseconds of dm_update_tf_batch over `items` [(ctx, tf_ptr, out_ptr)] with
    `tuning` (an int: CTAs per SM, or a (CTAs per SM, loads per stage) pair)."""
    stream = torch.cuda.current_stream(device)
    sp = ctypes.c_void_p(stream.cuda_stream)
    flush = _flusher(device)
    items = A.PreparedBatch(items) if not isinstance(items, A.PreparedBatch) else items
    for _ in range(warmup):
        A.dm_update_tf_batch(items, tuning, sp)
    ts = []
    for _ in range(reps):
        flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        A.dm_update_tf_batch(items, tuning, sp)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b) * 1e3)
    return float(np.percentile(ts, 50))


def tune(build_items, target_us: float, blocks=(4, 8), reps=20, device="cuda",
         ctas_per_sm=CTAS_PER_SM, loads_per_stage=LOADS_PER_STAGE) -> TuneResult:
    """build_items(block) -> items [(ctx, tf_ptr, out_ptr)] for that block size (the caller
    builds or reuses the partitioned maps).  Block sizes are tried finest first; the first
    whose best schedule meets `target_us` is chosen, else the fastest one seen."""
    table = {}
    chosen = None
    for b in blocks:
        items = A.PreparedBatch(build_items(b))
        for c in ctas_per_sm:
            for kb in loads_per_stage:
                table[(b, c, kb)] = time_batch(items, (c, kb), reps=reps, device=device)
        t, c, kb = min((table[(b, c, kb)], c, kb) for c in ctas_per_sm for kb in loads_per_stage)
        if t <= target_us:
            chosen = (b, c, kb, t)
            break
        if chosen is None or t < chosen[3]:
            chosen = (b, c, kb, t)
    return TuneResult(block=chosen[0], ctas_per_sm=chosen[1], loads_per_stage=chosen[2],
                      p50_us=chosen[3], table=table)
