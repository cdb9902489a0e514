"""Tile-shape autotuning for the 2-D FP32 kernels.

The tiled kernels are compiled for five tile configurations (1: 32x32, 2: 32x16, 3: 64x16
targets per CTA, 4: 32x16 with registers budgeted for 4 CTAs per SM, 5: 32x32 on a persistent CTA
per SM that stages its next tiles while it computes).  Which one is fastest
depends on the grid sizes (ragged edge tiles, number of CTAs against 152 SMs) and on how far the
flow moves nodes (window size).  The tuner times each
configuration on the caller's own workload through the public API (CUDA events, after warm-up)
and returns the fastest.  Every configuration computes the same result.
"""
from __future__ import annotations

import statistics
from typing import Callable, Dict, Sequence

import torch

from . import sl

CONFIGS = (1, 2, 3, 4, 5)


def _time(fn: Callable[[], None], repeats: int, warmup: int, stream) -> float:
    for _ in range(warmup):
        fn()
    times = []
    for _ in range(repeats):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        times.append((a, b))
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in times)


def tune_grid(workload, steps_per_trial: int = 2, repeats: int = 5, warmup: int = 2,
              configs: Sequence[int] = CONFIGS) -> Dict:
    """Best tile configuration for sl_step on one 2-D FP32 grid of this workload."""
    stream = torch.cuda.current_stream()
    fields = torch.tensor(workload.fields, dtype=torch.float32, device="cuda")
    timings = {}
    for cfg in configs:
        g = sl.grid_for(workload, sl.SL_F32, tile_config=cfg)
        f = fields.clone()
        s = torch.empty_like(f)
        timings[cfg] = _time(lambda: g.step(f, s, 0.0, workload.dt, steps_per_trial), repeats, warmup, stream)
        g.close()
    best = min(timings, key=timings.get)
    return {"best": best, "ms_per_call": timings}


def tune_batch(workloads: Sequence, steps_per_trial: int = 2, repeats: int = 3, warmup: int = 1,
               configs: Sequence[int] = CONFIGS, use_graph: bool = False) -> Dict:
    """Best tile configuration for a batch of 2-D FP32 grids (sl_batch_step)."""
    stream = torch.cuda.Stream()
    timings = {}
    base = [torch.tensor(wl.fields, dtype=torch.float32, device="cuda") for wl in workloads]
    for cfg in configs:
        grids = [sl.grid_for(wl, sl.SL_F32, tile_config=cfg) for wl in workloads]
        fields = [b.clone() for b in base]
        scratch = [torch.empty_like(b) for b in base]
        batch = sl.Batch(grids, fields, scratch, [0.0] * len(workloads), [wl.dt for wl in workloads],
                         tile_config=cfg)
        with torch.cuda.stream(stream):
            timings[cfg] = _time(lambda: batch.step(steps_per_trial, use_graph=use_graph, stream=stream),
                                 repeats, warmup, stream)
        batch.close()
        for g in grids:
            g.close()
    best = min(timings, key=timings.get)
    return {"best": best, "ms_per_call": timings}
