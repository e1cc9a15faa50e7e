"""Autotuner of the backward accumulation (the balancing-threshold tuning of
Sec. V-A3, widened to the tier and the pixel-to-lane layout).

The paper times one gradient-kernel iteration per threshold value and keeps
the fastest, repeating every N = 2000 iterations.  Here a candidate is a full
``gsr_backward_opts`` (tier, threshold, lane layout); each is timed with CUDA
events on the launching stream after one warm-up launch, the L2 flushed
between launches, and the median kept.
"""
from __future__ import annotations

import dataclasses
import statistics

import torch

from . import gsr

L2_FLUSH_BYTES = 256 << 20   # larger than the 129 MB L2


def default_candidates(store_T=True):
    """Tier (warp, hybrid, block, cluster) x threshold x pixel-to-lane layout
    x pixels per thread (1: 8 warps per 16x16 tile, 2: 4 warps)."""
    c = []
    for ppt in (1, 2):
        for lay in (0, 1):
            c.append(("warp", 0, lay, ppt))
            for thr in (4, 8, 12, 16, 20, 24, 28, 32):
                c.append(("hybrid", thr, lay, ppt))
            for thr in (0, 4, 8, 16):
                c.append(("block", thr, lay, ppt))
            for thr in (0, 8, 16):
                c.append(("cluster", thr, lay, ppt))
    return [gsr.backward_opts(m, t, l, store_T, p) for (m, t, l, p) in c]


def opts_key(o) -> tuple:
    return (int(o.reduce_mode), int(o.threshold), int(o.lane_layout), int(o.store_T),
            max(1, int(o.pixels_per_thread)))


def opts_name(o) -> str:
    inv = {v: k for k, v in gsr.REDUCE_NAMES.items()}
    return f"{inv[int(o.reduce_mode)]}-thr{int(o.threshold)}-lay{int(o.lane_layout)}-ppt{max(1, int(o.pixels_per_thread))}" + \
        ("" if o.store_T else "-recompute")


def parse_opts_name(name: str):
    """Inverse of ``opts_name``: 'hybrid-thr16-lay1-ppt2[-recompute]'."""
    parts = name.split("-")
    mode = parts[0]
    kv = {p[:3]: int(p[3:]) for p in parts[1:] if p[:3] in ("thr", "lay", "ppt")}
    return gsr.backward_opts(mode, kv.get("thr", 0), kv.get("lay", 0), "recompute" not in parts,
                             kv.get("ppt", 1))


class L2Flusher:
    def __init__(self, device):
        self.buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def __call__(self):
        self.buf.fill_(1.0)


def time_backward(vb, bg, dL_dimage, opts, reps=5, flush=None, stream=None):
    """Median CUDA-event time (ms) of gsr_backward with ``opts``."""
    stream = stream or torch.cuda.current_stream()
    times = []
    with torch.cuda.stream(stream):
        vb.grad2d.zero_()
        vb.backward(bg, dL_dimage, opts, stream)  # warm-up
        for _ in range(reps):
            if flush:
                flush()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            vb.backward(bg, dL_dimage, opts, stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    return statistics.median(times)


@dataclasses.dataclass
class TuneResult:
    best: object
    best_ms: float
    table: dict


def tune(vb, bg, dL_dimage, candidates=None, reps=5, flush=None) -> TuneResult:
    candidates = candidates or default_candidates(vb.final_T is not None)
    table = {}
    best, best_ms = None, float("inf")
    for o in candidates:
        ms = time_backward(vb, bg, dL_dimage, o, reps, flush)
        table[opts_name(o)] = ms
        if ms < best_ms:
            best, best_ms = o, ms
    vb.grad2d.zero_()
    return TuneResult(best, best_ms, table)


class Autotuner:
    """Keeps the best options per workload key and re-tunes every
    ``period`` calls (2000 in the paper)."""

    def __init__(self, period=2000, candidates=None, reps=3):
        self.period = period
        self.candidates = candidates
        self.reps = reps
        self._best = {}
        self._calls = {}

    def opts(self, key, vb, bg, dL_dimage, flush=None):
        n = self._calls.get(key, 0)
        if key not in self._best or (self.period and n % self.period == 0 and n > 0):
            self._best[key] = tune(vb, bg, dL_dimage, self.candidates, self.reps, flush).best
        self._calls[key] = n + 1
        return self._best[key]
