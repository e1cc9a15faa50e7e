#!/usr/bin/env python
"""Benchmark of the splat-rasterizer hot path on GB300.

A step is one pass of the whole path over one view of the workload:
projection (grad2d zeroed in the same pass), tile binning and sort, forward
blend, L1 loss gradient, backward blend with per-splat gradient accumulation
(the autotuned reduction tier), and backward projection to the 3D parameters.
The unit is the splat-grad update: one of the 9 gradient values of one active
(pixel, splat) pair, i.e. 9 x P_active per step for every tier.

``--impl ours`` (default) prints one JSON line with the whole-step throughput,
the backward kernel alone for the plain-atomicAdd tier and the reduced tiers,
the roofline of the backward kernel, the CPU oracle on a bounded sample, an
end-to-end number through host buffers, and the SM clocks seen meanwhile.
``--impl reference`` times the FP64 CPU oracle on the same workload.
Multi-GPU (torchrun): independent replicas, one view per rank.
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

METRIC = "backward-raster ms/iter and splat-grad updates/s: reduced vs plain atomicAdd"
UNIT = "splat-grad updates/s"
FP32_LANES_PER_SM = 128
# Algorithmic FP32 lane operations of the backward (an FMA counts as one):
#   per examined (pixel, splat) pair: offset (2), quadratic form (7), exp (2),
#     opacity product, cap and floor tests (4), position test (2) -> 17;
#   per active pair: transmittance recovery (3), colour dot (3), dL/dalpha (3),
#     suffix update (2), colour grads (3), opacity and sigma grads (3), conic
#     grads (8), position grads (6), accumulation of 9 values (9) -> 40.
OPS_PER_EXAMINED = 17
OPS_PER_ACTIVE = 40


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)),
                    source="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling every 20 ms on a reader thread.  Each sample is
    stamped when it arrives; only samples that arrive between ``mark()``
    calls (the timed region) are summarised.  ``start`` returns once the
    first sample has arrived, so sampling is running when the timed region
    begins."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, device_index):
        self.proc = None
        self.samples = []  # (arrival time, line)
        self.window = [None, None]
        self.device_index = device_index
        self.thread = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), line))

    def start(self):
        import threading

        import torch
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms",
               str(self.PERIOD_MS)]
        try:
            p = torch.cuda.get_device_properties(self.device_index)
            bus = f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
            cmd += ["-i", bus]
        except Exception:
            pass
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t_end = time.perf_counter() + 10.0
        while not self.samples and time.perf_counter() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def mark(self):
        """First call: the timed region starts; second call: it ends."""
        self.window[0 if self.window[0] is None else 1] = time.perf_counter()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(2.0 * self.PERIOD_MS / 1e3)  # the sample taken as the region ended
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        t0, t1 = self.window
        if t0 is None or t1 is None:
            return None
        t1 += self.PERIOD_MS / 1e3
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, line in self.samples:
            if not t0 <= t <= t1:
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "period_ms": self.PERIOD_MS,
                "window_s": t1 - t0, "note": "samples arriving during the timed steps"}


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------
def make_workload(name, seed):
    from paper_2401_05345_gb300 import scenes as S
    if name == "single_view":
        scene, cam = S.single_view_workload(seed)
        desc = ("single view: 500k Gaussians from a 64-component anisotropic mixture (std 0.05-0.5), "
                "log-scales N(-4.5,0.7), SH degree 3, 1297x840, 16x16 tiles, L1 loss vs a U[0,1] target")
    elif name == "tiny":
        scene, cam = S.tiny_workload(seed)
        desc = "tiny: 1,000 Gaussians in [-1,1]^3, RGB, 128x128"
    else:
        raise SystemExit(f"unknown workload {name}")
    target = S.target_image(seed, cam.width, cam.height)
    return scene, cam, target, desc


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate_over_ranks(tot_ms, e2e_ms, units, world, device):
    """Whole-job numbers of the replicas (one view per rank, no data-path
    collective): the slowest rank's device and end-to-end times, since the
    job ends with its last rank, and the units of all ranks."""
    if world <= 1:
        return tot_ms, e2e_ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([tot_ms, e2e_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), float(u[0])


# ----------------------------------------------------------------------------
# CPU oracle on a bounded sample (band of tile rows)
# ----------------------------------------------------------------------------
class OracleSample:
    """The FP64 oracle pipeline on a bounded sample of the workload.  The
    whole-scene stages (projection, binning, backward projection) run once and
    are timed; each sample then rasterizes (forward, L1 gradient, backward) a
    band of ``rows`` tile rows (``cols`` tile columns of them, centred, if
    given) and is charged the band's share of the whole-scene stages."""

    def __init__(self, scene, cam, target, rows, cols=None):
        from oracle import oracle as O
        O.build()
        self.O, self.scene, self.cam, self.target = O, scene, cam, target
        W, H = cam.width, cam.height
        self.gx, self.gy = (W + 15) // 16, (H + 15) // 16
        self.rows = max(1, min(rows, self.gy))
        self.cols = self.gx if cols is None else max(1, min(int(cols), self.gx))
        t0 = time.perf_counter()
        self.pp = O.preprocess(scene, cam)
        self.keys, self.pl, self.ranges = O.bin_sort(self.pp["uv"], self.pp["depth"], self.pp["radius"], W, H)
        t1 = time.perf_counter()
        O.backproject(scene, cam, np.zeros((scene.n, 9)), mags=False)
        t2 = time.perf_counter()
        self.t_global = t2 - t0

    def run(self, band_index=0):
        O, pp, cam = self.O, self.pp, self.cam
        W, H = cam.width, cam.height
        r0 = (self.gy // 2 - self.rows // 2 + band_index) % max(1, self.gy - self.rows + 1)
        c0 = (self.gx - self.cols) // 2
        mask = np.zeros((self.gy, self.gx), np.uint8)
        mask[r0:r0 + self.rows, c0:c0 + self.cols] = 1
        frac = self.rows * self.cols / (self.gy * self.gx)
        bg = np.zeros(3)
        t0 = time.perf_counter()
        fwd = O.render(W, H, self.ranges, self.pl, pp["uv"], pp["conic"], pp["opacity"], pp["rgb"], bg, None,
                       extras=False, tile_mask=mask.reshape(-1))
        band = np.zeros((H, W), bool)
        band[r0 * 16:min(H, (r0 + self.rows) * 16), c0 * 16:min(W, (c0 + self.cols) * 16)] = True
        dimg = np.where(band[None], np.sign(fwd["image"] - self.target), 0.0).astype(np.float32)
        out = O.render(W, H, self.ranges, self.pl, pp["uv"], pp["conic"], pp["opacity"], pp["rgb"], bg, dimg,
                       extras=False, tile_mask=mask.reshape(-1))
        t1 = time.perf_counter()
        updates = 9 * int(out["n_active"][band].sum())
        seconds = (t1 - t0) + frac * self.t_global
        part = (f"{self.rows} of {self.gy} tile rows" if self.cols == self.gx else
                f"{self.rows} x {self.cols} of {self.gy} x {self.gx} tiles")
        desc = (f"FP64 oracle, 1 thread: forward + L1 gradient + backward on {part} "
                f"per sample; projection + binning + backward projection of the whole scene "
                f"({self.t_global:.2f} s, timed once) charged at {frac:.4f} per sample")
        return updates, seconds, desc


REF_BUDGET_S = 120.0  # oracle seconds of a reference run (warm-up and timed steps)


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    scene, cam, target, desc = make_workload(args.workload, args.seed)
    vals, times = [], []
    note = ""
    smp = OracleSample(scene, cam, target, args.cpu_rows)
    # each step is a band sized so that the W + K steps take about REF_BUDGET_S
    # of oracle time: the first warm-up step measures the band's cost
    t_probe = time.perf_counter()
    smp.run(0)
    per_tile = (time.perf_counter() - t_probe) / (smp.rows * smp.cols)
    tiles = REF_BUDGET_S / max(1, args.warmup + args.steps) / per_tile
    if tiles < smp.rows * smp.cols:
        rows = max(1, min(smp.rows, int(tiles // smp.gx)))
        cols = max(1, min(smp.gx, int(tiles // rows)))
        smp.rows, smp.cols = rows, cols
    for i in range(args.warmup + args.steps):
        upd, sec, note = smp.run(i)
        if i >= args.warmup:
            vals.append(upd)
            times.append(sec)
    value = sum(vals) / sum(times)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "sample": f"{args.cpu_rows} tile rows per step"},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": note},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# the CUDA path
# ----------------------------------------------------------------------------
def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("raster.cu", "raster_common.cuh", "gsr_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2401_05345_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel_hash, opts_name, n_pairs):
    """DRAM bytes per launch of the backward from the committed ncu summary,
    if it was taken on this exact kernel source and tier; else None."""
    p = os.path.join(ROOT, "profiles", "backward_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(opts_name)
    if not e or e.get("kernel_hash") != kernel_hash:
        return None
    return float(e["dram_bytes_per_launch"])


def ingest_traffic(csv_path, single_opts=None):
    """Writes profiles/backward_traffic.json from the ncu CSV of a
    ``--profile`` run captured with
    ``--metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum -k regex:backward_kernel``.
    With ``single_opts`` (a tier name) the capture holds one launch of that
    tier, whose entry replaces the old one (the other tiers' entries stay,
    each with the source hash it was taken on); otherwise it is a
    ``--profile-tiers`` run whose last launches are
    the tier launches, one per autotune candidate in order (the cluster
    tier's own kernel does not match)."""
    import csv

    from paper_2401_05345_gb300 import autotune, gsr
    launches = {}
    with open(csv_path) as f:
        rows = [r for r in csv.reader(f) if r]
    hdr = next(i for i, r in enumerate(rows) if r[0] == "ID")
    cols = rows[hdr]
    for r in rows[hdr + 1:]:
        if len(r) != len(cols):
            continue
        d = dict(zip(cols, r))
        if "backward_kernel" not in d["Kernel Name"]:
            continue
        v = float(d["Metric Value"].replace(",", ""))
        unit = d["Metric Unit"].lower()
        scale = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "ns": 1e-3, "nsecond": 1e-3,
                 "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}.get(unit, 1.0)
        launches.setdefault(int(d["ID"]), {})[d["Metric Name"]] = v * scale
    # the cluster tier's kernel (backward_cluster_kernel) is not in the capture
    names = [single_opts] if single_opts else [
        autotune.opts_name(o) for o in autotune.default_candidates() if o.reduce_mode != gsr.REDUCE_CLUSTER]
    ids = sorted(launches)
    if len(ids) < len(names):
        raise SystemExit(f"{len(ids)} backward launches in {csv_path}, {len(names)} tiers expected")
    kh = kernel_source_hash()
    run = ("bench.py --profile --steps 1 --warmup 3, one launch of the benched tier (-s 7 -c 1)" if single_opts
           else "bench.py --profile --profile-tiers")
    path = os.path.join(ROOT, "profiles", "backward_traffic.json")
    out = {}
    if single_opts and os.path.exists(path):  # one tier recaptured: the other tiers' entries are kept
        with open(path) as f:
            out = json.load(f)
    out["kernel_hash"] = kh
    out["source"] = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                     "--clock-control none -k regex:backward_kernel (cold L2 per launch) of " + run)
    for name, i in zip(names, ids[-len(names):]):
        m = launches[i]
        rd, wr = m["dram__bytes_read.sum"], m["dram__bytes_write.sum"]
        out[name] = {"kernel_hash": kh, "dram_bytes_per_launch": rd + wr, "dram_read": rd, "dram_write": wr,
                     "ncu_us": m["gpu__time_duration.sum"]}
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {path}: {len(names)} tiers, kernel hash {kh}")
    return 0


def large_scene_autograd(dev, flush, reps=5):
    """The large differentiation workload (3M Gaussians, SH3, 1920x1080):
    one training step through GaussianModel and the autograd Function
    (forward, L1 loss in torch, backward into the raw parameters), with the
    transmittance stored between the passes or recomputed by the backward.
    Median CUDA-event time of ``reps`` steps (L2 flushed before each) and the
    peak device memory of a step."""
    import torch

    from paper_2401_05345_gb300 import autograd as AG
    from paper_2401_05345_gb300 import gsr
    from paper_2401_05345_gb300 import scenes as S
    scene, cam = S.large_workload(0)
    model = AG.GaussianModel(scene, dev)
    target = torch.from_numpy(S.target_image(0, cam.width, cam.height)).to(dev)
    out = {"workload": f"large: {scene.n} Gaussians (256-component mixture), SH degree 3, "
                       f"{cam.width}x{cam.height}, L1 loss, autograd"}
    cap = None
    for key, store_T in (("store", True), ("recompute", False)):
        settings = AG.RasterSettings(cam, (0.0, 0.0, 0.0), gsr.default_backward_opts(store_T), store_T, cap)

        def step():
            model.zero_grad(set_to_none=False)
            loss = (model(settings) - target).abs().sum()
            loss.backward()
        step()  # first step: allocations, key capacity
        torch.cuda.synchronize()
        ts = []
        for r in range(reps):
            flush()
            torch.cuda.synchronize()
            torch.cuda.reset_peak_memory_stats(dev)
            base = torch.cuda.memory_allocated(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        out[f"ms_{key}"] = statistics.median(ts)
        out[f"step_peak_mb_{key}"] = (torch.cuda.max_memory_allocated(dev) - base) / 2 ** 20
    out["per_pixel_state_mb_saved"] = 8.0 * cam.width * cam.height / 2 ** 20
    out["note"] = ("per step: projection, synchronous binning, forward, torch L1, backward, backward projection, "
                   "torch activation backward; the view buffers come from the settings' pool (allocated by the untimed first step)")
    return out


RED_PATTERNS = ((0, "distinct"), (1, "one_address_per_warp"), (2, "nine_lanes_one_record"),
                (3, "nine_per_lane_one_record"), (4, "v4_distinct"), (5, "v4_v4_scalar_per_lane_one_record"),
                (6, "nine_per_lane_own_record"))


def l2_red_sweep(dev, n_sm, stream, reps=3):
    """gsr_bench_red over its access patterns and 1, 2, 4 and 8 CTAs per SM
    (48 MB buffer: L2-resident); per pattern the best launch (median of reps)
    in floats added per second."""
    import torch

    from paper_2401_05345_gb300 import gsr
    red_buf = torch.zeros(12 * 1_000_000, dtype=torch.float32, device=dev)
    out = {}
    for pat, name in RED_PATTERNS:
        best = None
        for per_sm in (1, 2, 4, 8):
            blocks = n_sm * per_sm
            iters = max(8, 512 // per_sm)
            gsr.gsr_bench_red(pat, blocks, 2, red_buf)
            ts = []
            for _ in range(reps):
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                adds = gsr.gsr_bench_red(pat, blocks, iters, red_buf)
                a1.record(stream)
                a1.synchronize()
                ts.append(a0.elapsed_time(a1) / 1e3)
            rate = adds / statistics.median(ts)
            if best is None or rate > best["adds_per_s"]:
                best = {"adds_per_s": rate, "ctas_per_sm": per_sm, "iters": iters}
        out[name] = best
    return out


def l2_lane_rates(dev, n_sm, stream, per_sm=8, iters=64):
    """Floats added per second by the access patterns of the accumulation
    tiers' warp steps, by active lanes a = 1..32 (8 CTAs per SM): pattern 3
    (PLAIN: 9 scalar reds per active lane into the step's record), pattern 5
    (sparse hybrid warp: two v4 reds and one scalar per active lane) and
    pattern 2 (reduced warp: one 9-lane red)."""
    import torch

    from paper_2401_05345_gb300 import gsr
    red_buf = torch.zeros(12 * 1_000_000, dtype=torch.float32, device=dev)

    def rate(pat, a):
        gsr.gsr_bench_red(pat, n_sm * per_sm, 2, red_buf, active_lanes=a)
        ts = []
        for _ in range(3):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            adds = gsr.gsr_bench_red(pat, n_sm * per_sm, iters, red_buf, active_lanes=a)
            a1.record(stream)
            a1.synchronize()
            ts.append(a0.elapsed_time(a1) / 1e3)
        return adds / statistics.median(ts)
    return {"plain": [None] + [rate(3, a) for a in range(1, 33)],
            "sparse": [None] + [rate(5, a) for a in range(1, 33)],
            "dense": rate(2, 32)}


def l2_time_model(counts, tier, threshold, lane_rates):
    """Seconds the L2 atomic units need for a backward's reds, from its
    steps by active lanes and the microbenchmark rates of the same access
    pattern; tier: 'plain', 'warp' or 'hybrid'."""
    t = 0.0
    for a, n in enumerate(counts["active_lane_hist"]):
        if a == 0 or n == 0:
            continue
        if tier == "plain":
            t += n * 9 * a / lane_rates["plain"][a]
        elif tier == "warp" or a >= threshold:
            t += n * 9 / lane_rates["dense"]
        else:
            t += n * 9 * a / lane_rates["sparse"][a]
    return t


def run_leg(argv, timeout_s):
    """Runs ``python argv`` from the repository root and returns the JSON
    object of its last output line, or {"error": ...}."""
    try:
        r = subprocess.run([sys.executable, *argv], cwd=ROOT, capture_output=True, text=True, timeout=timeout_s)
    except subprocess.TimeoutExpired:
        return {"error": f"timed out after {timeout_s} s"}
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    if r.returncode != 0 or not lines:
        tail = (r.stderr or r.stdout).strip().splitlines()[-3:]
        return {"error": f"exit {r.returncode}: " + " | ".join(tail)}
    return json.loads(lines[-1])


def run_ours(args):
    import torch

    from paper_2401_05345_gb300 import autotune, gsr, pipeline

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    gsr.lib()
    peaks = load_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count

    scene, cam, target_np, desc = make_workload(args.workload, args.seed + rank)
    bg = (0.0, 0.0, 0.0)
    sc = pipeline.SceneTensors.from_scene(scene, dev)
    grads = sc.zeros_like_params()
    target = torch.from_numpy(target_np).to(dev)
    R = pipeline.Renderer(scene.n, cam, dev)
    vb = R.vb
    flush = autotune.L2Flusher(dev)
    stream = torch.cuda.current_stream()

    # first pass (untimed): sizes, statistics of the traversal
    R.step(sc, target, bg, grads)
    torch.cuda.synchronize()

    # plain atomicAdd vs reduced tiers, backward kernel alone (untimed for the step)
    if args.profile:
        best = autotune.parse_opts_name(args.opts)
        tune_table, t_plain = {}, None
    else:
        tr = autotune.tune(vb, bg, R.dimg, reps=3, flush=flush)
        best = tr.best
        tune_table = tr.table
    R.opts = best
    best_name = autotune.opts_name(best)
    hist = torch.zeros(38, dtype=torch.int64, device=dev)
    gsr.gsr_backward_stats(vb.W, vb.H, 16, 16, vb.tile_ranges, vb.point_list, vb.splat2d, vb.n_contrib, hist,
                           int(best.lane_layout))
    h = hist.cpu().numpy().astype(np.int64)
    p_active, p_exam, warp_steps = int(h[33]), int(h[34]), int(h[35])
    culled_in, culled_in_idle = int(h[36]), int(h[37])
    units = 9 * p_active

    def step_once(on_backward=None):
        # one view per step: the 3D gradients are written, not accumulated;
        # binning does not wait for its key count (checked after the steps)
        R.step(sc, target, bg, grads, on_backward=on_backward, accumulate=False, sync_bin=False)

    for _ in range(args.warmup):
        step_once()
    torch.cuda.synchronize()

    # the step as one CUDA graph (pipeline.StepGraph); the backward is timed
    # by external events recorded inside the graph on every replay.  Without
    # external events (or with --stream-launches) the steps are launched
    # kernel by kernel.
    graph, gev = None, None
    if not args.stream_launches:
        try:
            gev = (torch.cuda.Event(enable_timing=True, external=True),
                   torch.cuda.Event(enable_timing=True, external=True))
        except TypeError:
            gev = None
    if gev is not None:
        graph = pipeline.StepGraph(R, sc, target, bg, grads, accumulate=False, backward_events=gev)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()

    # timed region: K steps, L2 flushed (untimed) before each
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if not args.profile:
        clocks.start()
    clocks.mark()
    wall0 = time.perf_counter()
    graph_bwd_ms = []
    for k in range(args.steps):
        flush()
        e0, e1, b0, b1 = ev[k]
        e0.record(stream)
        if graph is not None:
            graph.replay()
            e1.record(stream)
            e1.synchronize()  # the graph's backward events are re-recorded by the next replay
            graph_bwd_ms.append(gev[0].elapsed_time(gev[1]))
        else:
            step_once(lambda begin, b0=b0, b1=b1: (b0 if begin else b1).record(stream))
            e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks.mark()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if not args.profile else None
    if not vb.check_bin():  # the key buffers come from the first (synchronous) pass
        raise SystemExit("binning capacity changed between steps")
    step_ms = [e0.elapsed_time(e1) for (e0, e1, _, _) in ev]
    bwd_ms = graph_bwd_ms if graph is not None else [b0.elapsed_time(b1) for (_, _, b0, b1) in ev]
    tot_ms = sum(step_ms)
    if args.profile:
        tiers = []
        if args.profile_tiers:
            # one backward launch per autotune candidate, in this order, for a
            # per-tier DRAM traffic capture
            for o in autotune.default_candidates():
                vb.backward(bg, R.dimg, o)
                tiers.append(autotune.opts_name(o))
            torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_run": True, "ms_per_step": tot_ms / args.steps,
                              "backward_ms": statistics.mean(bwd_ms), "opts": best_name,
                              "kernel_hash": kernel_source_hash(),
                              "tier_order": tiers}), flush=True)
        return 0

    # backward kernel alone: plain atomicAdd vs the reduced tiers
    reps = 10
    lay, ppt = int(best.lane_layout), max(1, int(best.pixels_per_thread))
    t_plain = autotune.time_backward(vb, bg, R.dimg, gsr.backward_opts("plain", 0, lay), reps, flush)
    t_warp = autotune.time_backward(vb, bg, R.dimg, gsr.backward_opts("warp", 0, lay, True, ppt), reps, flush)
    t_best = autotune.time_backward(vb, bg, R.dimg, best, reps, flush)
    t_block = autotune.time_backward(vb, bg, R.dimg, gsr.backward_opts("block", 0, lay, True, ppt), reps, flush)
    thr_c = int(best.threshold) if int(best.reduce_mode) in (gsr.REDUCE_HYBRID, gsr.REDUCE_CLUSTER) else 12
    t_cluster = autotune.time_backward(vb, bg, R.dimg, gsr.backward_opts("cluster", thr_c, lay, True, ppt), reps,
                                       flush)
    t_recompute = autotune.time_backward(
        vb, bg, R.dimg, gsr.backward_opts(int(best.reduce_mode), int(best.threshold), lay, False, ppt), reps, flush)
    # the reduction alone: the best tier's mode and threshold at the plain
    # tier's one pixel per thread (same lane layout, no block masks)
    best_ppt1 = gsr.backward_opts(int(best.reduce_mode), int(best.threshold), lay, True, 1)
    t_best_ppt1 = autotune.time_backward(vb, bg, R.dimg, best_ppt1, reps, flush)
    # global red traffic of the plain and the best tier (exact counts of the
    # same traversal)
    rc_plain = vb.red_counts(gsr.backward_opts("plain", 0, lay))
    rc_best = (vb.red_counts(best) if int(best.reduce_mode) in (gsr.REDUCE_PLAIN, gsr.REDUCE_WARP, gsr.REDUCE_HYBRID)
               else None)
    # deterministic tier (no float atomics): backward + per-Gaussian reduction
    det_ts = []
    det_opts = gsr.backward_opts("warp", 0, lay, True, ppt)
    vb.backward_deterministic(bg, R.dimg, det_opts)
    for _ in range(reps):
        flush()
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        vb.backward_deterministic(bg, R.dimg, det_opts)
        d1.record(stream)
        d1.synchronize()
        det_ts.append(d0.elapsed_time(d1))
    t_det = statistics.median(det_ts)
    # binning: the hand-written sorts against the same binning through CUB
    def time_bin(library):
        sb = gsr.gsr_bin_scratch_bytes(vb.n, vb.W, vb.H, 16, 16, vb.key_capacity, library=library)
        scr = torch.empty(sb, dtype=torch.uint8, device=dev)
        ts = []
        for r in range(reps + 1):
            flush()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            gsr.gsr_bin_sort(vb.n, vb.W, vb.H, 16, 16, vb.splat2d, vb.radius, vb.key_capacity, scr, vb.point_list,
                             vb.tile_ranges, None, stream, library=library)
            a1.record(stream)
            a1.synchronize()
            if r:
                ts.append(a0.elapsed_time(a1))
        return statistics.median(ts)
    t_bin_lib = time_bin(True)
    t_bin_own = time_bin(False)
    sweep = {}
    for thr in (4, 8, 12, 16, 20, 24, 28, 32):
        sweep[str(thr)] = autotune.time_backward(
            vb, bg, R.dimg, gsr.backward_opts("hybrid", thr, lay, True, ppt), 5, flush)

    large = large_scene_autograd(dev, flush) if args.workload == "single_view" else None
    # the batched persistent launch (4 scenes, 32 views) and the serving loop
    # (16 concurrent scene-fitting jobs), each in a process of its own on this
    # GPU after the timed steps (a fresh allocator and context per workload)
    batched_res, serving_res = None, None
    if args.workload == "single_view" and world == 1:
        if not args.no_batched:
            batched_res = run_leg(["-m", "paper_2401_05345_gb300.batched"], 600)
        if not args.no_serving:
            serving_res = run_leg(["-m", "paper_2401_05345_gb300.serving", "--steps", str(args.serving_steps)], 900)

    # L2 atomic (red) throughput, the roofline of the atomic accumulation:
    # every access pattern at 1-8 CTAs of 256 threads per SM; the peak is
    # the best of all of them
    red = l2_red_sweep(dev, n_sm, stream)
    red_peak_name, red_peak = max(((k, v["adds_per_s"]) for k, v in red.items()), key=lambda kv: kv[1])
    lane_rates = l2_lane_rates(dev, n_sm, stream)
    inv_modes = {v: k for k, v in gsr.REDUCE_NAMES.items()}
    t_l2_plain = l2_time_model(rc_plain, "plain", 0, lane_rates)
    t_l2_best = (l2_time_model(rc_best, inv_modes[int(best.reduce_mode)], int(best.threshold), lane_rates)
                 if rc_best else None)

    # divergent-destination accumulation (Sec. V-A1): plain atomics vs the
    # serialized warp reduction (SW-S) vs the sorted segmented reduction
    scat = {}
    rng = np.random.default_rng(5)
    n_items, rows = 1 << 22, 500_000
    vals_t = torch.from_numpy(rng.normal(size=(n_items, 9)).astype(np.float32)).to(dev)
    out_t = torch.zeros((rows, 12), device=dev)
    for distinct in (1, 2, 4, 8, 32):
        pools = rng.integers(0, rows, size=(n_items // 32, distinct))
        pick = rng.integers(0, distinct, size=(n_items // 32, 32))
        idx_np = np.take_along_axis(pools, pick, axis=1).reshape(-1).astype(np.int32)
        idx_t = torch.from_numpy(idx_np).to(dev)
        row = {}
        for name, m, thr in (("plain", 0, 0), ("serial_thr2", 1, 2), ("serial_thr8", 1, 8), ("sorted", 2, 0)):
            ts = []
            for r in range(4):
                flush()
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                gsr.gsr_scatter_add9(n_items, idx_t, vals_t, out_t, 12, m, thr)
                a1.record(stream)
                a1.synchronize()
                if r:
                    ts.append(a0.elapsed_time(a1))
            row[name] = statistics.median(ts)
        scat[str(distinct)] = row

    # cube-map texture workload (environment-map learning, Sec. VI): forward
    # sample and the texture-gradient accumulation tiers, L2 flushed before
    # each; two mip levels of the cube map (moderate and heavy contention)
    from paper_2401_05345_gb300 import scenes as S
    tex_results = {}
    for TR in (128, 32):
        dirs_np, tex_np, dlt_np = S.cubemap_workload(0, R=TR)
        TH, TW = dirs_np.shape[:2]
        dirs_t = torch.from_numpy(dirs_np).to(dev)
        tex_t = torch.from_numpy(tex_np).to(dev)
        dlt_t = torch.from_numpy(dlt_np).to(dev)
        tout = torch.zeros((TH, TW, 3), device=dev)
        tgrad = torch.zeros((6, TR, TR, 4), device=dev)
        n_tex_px = int((np.abs(dirs_np).max(-1) > 0).sum())

        def time_tex(fn, r=5, tgrad=tgrad):
            ts = []
            for i in range(r + 1):
                tgrad.zero_()
                flush()
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                fn()
                a1.record(stream)
                a1.synchronize()
                if i:
                    ts.append(a0.elapsed_time(a1))
            return statistics.median(ts)
        tex_ms = {"forward": time_tex(lambda: gsr.gsr_cube_forward(TW, TH, dirs_t, TR, tex_t, tout))}
        for name, thr in (("plain", 0), ("plain_v4", 0), ("serial", 0), ("serial", 2), ("serial", 8),
                          ("sorted", 0), ("block", 0)):
            tex_ms[f"backward_{name}_thr{thr}"] = time_tex(
                lambda name=name, thr=thr: gsr.gsr_cube_backward(TW, TH, dirs_t, dlt_t, TR, tgrad, name, thr))
        tex_best = min((v, k) for k, v in tex_ms.items() if k.startswith("backward"))
        tex_results[f"R{TR}"] = {
            "workload": f"mirror sphere {TW}x{TH}, {n_tex_px} sampled pixels, cube map 6x{TR}x{TR} (RGB + pad), "
                        f"{4 * n_tex_px / (6 * TR * TR):.1f} taps per texel",
            "ms": tex_ms, "best": tex_best[1],
            "updates_per_s_plain": 12 * n_tex_px / (tex_ms["backward_plain_thr0"] / 1e3),
            "updates_per_s_best": 12 * n_tex_px / (tex_best[0] / 1e3),
            "speedup_best_vs_plain": tex_ms["backward_plain_thr0"] / tex_best[0],
            "plain_frac_of_l2_red_peak": (12 * n_tex_px / (tex_ms["backward_plain_thr0"] / 1e3)) / red_peak}

    # end to end through the public API with host buffers.  A training step's
    # input is its target image (the scene is model state that stays on the
    # device, like a network's weights) and its result the loss: every step
    # copies the target from pinned host memory, runs, and reads the loss
    # back.  Second reading: the whole scene uploaded again every step too.
    loss_host = torch.zeros(1, dtype=torch.float32).pin_memory()
    target_host = target.cpu().pin_memory()
    scene_host = [t.detach().cpu().pin_memory() for t in sc.tensors()]

    # the step graphs are captured again here: the measurements above may have
    # regrown the view's buffers
    e2e_graph = pipeline.StepGraph(R, sc, target, bg, grads, accumulate=False) if graph is not None else None
    e2e_pipe = pipeline.StepPipeline(R, sc, bg, grads) if graph is not None else None

    def e2e_pipelined():
        # two steps in flight: the upload of step k+1 overlaps the kernels of
        # step k; every step's loss is read back (one step later)
        for _ in range(2):
            e2e_pipe.result(e2e_pipe.submit(target_host))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prev = None
        for k in range(args.steps):
            h = e2e_pipe.submit(target_host)
            if prev is not None:
                e2e_pipe.result(prev)
            prev = h
        e2e_pipe.result(prev)
        return [1e3 * (time.perf_counter() - t0) / args.steps] * args.steps

    def e2e_run(with_scene, pipelined=True):
        if not with_scene and pipelined and e2e_pipe is not None:
            return e2e_pipelined()
        ms = []
        torch.cuda.synchronize()
        for k in range(args.steps):
            t0 = time.perf_counter()
            if with_scene:
                for d, hsrc in zip(sc.tensors(), scene_host):
                    d.copy_(hsrc, non_blocking=True)
            target.copy_(target_host, non_blocking=True)
            if e2e_graph is not None:
                e2e_graph.replay()
            else:
                step_once()
            loss_host.copy_(R.loss, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            ms.append(1e3 * (time.perf_counter() - t0))
        return ms
    e2e_ms = e2e_run(False)
    e2e_seq_ms = e2e_run(False, pipelined=False)
    e2e_scene_ms = e2e_run(True)
    if not vb.check_bin():
        raise SystemExit("binning capacity changed between steps")
    h2d = target_host.numel() * target_host.element_size()
    h2d_scene = h2d + sum(t.numel() * t.element_size() for t in scene_host)

    # aggregate over ranks
    import torch.distributed as dist
    tot_ms, e2e_tot, units_all = aggregate_over_ranks(tot_ms, sum(e2e_ms), units * args.steps, world, dev)
    value = units_all / (tot_ms / 1e3)
    e2e_value = units_all / (e2e_tot / 1e3)

    # roofline of the dominant kernel (the reduced backward): FP32 ALU issue
    bwd_avg_s = statistics.mean(bwd_ms) / 1e3
    ops = OPS_PER_EXAMINED * p_exam + OPS_PER_ACTIVE * p_active
    peak_ops = n_sm * FP32_LANES_PER_SM * peaks["sm_max_mhz"] * 1e6
    achieved = ops / bwd_avg_s
    # the same with only the pairs the warps evaluate: (warp, splat) steps
    # that pass the per-warp cull, 32 lanes x pixels per thread each
    exec_pairs = rc_best["warp_steps"] * 32 * ppt if rc_best else None
    ops_exec = OPS_PER_EXAMINED * exec_pairs + OPS_PER_ACTIVE * p_active if exec_pairs else None
    traffic = traffic_from_profile(kernel_source_hash(), best_name, p_active)
    # algorithmic bytes of one backward: 4 B id + 36 B attributes per list
    # entry, 12 B dL/dimage + 4 B final_T + 4 B n_contrib per pixel, one read
    # and one write of the 36 B gradient record per visible splat
    n_vis = int((vb.radius[:scene.n] > 0).sum().item())
    alg_bytes = 40.0 * vb.n_keys + 20.0 * vb.W * vb.H + 72.0 * n_vis
    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            smp = OracleSample(scene, cam, target_np, args.cpu_rows)
            upd, sec = 0, 0.0
            for i in range(args.cpu_samples):
                u, t_, note = smp.run(i)
                upd, sec = upd + u, sec + t_
            cpu = {"value": upd / sec, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": note}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "ms_per_step_median": statistics.median(step_ms),
            "ms_per_step_p90": float(np.percentile(step_ms, 90)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded generator standing in for the paper's captured scenes)",
            "config": {"workload": desc, "parallelism": f"replicas x{world}",
                       "l2": "flushed before every timed step (256 MiB write, outside the step events)",
                       "backward_opts": best_name, "bg": list(bg),
                       "launch": "one CUDA graph per step (pipeline.StepGraph)" if graph is not None
                                 else "kernel by kernel on one stream"},
            "roofline": {"bound": "alu", "kernel": f"backward_kernel ({best_name})",
                         "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "T fp32-ops/s",
                         "frac": achieved / peak_ops, "traffic": traffic,
                         "peak_source": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                        f"{peaks['sm_max_mhz']:.0f} MHz ({peaks['source']} max SM clock)",
                         "ops_per_launch": ops, "launch_ms": bwd_avg_s * 1e3,
                         "frac_executed_pairs": (ops_exec / bwd_avg_s / peak_ops) if ops_exec else None,
                         "executed_pairs": exec_pairs,
                         "note": "frac counts 17 ops for every examined pair (P_examined, up to each pixel's "
                                 "last contributor); frac_executed_pairs only for the pairs of the (warp, splat) "
                                 "steps that pass the per-warp cull"},
            "backward_raster": {
                "ms_plain_atomicAdd": t_plain, "ms_warp": t_warp, "ms_block": t_block,
                "ms_cluster_dsmem": t_cluster, "cluster_threshold": thr_c,
                "ms_best": t_best, "best": best_name, "ms_best_recompute_T": t_recompute,
                "ms_deterministic_no_atomics": t_det,
                "speedup_best_vs_plain": t_plain / t_best,
                "ms_best_mode_one_pixel_per_thread": t_best_ppt1,
                "speedup_reduction_alone_vs_plain": t_plain / t_best_ppt1,
                "speedup_note": "speedup_best_vs_plain: plain (1 px/thread) against the autotuned tier (its "
                                "pixels per thread and the forward's block masks); speedup_reduction_alone: "
                                "the best tier's mode and threshold at 1 px/thread and the same lane layout",
                "updates_per_s_plain": units / (t_plain / 1e3),
                "updates_per_s_best": units / (t_best / 1e3),
                "hybrid_threshold_sweep_ms": sweep, "autotune_ms": tune_table,
                "l2_atomic_roofline": {
                    "peak_adds_per_s": red_peak,
                    "peak_source": f"gsr_bench_red, best of {len(RED_PATTERNS)} access patterns x 1-8 CTAs per SM "
                                   f"on the same GPU ({red_peak_name})",
                    "model": "frac = (seconds the L2 atomic units need for the launch's reds: its warp steps by "
                             "active lanes, each at the gsr_bench_red rate of the same access pattern with that "
                             "many lanes) / (the launch's measured time); frac_of_peak_adds = achieved adds/s / "
                             "peak_adds_per_s",
                    "plain": {"adds": rc_plain["adds"], "lane_reds": rc_plain["lane_reds"],
                              "achieved_adds_per_s": rc_plain["adds"] / (t_plain / 1e3),
                              "l2_time_ms": t_l2_plain * 1e3, "frac": t_l2_plain / (t_plain / 1e3),
                              "frac_of_peak_adds": rc_plain["adds"] / (t_plain / 1e3) / red_peak},
                    "best": ({"tier": best_name, "adds": rc_best["adds"], "lane_reds": rc_best["lane_reds"],
                              "red_instructions": rc_best["red_instructions"],
                              "red_v4_instructions": rc_best["red_v4_instructions"],
                              "achieved_adds_per_s": rc_best["adds"] / (t_best / 1e3),
                              "l2_time_ms": t_l2_best * 1e3, "frac": t_l2_best / (t_best / 1e3),
                              "frac_of_peak_adds": rc_best["adds"] / (t_best / 1e3) / red_peak,
                              "adds_vs_plain": rc_best["adds"] / rc_plain["adds"]} if rc_best else None),
                    "lane_rates_adds_per_s": {"plain_9_per_lane_one_record": lane_rates["plain"][1:],
                                              "sparse_v4_v4_scalar_one_record": lane_rates["sparse"][1:],
                                              "dense_9_lane_red": lane_rates["dense"]}},
                "algorithmic_bytes_best": alg_bytes,
                "hbm_gbs_best": alg_bytes / (t_best * 1e-3) / 1e9,
            },
            "binning_ms": {"hand_written_sorts": t_bin_own, "cub_radix_sorts": t_bin_lib,
                           "note": "same outputs; each includes its one host sync for the key count"},
            "texture_gradient": tex_results,
            "l2_red_adds_per_s": red,
            "traffic_counts_red": {"plain": rc_plain, "best": rc_best},
            "differentiation_large": large,
            "batched": batched_res,
            "serving": serving_res,
            "divergent_accumulation_ms": {"items": n_items, "records": rows,
                                          "by_distinct_destinations_per_warp": scat},
            "traffic_counts": {"P_active": p_active, "P_examined": p_exam, "P_ts": vb.n_keys,
                               "warp_steps": warp_steps, "warp_steps_after_cull": culled_in,
                               "warp_steps_after_cull_without_active_lane": culled_in_idle,
                               "active_lane_hist": h[:33].tolist()},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4,
                    "ms_per_step": e2e_tot / args.steps,
                    "inputs": "target image per step (scene parameters are device-resident model state)",
                    "pipelining": "two steps in flight (pipeline.StepPipeline): the target upload of a step overlaps "
                                  "the previous step's kernels; each step's loss is read back"
                                  if e2e_pipe is not None else "none"},
            "e2e_sequential": {"value": units * args.steps / (sum(e2e_seq_ms) / 1e3), "unit": UNIT,
                               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4,
                               "ms_per_step": sum(e2e_seq_ms) / args.steps,
                               "inputs": "as e2e, one step at a time: upload, step, loss read, wait"},
            "e2e_scene_upload": {"value": units * args.steps / (sum(e2e_scene_ms) / 1e3), "unit": UNIT,
                                 "h2d_bytes_per_step": h2d_scene, "d2h_bytes_per_step": 4,
                                 "ms_per_step": sum(e2e_scene_ms) / args.steps,
                                 "inputs": "all scene parameters and the target image uploaded every step"},
            "clocks": clk,
            "gpu_launches": args.steps * LAUNCHES_PER_STEP,
            "wall_s_timed_region": wall,
            "peaks": peaks,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# Kernels of libgsr launched per step: preprocess; binning (depth keys, three
# column scans and three radix scatter passes, the last also writing the tile
# rectangles; entry prefixes, block x tile counts with the slice starts,
# column scan + ranges + tile order, placement); forward with the L1 loss in
# its epilogue, backward, backward projection.
LAUNCHES_PER_STEP = 15


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="single_view")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-rows", type=int, default=2, help="tile rows of the oracle sample")
    ap.add_argument("--cpu-samples", type=int, default=4, help="oracle samples for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true", help="only warm-up + timed steps (for ncu)")
    ap.add_argument("--stream-launches", action="store_true",
                    help="launch the steps kernel by kernel instead of replaying one CUDA graph")
    ap.add_argument("--opts", default="hybrid-thr24-lay1-ppt2", help="backward tier of a --profile run")
    ap.add_argument("--profile-tiers", action="store_true",
                    help="--profile: then one backward launch per autotune candidate")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched persistent-launch leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--serving-steps", type=int, default=125, help="steps per job of the serving leg")
    ap.add_argument("--ingest-traffic", metavar="CSV",
                    help="write profiles/backward_traffic.json from the ncu CSV of a --profile-tiers capture")
    args = ap.parse_args()
    if args.ingest_traffic:
        return ingest_traffic(args.ingest_traffic, None if args.profile_tiers else args.opts)
    if args.warmup < 3 and not args.profile:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
