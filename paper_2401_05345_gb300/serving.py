"""Serving loop for concurrent scene-fitting jobs.

Each job fits one Gaussian scene to target views: every request is one
training step (render, L1 loss, backward, backward projection, activation
backward, Adam), the iteration of Sec. II-B (Fig. 2).  A job's parameters,
gradients, Adam moments and sort buffers stay on the device while it is
admitted.

* Admission by HBM footprint: a job is admitted (first fit, in arrival order)
  when its device footprint fits in what the budget leaves; a job larger than
  the whole budget is refused.  Its memory is released when its last step
  completes or it is cancelled, and waiting jobs are admitted then.
* Continuous batching: requests arrive over time (Poisson); whenever one of
  the ``slots`` CUDA streams is idle, the oldest ready request (its job
  admitted and not already stepping) is issued on it, so steps of different
  jobs overlap on the device and new arrivals join while others run.
* Checkpoint and readmission: with ``evict_after`` set, a new waiting job
  that does not fit and has waited that long makes the scheduler evict idle
  admitted jobs (oldest admission first, each after at least ``quantum``
  steps since its admission) when that frees enough memory.  An evicted
  job's parameters, Adam moments and Adam step count go to pinned host
  memory; it rejoins the waiting list and is restored from that checkpoint
  when it is admitted again, so its steps continue exactly where they
  stopped.
* Latency of a request = device completion time - arrival time (queueing
  included); p50 / p99 and steps/s are reported.

``Scheduler`` is pure host logic (tested on the CPU with a fake executor);
``GpuExecutor`` runs the steps through libgsr.
"""
from __future__ import annotations

import dataclasses
import heapq
import json
import math
import time

import numpy as np

# ----------------------------------------------------------------------------
# host-side scheduling
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Job:
    job_id: int
    n: int                     # Gaussians
    steps: int                 # requests this job will make
    arrival: float             # seconds
    footprint: int = 0         # device bytes while admitted
    state: str = "waiting"     # waiting | admitted | done | refused | cancelled
    done_steps: int = 0
    busy: bool = False
    payload: object = None     # executor data (scene, camera, targets)
    waiting_since: float = 0.0  # when the job last entered the waiting list
    admitted_at: float = 0.0
    steps_at_admit: int = 0
    evictions: int = 0


@dataclasses.dataclass(order=True)
class Request:
    arrival: float
    job_id: int
    step: int


@dataclasses.dataclass
class Result:
    job_id: int
    step: int
    arrival: float
    issued: float
    completed: float
    loss: float


class Scheduler:
    """Admission by footprint and continuous batching over ``slots``;
    eviction of idle admitted jobs for a waiting one (``evict_after``
    seconds of waiting, None = never; an admitted job runs ``quantum`` steps
    before it may be evicted)."""

    def __init__(self, budget_bytes: int, slots: int, evict_after=None, quantum: int = 1):
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.evict_after = evict_after
        self.quantum = max(1, int(quantum))
        self.jobs: dict[int, Job] = {}
        self.used = 0
        self.pending: list[Request] = []      # arrived, not issued (heap by arrival)
        self.waiting: list[int] = []          # job ids waiting for admission, arrival order
        self.events: list[str] = []
        self.peak_used = 0

    def add_job(self, job: Job):
        self.jobs[job.job_id] = job
        if job.footprint > self.budget:
            job.state = "refused"
            self.events.append(f"refuse {job.job_id}")
            return False
        job.waiting_since = job.arrival
        self.waiting.append(job.job_id)
        return True

    def admit(self, on_admit, now=0.0):
        """First-fit admission in arrival order (evicted jobs rejoin at the
        end of the list)."""
        still = []
        for jid in self.waiting:
            job = self.jobs[jid]
            if job.state != "waiting":
                continue
            if self.used + job.footprint <= self.budget:
                on_admit(job)
                job.state = "admitted"
                job.admitted_at = now
                job.steps_at_admit = job.done_steps
                self.used += job.footprint
                self.peak_used = max(self.peak_used, self.used)
                self.events.append(f"admit {jid}")
            else:
                still.append(jid)
        self.waiting = still

    def maybe_evict(self, now, on_evict):
        """Evicts idle admitted jobs for the first new waiting job (one that
        has not run yet) that does not fit, once it has waited
        ``evict_after`` seconds and if that frees enough memory for it.
        Evicted jobs wait for memory like any other, so two jobs never evict
        each other in turn.  Returns the evicted jobs."""
        if self.evict_after is None:
            return []
        for jid in self.waiting:
            job = self.jobs[jid]
            if job.state != "waiting" or self.used + job.footprint <= self.budget:
                continue  # admit() takes the ones that fit
            if job.done_steps or job.evictions:
                continue
            if now - job.waiting_since < self.evict_after:
                return []
            cands = sorted((j for j in self.jobs.values()
                            if j.state == "admitted" and not j.busy and j.done_steps < j.steps
                            and j.done_steps - j.steps_at_admit >= self.quantum),
                           key=lambda j: (j.admitted_at, j.job_id))
            free, chosen = self.budget - self.used, []
            for c in cands:
                if free >= job.footprint:
                    break
                chosen.append(c)
                free += c.footprint
            if free < job.footprint:
                return []
            for c in chosen:
                on_evict(c)
                c.state = "waiting"
                c.evictions += 1
                c.waiting_since = now
                self.used -= c.footprint
                self.waiting.append(c.job_id)
                self.events.append(f"evict {c.job_id}")
            return chosen
        return []

    def arrive(self, req: Request):
        job = self.jobs[req.job_id]
        if job.state in ("refused", "cancelled", "done"):
            return
        heapq.heappush(self.pending, req)

    def next_ready(self):
        """Oldest arrived request whose job is admitted and idle and whose
        step is that job's next one."""
        skipped, found = [], None
        while self.pending:
            r = heapq.heappop(self.pending)
            job = self.jobs[r.job_id]
            if job.state in ("cancelled", "refused", "done"):
                continue
            if job.state == "admitted" and not job.busy and r.step == job.done_steps:
                found = r
                break
            skipped.append(r)
        for r in skipped:
            heapq.heappush(self.pending, r)
        if found is not None:
            self.jobs[found.job_id].busy = True
        return found

    def complete(self, job_id, on_release):
        job = self.jobs[job_id]
        job.busy = False
        job.done_steps += 1
        if job.done_steps >= job.steps and job.state == "admitted":
            job.state = "done"
            self._release(job, on_release)

    def cancel(self, job_id, on_release):
        job = self.jobs[job_id]
        if job.state == "admitted" and not job.busy:
            self._release(job, on_release)
        elif job.state == "waiting":
            self.waiting = [j for j in self.waiting if j != job_id]
        job.state = "cancelled"
        self.events.append(f"cancel {job_id}")

    def _release(self, job, on_release):
        self.used -= job.footprint
        on_release(job)
        self.events.append(f"release {job.job_id}")

    def all_finished(self):
        return all(j.state in ("done", "refused", "cancelled") for j in self.jobs.values())


def poisson_requests(jobs, rate_per_job, seed):
    """Per job, step requests after its arrival with exponential gaps."""
    rng = np.random.default_rng(seed)
    reqs = []
    for j in jobs:
        t = j.arrival
        for s in range(j.steps):
            t += rng.exponential(1.0 / rate_per_job)
            reqs.append(Request(t, j.job_id, s))
    reqs.sort()
    return reqs


def percentile(xs, q):
    if not xs:
        return float("nan")
    return float(np.percentile(np.asarray(xs, np.float64), q))


def summarize(results, wall_s, requests=None):
    """Latency percentiles and throughput.  With ``requests``, also the
    time-averaged offered rate and a steady-state window: the span between
    the 10th and the 90th percentile of arrival times, with the completions
    per second inside it and the latency of the requests that arrived in it."""
    lat = [1e3 * (r.completed - r.arrival) for r in results]
    out = {"requests": len(results), "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
           "mean_ms": float(np.mean(lat)) if lat else float("nan"),
           "steps_per_s": len(results) / wall_s if wall_s > 0 else float("nan"), "wall_s": wall_s}
    if requests:
        arr = np.sort(np.asarray([q.arrival for q in requests], np.float64))
        span = arr[-1] - arr[0]
        out["offered_per_s"] = (len(arr) - 1) / span if span > 0 else float("inf")
        t_a, t_b = np.percentile(arr, 10), np.percentile(arr, 90)
        if t_b > t_a:
            done = np.asarray([r.completed for r in results], np.float64)
            lw = [x for x, r in zip(lat, results) if t_a <= r.arrival <= t_b]
            out["steady"] = {"window_s": float(t_b - t_a),
                             "completed_per_s": float(((done >= t_a) & (done <= t_b)).sum() / (t_b - t_a)),
                             "offered_per_s": float(((arr >= t_a) & (arr <= t_b)).sum() / (t_b - t_a)),
                             "p50_ms": percentile(lw, 50), "p99_ms": percentile(lw, 99)}
    return out


def serve(scheduler: Scheduler, requests, executor, cancel_at=None, poll_sleep=0.0):
    """Runs the loop until every job is finished.  ``requests`` are released
    at their arrival times (seconds from start); ``executor`` provides
    load/unload/issue/poll/now.  ``cancel_at``: {job_id: time}."""
    results = []
    inflight = {}  # slot -> (request, handle)
    free_slots = list(range(scheduler.slots))
    reqs = list(requests)
    ri = 0
    cancel_at = dict(cancel_at or {})
    t0 = executor.now()
    while True:
        now = executor.now() - t0
        while ri < len(reqs) and reqs[ri].arrival <= now:
            scheduler.arrive(reqs[ri])
            ri += 1
        for jid, tc in list(cancel_at.items()):
            if tc <= now and not scheduler.jobs[jid].busy:
                scheduler.cancel(jid, executor.unload)
                del cancel_at[jid]
        evict = getattr(executor, "evict", None)
        if evict is not None:
            scheduler.maybe_evict(now, evict)
        scheduler.admit(executor.load, now)
        while free_slots:
            r = scheduler.next_ready()
            if r is None:
                break
            slot = free_slots.pop()
            inflight[slot] = (r, executor.issue(slot, scheduler.jobs[r.job_id], r.step), now)
        for slot in list(inflight):
            r, h, issued = inflight[slot]
            done = executor.poll(h)
            if done is not None:
                completed, loss = done
                results.append(Result(r.job_id, r.step, r.arrival, issued, completed - t0, loss))
                scheduler.complete(r.job_id, executor.unload)
                del inflight[slot]
                free_slots.append(slot)
        if scheduler.all_finished() and not inflight:
            break
        if ri >= len(reqs) and not inflight and not scheduler.pending:
            break  # nothing can arrive or complete any more (e.g. a job is still waiting forever)
        if poll_sleep:
            time.sleep(poll_sleep)
    return results

# ----------------------------------------------------------------------------
# GPU executor
# ----------------------------------------------------------------------------


def job_footprint(n, sh_degree, width, height, keys_per_gaussian=16):
    """Device bytes of one admitted job: raw params, gradients and two Adam
    moments (4 x 59 floats per Gaussian at SH degree 3), activated scale and
    opacity, the view buffers (2D records, gradient records, radius, bins and
    binning scratch sized for ``keys_per_gaussian`` keys per Gaussian),
    images, loss gradient and target."""
    k = 1 if sh_degree < 0 else (sh_degree + 1) ** 2
    per = 3 + 3 + 4 + 1 + 3 * k
    params = 4 * per * 4 * n
    act = 16 * n + 16 * n
    keys = keys_per_gaussian * n
    view = 48 * n + 48 * n + 4 * n + 4 * keys + (20 * keys + 4 * n + (8 << 20))
    img = 4 * width * height * (3 * 3 + 2)
    return params + act + view + img


class _Step:
    """An issued step: phase 1 (render, loss, backward, 3D gradients) then,
    once its binning is known to have fitted, phase 2 (Adam)."""

    __slots__ = ("phase", "event", "st", "job_id", "step", "stream")

    def __init__(self, st, job_id, step, stream):
        self.phase, self.event = 1, None
        self.st, self.job_id, self.step, self.stream = st, job_id, step, stream


class GpuExecutor:
    """Runs job steps on CUDA streams through libgsr.

    The host never waits for the GPU.  A step is issued in two phases on its
    slot's stream.  Phase 1 bins asynchronously and ends with one copy of the
    loss and the binning status to pinned host memory.  ``poll`` reads them
    once phase 1 has finished.  If the lists fitted, phase 2 (the Adam update)
    is enqueued.  If the key buffers overflowed, phase 1 changed no parameter
    or moment, so the buffers are grown and phase 1 runs again.
    key_capacity_per_gaussian sizes each job's key buffers at load."""

    def __init__(self, device, slots, opts, lr=1e-3, bg=(0.0, 0.0, 0.0), deterministic=False,
                 key_capacity_per_gaussian=16):
        import torch

        from . import gsr, pipeline
        self.torch, self.gsr, self.pipeline = torch, gsr, pipeline
        self.device = device
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.opts = opts
        self.deterministic = deterministic
        self.lr = lr
        self.bg = bg
        self.key_capacity_per_gaussian = key_capacity_per_gaussian
        self.rebins = 0  # phase-1 reruns after a key-buffer overflow
        self.copy_stream = torch.cuda.Stream(device=device)
        self._unloading = []  # (job id, pinned host copy, event, device state)
        self._final_params = {}
        self.checkpoints = {}  # job id -> (pinned host [P | M | V], Adam step count, copy event)
        self._evicting = []    # (copy event, device state kept until the copy has finished)
        self.evictions = 0
        self.t0_event = torch.cuda.Event(enable_timing=True)
        self.t0_event.record()
        self.t0_host = time.perf_counter()
        self.loaded = {}
        self.loss_log = {}

    def now(self):
        return time.perf_counter() - self.t0_host

    # job state on the device ------------------------------------------------
    def load(self, job):
        """Allocates the job's device state and queues the upload of its
        parameters and targets on the copy stream; nothing waits.  Steps of
        the job wait for the upload on the GPU (``issue``)."""
        torch = self.torch
        data = job.payload if isinstance(job.payload, JobData) else prepare_job_data(*job.payload)
        n, sizes, offs = data.n, data.sizes, data.offsets
        self._reap()
        ckpt = self.checkpoints.pop(job.job_id, None)
        with torch.cuda.stream(self.copy_stream):
            P = torch.empty(data.params.numel(), dtype=torch.float32, device=self.device)
            if ckpt is None:
                P.copy_(data.params, non_blocking=True)
                M, V = torch.zeros_like(P), torch.zeros_like(P)
            else:  # readmitted: parameters and moments from the checkpoint (ordered after its copy)
                m = P.numel()
                P.copy_(ckpt[0][:m], non_blocking=True)
                M, V = torch.empty_like(P), torch.empty_like(P)
                M.copy_(ckpt[0][m:2 * m], non_blocking=True)
                V.copy_(ckpt[0][2 * m:], non_blocking=True)
            views = [P[offs[i]:offs[i] + sizes[i]] for i in range(5)]
            G = torch.zeros_like(P)
            gv = [G[offs[i]:offs[i] + sizes[i]] for i in range(5)]
            targets = []
            for t in data.targets:
                d = torch.empty(t.shape, dtype=torch.float32, device=self.device)
                d.copy_(t, non_blocking=True)
                targets.append(d)
            st = dict(P=P, G=G, M=M, V=V, pv=views, gv=gv, n=n,
                      sh=data.sh_degree, scale=torch.empty(3 * n, device=self.device),
                      opac=torch.empty(n, device=self.device), dscale=torch.empty(3 * n, device=self.device),
                      dopac=torch.empty(n, device=self.device),
                      vb=self.pipeline.ViewBuffers(n, data.cam, self.device,
                                                   max(1024, int(self.key_capacity_per_gaussian * n))),
                      targets=targets, loss=torch.zeros(1, device=self.device),
                      loss_host=torch.zeros(1).pin_memory(),
                      bin_host=torch.zeros(2, dtype=torch.int32).pin_memory(),
                      adam_step=0 if ckpt is None else ckpt[1])
            st["dimg"] = torch.empty_like(st["vb"].image)
            st["ready"] = torch.cuda.Event()
            st["ready"].record(self.copy_stream)
        self.loaded[job.job_id] = st

    def unload(self, job):
        """Queues the copy of the job's final parameters to pinned host
        memory; the device state is released once that copy has finished
        (the scheduler already counts the footprint as free)."""
        torch = self.torch
        st = self.loaded.pop(job.job_id, None)
        if st is None:
            return
        host = torch.empty(st["P"].numel(), dtype=torch.float32).pin_memory()
        with torch.cuda.stream(self.copy_stream):
            if "done" in st:  # the job's last step (a job cancelled before any step has none)
                self.copy_stream.wait_event(st["done"])
            host.copy_(st["P"], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.copy_stream)
        self._unloading.append((job.job_id, host, ev, st))

    def evict(self, job):
        """Checkpoints an admitted, idle job: its parameters, Adam moments
        and Adam step count go to pinned host memory (queued on the copy
        stream after the job's last step); its device state is released once
        that copy has finished.  ``load`` restores the job from it."""
        torch = self.torch
        st = self.loaded.pop(job.job_id)
        m = st["P"].numel()
        host = torch.empty(3 * m, dtype=torch.float32).pin_memory()
        with torch.cuda.stream(self.copy_stream):
            if "done" in st:
                self.copy_stream.wait_event(st["done"])
            host[:m].copy_(st["P"], non_blocking=True)
            host[m:2 * m].copy_(st["M"], non_blocking=True)
            host[2 * m:].copy_(st["V"], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.copy_stream)
        self.checkpoints[job.job_id] = (host, st["adam_step"], ev)
        self._evicting.append((ev, st))
        self.evictions += 1

    def _reap(self, wait=False):
        """Moves finished final-parameter copies to final_params and drops
        those jobs' device state (and that of evicted jobs whose checkpoint
        copy has finished)."""
        self._evicting = [(ev, st) for ev, st in self._evicting if not ev.query()]
        keep = []
        for jid, host, ev, st in self._unloading:
            if wait:
                ev.synchronize()
            if ev.query():
                self._final_params[jid] = host.numpy()
            else:
                keep.append((jid, host, ev, st))
        self._unloading = keep

    @property
    def final_params(self):
        """Final raw parameters of every unloaded job (waits for pending copies)."""
        self._reap(wait=True)
        return self._final_params

    def issue(self, slot, job, step):
        h = _Step(self.loaded[job.job_id], job.job_id, step, self.streams[slot])
        self._phase1(h)
        return h

    def _phase1(self, h):
        torch, gsr = self.torch, self.gsr
        st, s = h.st, h.stream
        n = st["n"]
        pv, gv, vb = st["pv"], st["gv"], st["vb"]
        s.wait_event(st["ready"])  # the job's upload (complete after its first step)
        with torch.cuda.stream(s):
            gsr.gsr_activate(n, pv[1], pv[3], st["scale"], st["opac"], s)
            sc = self.pipeline.SceneTensors(pv[0], st["scale"], pv[2], st["opac"], pv[4], st["sh"])
            vb.preprocess(sc, zero_grad=True, stream=s)
            vb.bin_async(s)
            vb.forward(self.bg, s)
            st["loss"].zero_()
            tgt = st["targets"][h.step % len(st["targets"])]
            gsr.gsr_l1_loss(vb.image.numel(), vb.image, tgt, st["dimg"], st["loss"], s)
            if self.deterministic:
                vb.backward_deterministic(self.bg, st["dimg"], self.opts, s)
            else:
                vb.backward(self.bg, st["dimg"], self.opts, s)
            st["G"].zero_()
            st["dscale"].zero_()
            st["dopac"].zero_()
            grads = self.pipeline.SceneTensors(gv[0], st["dscale"], gv[2], st["dopac"], gv[4], st["sh"])
            vb.backward_project(sc, grads, s)
            gsr.gsr_activate_backward(n, st["scale"], st["opac"], st["dscale"], st["dopac"], gv[1], gv[3], s)
            st["loss_host"].copy_(st["loss"], non_blocking=True)
            st["bin_host"].copy_(vb.bin_count, non_blocking=True)
            h.event = torch.cuda.Event(enable_timing=True)
            h.event.record(s)
        h.phase = 1

    def _phase2(self, h):
        torch, gsr = self.torch, self.gsr
        st, s = h.st, h.stream
        with torch.cuda.stream(s):
            st["adam_step"] += 1
            gsr.gsr_adam_step(st["P"].numel(), st["P"], st["G"], st["M"], st["V"], self.lr, 0.9, 0.999, 1e-8,
                              st["adam_step"], s)
            h.event = torch.cuda.Event(enable_timing=True)
            h.event.record(s)
            st["done"] = h.event
        h.phase = 2

    def poll(self, h):
        if not h.event.query():
            return None
        st = h.st
        if h.phase == 1:
            cnt, status = (int(x) for x in st["bin_host"])
            # grown key buffers are allocated (and zeroed) on the step's own
            # stream, ordered before the rerun that uses them
            with self.torch.cuda.stream(h.stream):
                fitted = st["vb"].apply_bin_status(cnt, status)
            if fitted:
                self._phase2(h)
            else:  # key buffers grown: the lists of this step were empty, run it again
                self.rebins += 1
                self._phase1(h)
            return None
        completed = self.t0_event.elapsed_time(h.event) / 1e3
        loss = float(st["loss_host"][0])
        self.loss_log.setdefault(h.job_id, []).append(loss)
        return completed + 0.0, loss


@dataclasses.dataclass
class JobData:
    """What a client submits with a job: the raw parameters packed in the
    executor's layout (mean, log-scale, quaternion, opacity logit, features;
    each segment starting on 16 bytes) in pinned host memory, the camera and
    the target images (pinned)."""
    n: int
    sh_degree: int
    sizes: list
    offsets: list
    params: object
    cam: object
    targets: list


def prepare_job_data(scene, cam, targets) -> JobData:
    import torch
    n = scene.n
    k = scene.feat.reshape(n, -1).shape[1]
    sizes = [3 * n, 3 * n, 4 * n, n, k * n]
    padded = [(x + 3) // 4 * 4 for x in sizes]
    offs = [int(x) for x in np.cumsum([0] + padded)]
    flat = np.zeros(offs[-1], np.float32)
    o = scene.opacity.astype(np.float64)
    parts = [scene.mean.reshape(-1), np.log(scene.scale.astype(np.float64)).reshape(-1), scene.quat.reshape(-1),
             np.log(o) - np.log1p(-o), scene.feat.reshape(-1)]
    for i, part in enumerate(parts):
        flat[offs[i]:offs[i] + sizes[i]] = part
    params = torch.from_numpy(flat).pin_memory()
    tg = [torch.from_numpy(np.ascontiguousarray(t, dtype=np.float32)).pin_memory() for t in targets]
    return JobData(n, int(scene.sh_degree), sizes, offs, params, cam, tg)


def make_jobs(spec, seed=0):
    """``spec``: list of (n, steps, arrival_s, width, height)."""
    from . import scenes as S
    jobs = []
    for i, (n, steps, arrival, w, h) in enumerate(spec):
        scene = S.gmm_scene(seed + 101 * i, n, 64, (-4.5, 0.7), 3)
        rng = np.random.default_rng(seed + 7 * i)
        cams = S.sphere_cameras(rng, 1, (0.0, 0.0, 0.0), 4.0, [(w, h)])
        targets = [S.target_image(seed + i, w, h)]
        jobs.append(Job(i, n, steps, arrival, job_footprint(n, 3, w, h),
                        payload=prepare_job_data(scene, cams[0], targets)))
    return jobs


def run_serving(spec, slots, budget_bytes, opts, rate_per_job, seed=0, device="cuda", jobs=None,
                deterministic=False, key_capacity_per_gaussian=16, evict_after=None, quantum=1):
    ex = GpuExecutor(device, slots, opts, deterministic=deterministic,
                     key_capacity_per_gaussian=key_capacity_per_gaussian)
    jobs = jobs if jobs is not None else make_jobs(spec, seed)
    for j in jobs:
        j.state, j.done_steps, j.busy, j.evictions = "waiting", 0, False, 0
    sch = Scheduler(budget_bytes, slots, evict_after, quantum)
    for j in jobs:
        sch.add_job(j)
    reqs = poisson_requests(jobs, rate_per_job, seed + 999)
    wall0 = time.perf_counter()
    res = serve(sch, reqs, ex)
    wall = time.perf_counter() - wall0
    return res, summarize(res, wall, reqs), ex, sch


def job_spec(n_jobs, steps, seed=0, min_n=100_000, max_n=2_000_000, gap_s=0.05):
    """The serving workload: N log-uniform in [min_n, max_n], SH degree 3,
    alternating 1297x840 and 1920x1080 views, jobs arriving ``gap_s`` apart
    on average (exponential gaps)."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(min_n), math.log(max_n), size=n_jobs)).astype(int)
    arrivals = np.cumsum(rng.exponential(gap_s, size=n_jobs))
    res_list = [(1297, 840), (1920, 1080)]
    return [(int(ns[i]), steps, float(arrivals[i]), *res_list[i % 2]) for i in range(n_jobs)]


SATURATED = 1e9  # requests per second per job: every request is there when its job arrives


def benchmark(n_jobs=16, steps=125, rate=10.0, slots=4, budget_gb=24.0, seed=0):
    """The serving measurement: continuous batching with the hybrid tier at
    a Poisson load of ``rate`` requests/s per job and saturated, and the jobs
    run one at a time with the plain atomicAdd tier, saturated (at the
    offered load one job at a time serves only as fast as that job's own
    requests arrive, about n_jobs * steps / rate seconds)."""
    import torch

    from . import gsr
    spec = job_spec(n_jobs, steps, seed)
    jobs = make_jobs(spec, seed)
    budget = int(budget_gb * (1 << 30))
    hybrid = gsr.backward_opts("hybrid", 24, 1, True, 2)
    _, offered, _, sch = run_serving(spec, slots, budget, hybrid, rate, seed, jobs=jobs)
    torch.cuda.synchronize()
    _, sat, _, _ = run_serving(spec, slots, budget, hybrid, SATURATED, seed, jobs=jobs)
    torch.cuda.synchronize()
    one_budget = max(j.footprint for j in jobs)
    _, seq, _, _ = run_serving(spec, 1, one_budget, gsr.backward_opts("plain", 0, 1), SATURATED, seed, jobs=jobs)
    torch.cuda.synchronize()
    return {"workload": f"{n_jobs} jobs, N log-uniform 100k-2M ({sum(j.n for j in jobs)} Gaussians in all), SH3, "
                        f"1297x840 / 1920x1080, {steps} steps (render, L1, backward, backward projection, Adam) "
                        f"each, jobs arriving about 50 ms apart",
            "continuous_batching_hybrid": dict(offered, rate_per_job=rate, slots=slots, budget_gb=budget_gb,
                                               peak_admitted_gb=sch.peak_used / (1 << 30)),
            "continuous_batching_hybrid_saturated": sat,
            "one_at_a_time_plain_saturated": seq}


def main():
    import argparse
    ap = argparse.ArgumentParser(description="serving benchmark: concurrent scene-fitting jobs")
    ap.add_argument("--jobs", type=int, default=16)
    ap.add_argument("--steps", type=int, default=125)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=24.0)
    ap.add_argument("--rate", type=float, default=10.0, help="step requests per second per job")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    print(json.dumps(benchmark(args.jobs, args.steps, args.rate, args.slots, args.budget_gb, args.seed)))


if __name__ == "__main__":
    main()
