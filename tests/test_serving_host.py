"""Host logic of the serving loop (no GPU): admission by footprint, refusal
of jobs larger than the budget, continuous batching over slots, one step at
a time per job, cancellation and memory release.  Failures are injected on
the host (fake executor with a virtual clock)."""
import pytest

from paper_2401_05345_gb300 import serving as SV


class FakeExecutor:
    def __init__(self, step_s=0.010, tick=0.0005):
        self.t = 0.0
        self.tick = tick
        self.step_s = step_s
        self.loaded, self.unloaded, self.issued = [], [], []
        self.inflight_jobs = set()
        self.max_concurrent = 0

    def now(self):
        self.t += self.tick
        return self.t

    def load(self, job):
        self.loaded.append(job.job_id)

    def unload(self, job):
        self.unloaded.append(job.job_id)

    def issue(self, slot, job, step):
        assert job.job_id not in self.inflight_jobs, "two steps of one job in flight"
        self.inflight_jobs.add(job.job_id)
        self.max_concurrent = max(self.max_concurrent, len(self.inflight_jobs))
        self.issued.append((job.job_id, step, self.t))
        return (job.job_id, step, self.t + self.step_s)

    def poll(self, h):
        jid, step, end = h
        if self.t >= end:
            self.inflight_jobs.discard(jid)
            return end, float(step)
        return None


def jobs(footprints, steps=3, arrival=0.0):
    return [SV.Job(i, 1000, steps, arrival, f) for i, f in enumerate(footprints)]


def test_admission_first_fit_and_refusal():
    sch = SV.Scheduler(100, 2)
    js = jobs([60, 50, 30, 120])
    for j in js:
        sch.add_job(j)
    assert js[3].state == "refused"
    ex = FakeExecutor()
    sch.admit(ex.load)
    assert ex.loaded == [0, 2] and sch.used == 90
    sch.jobs[0].done_steps = 2
    sch.complete(0, ex.unload)   # job 0 finishes its last step
    assert ex.unloaded == [0] and sch.used == 30
    sch.admit(ex.load)
    assert ex.loaded == [0, 2, 1] and sch.used == 80


def test_serving_runs_every_request_with_overlap_and_memory_bound():
    js = jobs([40, 40, 40, 40], steps=4)
    sch = SV.Scheduler(100, 3)     # two jobs fit at a time
    for j in js:
        sch.add_job(j)
    reqs = SV.poisson_requests(js, rate_per_job=500.0, seed=1)
    ex = FakeExecutor()
    res = SV.serve(sch, reqs, ex)
    assert len(res) == 16
    assert sch.peak_used <= 100
    assert ex.max_concurrent == 2           # overlap, bounded by admission
    for j in js:                             # steps of a job complete in order
        steps = [r.step for r in sorted(res, key=lambda r: r.completed) if r.job_id == j.job_id]
        assert steps == [0, 1, 2, 3]
    assert all(r.completed >= r.arrival for r in res)
    st = SV.summarize(res, 1.0)
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_late_arrivals_join_while_others_run():
    js = [SV.Job(0, 1, 6, 0.0, 10), SV.Job(1, 1, 2, 0.02, 10)]
    sch = SV.Scheduler(100, 2)
    for j in js:
        sch.add_job(j)
    reqs = SV.poisson_requests(js, rate_per_job=1000.0, seed=2)
    ex = FakeExecutor(step_s=0.01)
    res = SV.serve(sch, reqs, ex)
    first1 = min(r.issued for r in res if r.job_id == 1)
    last0 = max(r.completed for r in res if r.job_id == 0)
    assert first1 < last0                    # job 1 started before job 0 finished
    assert ex.max_concurrent == 2


def test_cancellation_releases_memory_and_drops_requests():
    js = jobs([60, 60], steps=50)
    sch = SV.Scheduler(100, 2)
    for j in js:
        sch.add_job(j)
    reqs = SV.poisson_requests(js, rate_per_job=2000.0, seed=3)
    ex = FakeExecutor(step_s=0.002)
    res = SV.serve(sch, reqs, ex, cancel_at={0: 0.01})
    assert sch.jobs[0].state == "cancelled"
    assert 0 in ex.unloaded and 1 in ex.loaded  # job 1 admitted after job 0 released its memory
    assert sum(1 for r in res if r.job_id == 1) == 50
    assert sum(1 for r in res if r.job_id == 0) < 50


def test_refused_job_runs_nothing():
    js = jobs([500, 10], steps=2)
    sch = SV.Scheduler(100, 1)
    for j in js:
        sch.add_job(j)
    ex = FakeExecutor()
    res = SV.serve(sch, SV.poisson_requests(js, 100.0, 4), ex)
    assert {r.job_id for r in res} == {1}
    assert 0 not in ex.loaded


def test_footprint_model_matches_the_recorded_per_gaussian_state():
    # params + grads + 2 Adam moments: 4 x 59 floats x 4 B = 944 B per Gaussian at SH degree 3
    a = SV.job_footprint(1000, 3, 16, 16)
    b = SV.job_footprint(2000, 3, 16, 16)
    assert b - a >= 944 * 1000


class EvictingExecutor(FakeExecutor):
    """Fake executor that also checkpoints: records evictions and which jobs
    were loaded back from a checkpoint."""

    def __init__(self, **kw):
        super().__init__(**kw)
        self.evicted, self.ckpt, self.restored = [], set(), []

    def evict(self, job):
        assert job.job_id not in self.inflight_jobs, "evicting a job with a step in flight"
        self.evicted.append(job.job_id)
        self.ckpt.add(job.job_id)

    def load(self, job):
        super().load(job)
        if job.job_id in self.ckpt:
            self.ckpt.discard(job.job_id)
            self.restored.append(job.job_id)


def test_eviction_makes_room_and_the_job_resumes():
    """Job 1 does not fit beside job 0: after waiting evict_after seconds it
    has job 0 checkpointed out (once job 0 ran its quantum of steps and is
    idle), runs, and job 0 is readmitted from its checkpoint and finishes
    every step exactly once, in order."""
    js = [SV.Job(0, 1, 12, 0.0, 60), SV.Job(1, 1, 3, 0.001, 70)]
    sch = SV.Scheduler(100, 2, evict_after=0.005, quantum=2)
    for j in js:
        sch.add_job(j)
    ex = EvictingExecutor(step_s=0.002)
    res = SV.serve(sch, SV.poisson_requests(js, 5000.0, 7), ex)
    assert ex.evicted == [0] and ex.restored == [0]
    ev = sch.events
    assert ev.index("evict 0") < ev.index("admit 1") < ev.index("release 1") < len(ev) - 1 - ev[::-1].index("admit 0")
    steps0 = [s for (j, s, _) in ex.issued if j == 0]
    assert steps0 == list(range(12))
    assert len(res) == 15 and sch.peak_used <= 100
    n_before = sum(1 for (j, s, t) in ex.issued if j == 0 and t < min(t1 for (j1, _, t1) in ex.issued if j1 == 1))
    assert n_before >= 2  # the quantum ran before the eviction


def test_no_eviction_without_a_waiting_limit_or_enough_memory():
    # evict_after None: job 1 waits for job 0 to finish
    js = [SV.Job(0, 1, 6, 0.0, 60), SV.Job(1, 1, 2, 0.001, 70)]
    sch = SV.Scheduler(100, 2)
    for j in js:
        sch.add_job(j)
    ex = EvictingExecutor(step_s=0.002)
    SV.serve(sch, SV.poisson_requests(js, 5000.0, 8), ex)
    assert ex.evicted == [] and sch.events.index("release 0") < sch.events.index("admit 1")
    # evicting every idle job would not free enough (job 1 has a step in
    # flight): nobody is evicted
    sch = SV.Scheduler(100, 2, evict_after=0.0)
    sch.add_job(SV.Job(0, 1, 5, 0.0, 40))
    sch.add_job(SV.Job(1, 1, 5, 0.0, 40))
    sch.admit(lambda j: None)
    for j in sch.jobs.values():
        j.done_steps = 1
    sch.jobs[1].busy = True
    big = SV.Job(2, 1, 5, 0.0, 70)
    sch.add_job(big)
    assert sch.maybe_evict(1.0, lambda j: None) == [] and sch.used == 80
    sch.jobs[1].busy = False  # now the two idle jobs free enough: both go, oldest admission first
    out = sch.maybe_evict(1.0, lambda j: None)
    assert [j.job_id for j in out] == [0, 1] and sch.used == 0
    sch.admit(lambda j: None, 1.0)
    assert big.state == "admitted" and sch.jobs[0].state == "waiting"
    # an evicted job does not evict others in its turn
    assert sch.maybe_evict(2.0, lambda j: None) == []


def test_busy_and_fresh_jobs_are_not_evicted():
    sch = SV.Scheduler(100, 2, evict_after=0.0, quantum=3)
    sch.add_job(SV.Job(0, 1, 9, 0.0, 60))
    sch.admit(lambda j: None)
    j0 = sch.jobs[0]
    sch.add_job(SV.Job(1, 1, 2, 0.0, 70))
    j0.done_steps = 2                      # fewer steps than the quantum since admission
    assert sch.maybe_evict(1.0, lambda j: None) == []
    j0.done_steps, j0.busy = 3, True      # a step in flight
    assert sch.maybe_evict(1.0, lambda j: None) == []
    j0.busy = False
    assert [j.job_id for j in sch.maybe_evict(1.0, lambda j: None)] == [0]
