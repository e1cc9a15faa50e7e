"""Serving loop on the GPU: continuous batching of concurrent scene-fitting
jobs (render + backward + Adam per request) with admission by HBM footprint.
Each job's results in the mix must be the same as when it runs alone: the
step losses within the 1e-5 relative tolerance (the loss sum and the
gradient accumulation are float sums in run-dependent order) and the final
parameters within
1e-5 |p| + 1e-3 lr * steps (the gradients of the two runs differ only by FP32
summation order, which Adam passes on scaled by lr / (|g| + eps))."""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2401_05345_gb300 import gsr
from paper_2401_05345_gb300 import serving as SV

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_05345_gb300 import build
    build.build()
    gsr.lib()
    return torch.device("cuda")


def test_each_job_same_alone_and_in_the_mix(dev):
    spec = [(20000, 4, 0.0, 160, 120), (40000, 4, 0.005, 200, 150), (30000, 4, 0.01, 160, 120),
            (25000, 4, 0.015, 200, 150)]
    jobs = SV.make_jobs(spec, seed=0)
    fps = sorted(j.footprint for j in jobs)
    budget = fps[-1] + fps[-2] + 1          # two jobs at a time: admission has to wait
    opts = gsr.backward_opts("hybrid", 8, 1)
    res, stats, ex, sch = SV.run_serving(None, 3, budget, opts, 400.0, seed=0, device=dev, jobs=jobs)
    assert len(res) == 16 and sch.peak_used <= budget
    assert any(e.startswith("admit") for e in sch.events[2:])   # someone was admitted later
    assert np.isfinite(stats["p50_ms"]) and stats["p99_ms"] >= stats["p50_ms"]
    lr = ex.lr
    for j in jobs:
        alone_job = dataclasses.replace(j, state="waiting", done_steps=0, busy=False)
        _, _, ex1, _ = SV.run_serving(None, 1, j.footprint, opts, 400.0, seed=0, device=dev, jobs=[alone_job])
        la, lm = np.array(ex1.loss_log[j.job_id]), np.array(ex.loss_log[j.job_id])
        np.testing.assert_allclose(lm, la, rtol=1e-5)
        pa, pm = ex1.final_params[j.job_id], ex.final_params[j.job_id]
        assert np.all(np.abs(pm - pa) <= 1e-5 * np.abs(pa) + 1e-3 * lr * j.steps)


def test_deterministic_tier_gives_bitwise_equal_jobs_alone_and_in_the_mix(dev):
    """With the atomic-free backward every step of a job is bit-identical
    whatever runs beside it: final parameters are equal bit for bit."""
    spec = [(20000, 3, 0.0, 160, 120), (30000, 3, 0.005, 200, 150), (25000, 3, 0.01, 160, 120)]
    jobs = SV.make_jobs(spec, seed=3)
    fps = sorted(j.footprint for j in jobs)
    opts = gsr.backward_opts("warp", 0, 1, True, 2)
    _, _, ex, sch = SV.run_serving(None, 3, fps[-1] + fps[-2] + 1, opts, 400.0, seed=3, device=dev, jobs=jobs,
                                   deterministic=True)
    for j in jobs:
        alone = dataclasses.replace(j, state="waiting", done_steps=0, busy=False)
        _, _, ex1, _ = SV.run_serving(None, 1, j.footprint, opts, 400.0, seed=3, device=dev, jobs=[alone],
                                      deterministic=True)
        np.testing.assert_array_equal(ex1.final_params[j.job_id], ex.final_params[j.job_id])


def test_key_buffer_overflow_reruns_the_render_phase(dev):
    """Jobs loaded with key buffers far too small for their lists: the first
    step of every job overflows, the executor grows the buffers and runs the
    render phase again before any Adam update, and every job ends with the
    same parameters, bit for bit (atomic-free backward), as a run whose
    buffers were large enough from the start."""
    spec = [(20000, 3, 0.0, 160, 120), (30000, 3, 0.005, 200, 150)]
    jobs = SV.make_jobs(spec, seed=5)
    budget = sum(j.footprint for j in jobs) + 1
    opts = gsr.backward_opts("warp", 0, 1, True, 2)
    _, _, ex_small, _ = SV.run_serving(None, 2, budget, opts, 400.0, seed=5, device=dev, jobs=jobs,
                                       deterministic=True, key_capacity_per_gaussian=0.01)
    assert ex_small.rebins >= len(jobs)
    _, _, ex_ok, _ = SV.run_serving(None, 2, budget, opts, 400.0, seed=5, device=dev, jobs=jobs,
                                    deterministic=True)
    assert ex_ok.rebins == 0
    for j in jobs:
        np.testing.assert_array_equal(ex_small.final_params[j.job_id], ex_ok.final_params[j.job_id])
        np.testing.assert_allclose(ex_small.loss_log[j.job_id], ex_ok.loss_log[j.job_id], rtol=1e-5)


def test_evicted_job_resumes_bit_identical(dev):
    """Checkpoint and readmission: the first job is evicted after two of its
    steps for a larger one that does not fit beside it, goes to pinned host
    memory (parameters, Adam moments, Adam step count) and is restored from
    there once the larger job is done.  With the atomic-free backward, both
    jobs end with the parameters of their runs alone, bit for bit."""
    spec = [(20000, 6, 0.0, 160, 120), (40000, 3, 0.002, 200, 150)]
    jobs = SV.make_jobs(spec, seed=9)
    budget = max(j.footprint for j in jobs) + 1   # one job at a time
    opts = gsr.backward_opts("warp", 0, 1, True, 2)
    res, _, ex, sch = SV.run_serving(None, 2, budget, opts, 400.0, seed=9, device=dev, jobs=jobs,
                                     deterministic=True, evict_after=0.0, quantum=2)
    assert ex.evictions == 1 and "evict 0" in sch.events and sch.events.count("admit 0") == 2
    assert len(res) == 9 and sch.peak_used <= budget
    steps0 = [r.step for r in sorted(res, key=lambda r: r.completed) if r.job_id == 0]
    assert steps0 == list(range(6))
    for j in jobs:
        alone = dataclasses.replace(j, state="waiting", done_steps=0, busy=False, evictions=0)
        _, _, ex1, _ = SV.run_serving(None, 1, j.footprint, opts, 400.0, seed=9, device=dev, jobs=[alone],
                                      deterministic=True)
        np.testing.assert_array_equal(ex1.final_params[j.job_id], ex.final_params[j.job_id])
        np.testing.assert_allclose(ex1.loss_log[j.job_id], ex.loss_log[j.job_id], rtol=1e-5)
