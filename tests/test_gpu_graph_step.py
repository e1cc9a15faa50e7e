"""A training step captured in a CUDA graph (pipeline.StepGraph) against the
same step launched kernel by kernel.  With the atomic-free backward every
stage is bitwise repeatable, so image, transmittance, lists and 3D gradients
must be equal bit for bit.  Only the loss is a float sum of block partials
added by atomics in run-dependent order: every add rounds to the running
sum's ulp, so two runs differ by a few ulp of the total per add, well inside
the 1e-5 relative tolerance used for such sums throughout the tests."""
import numpy as np
import pytest
import torch

from paper_2401_05345_gb300 import gsr, pipeline
from paper_2401_05345_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_05345_gb300 import build
    build.build()
    gsr.lib()
    return torch.device("cuda")


def _setup(dev, scene, cam, seed=0, deterministic=True, key_capacity=None):
    sc = pipeline.SceneTensors.from_scene(scene, dev)
    grads = sc.zeros_like_params()
    target = torch.from_numpy(S.target_image(seed, cam.width, cam.height)).to(dev)
    R = pipeline.Renderer(scene.n, cam, dev, opts=gsr.backward_opts("warp", 0, 1, True, 2),
                          deterministic=deterministic, key_capacity=key_capacity)
    return sc, grads, target, R


def _snapshot(R, grads):
    vb = R.vb
    out = {"loss": float(R.loss.item()), "image": vb.image.clone(), "final_T": vb.final_T.clone(),
           "n_contrib": vb.n_contrib.clone(), "ranges": vb.tile_ranges.clone(),
           "list": vb.point_list[:vb.n_keys].clone()}
    for name, t in zip(("mean", "scale", "quat", "opacity", "feat"), grads.tensors()):
        out["d" + name] = t.clone()
    return out


def _assert_same(a, b):
    assert a["loss"] == pytest.approx(b["loss"], rel=1e-5)
    for k in a:
        if k != "loss":
            assert torch.equal(a[k], b[k]), k


def _stream_step(R, sc, target, grads):
    bg = (0.0, 0.0, 0.0)
    R.step(sc, target, bg, grads, accumulate=False)
    torch.cuda.synchronize()
    return _snapshot(R, grads)


@pytest.mark.parametrize("which", ["tiny", "gmm-60k"])
def test_graph_replay_equals_stream_step_bitwise(dev, which):
    if which == "tiny":
        scene, cam = S.tiny_workload(0)
    else:
        scene = S.gmm_scene(1, 60_000, components=16)
        cam = S.front_camera(640, 416)
    sc, grads, target, R = _setup(dev, scene, cam)
    ref = _stream_step(R, sc, target, grads)
    g = pipeline.StepGraph(R, sc, target, (0.0, 0.0, 0.0), grads, accumulate=False)
    for _ in range(3):  # every replay recomputes the same step
        grads.mean.fill_(123.0)
        g.replay()
        torch.cuda.synchronize()
        assert g.ok()
        _assert_same(_snapshot(R, grads), ref)


def test_graph_replay_follows_new_inputs(dev):
    """Inputs are copied into the captured tensors: a new target and moved
    Gaussians give the stream step's result on those inputs."""
    scene = S.gmm_scene(2, 40_000, components=8)
    cam = S.front_camera(512, 384)
    sc, grads, target, R = _setup(dev, scene, cam)
    g = pipeline.StepGraph(R, sc, target, (0.0, 0.0, 0.0), grads, accumulate=False)
    target.copy_(torch.from_numpy(S.target_image(7, cam.width, cam.height)).to(dev))
    sc.mean.add_(0.01)
    g.replay()
    torch.cuda.synchronize()
    assert g.ok()
    got = _snapshot(R, grads)
    ref = _stream_step(R, sc, target, grads)
    _assert_same(got, ref)


def test_graph_reports_key_overflow_and_recaptures(dev):
    """Growing the splats after capture overflows the captured key buffers:
    every tile range of the replay is empty (nothing reads the lists),
    ok() is False and grows the buffers, and a new capture gives the stream
    step's result."""
    scene = S.gmm_scene(3, 30_000, components=8)
    cam = S.front_camera(512, 384)
    sc, grads, target, R = _setup(dev, scene, cam)
    R.vb.bin()  # the synchronous pass sizes the buffers to this scene
    g = pipeline.StepGraph(R, sc, target, (0.0, 0.0, 0.0), grads, accumulate=False)
    cap0 = R.vb.key_capacity
    sc.scale.mul_(10.0)  # each splat now covers many more tiles
    g.replay()
    torch.cuda.synchronize()
    assert int(R.vb.tile_ranges.max().item()) == 0
    assert not g.ok()
    assert R.vb.key_capacity > cap0
    g = pipeline.StepGraph(R, sc, target, (0.0, 0.0, 0.0), grads, accumulate=False)
    g.replay()
    torch.cuda.synchronize()
    assert g.ok()
    got = _snapshot(R, grads)
    _assert_same(got, _stream_step(R, sc, target, grads))


def test_graph_backward_events_time_the_backward(dev):
    """External events recorded inside the graph time the backward launch
    on every replay; the atomic tiers replay within float tolerance."""
    scene = S.gmm_scene(4, 50_000, components=16)
    cam = S.front_camera(640, 416)
    sc, grads, target, R = _setup(dev, scene, cam, deterministic=False)
    R.opts = gsr.backward_opts("hybrid", 12, 1, True, 2)
    ref = _stream_step(R, sc, target, grads)
    try:
        ev = (torch.cuda.Event(enable_timing=True, external=True),
              torch.cuda.Event(enable_timing=True, external=True))
    except TypeError:
        pytest.skip("this torch has no external events")
    g = pipeline.StepGraph(R, sc, target, (0.0, 0.0, 0.0), grads, accumulate=False, backward_events=ev)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert 0.0 < ev[0].elapsed_time(ev[1]) < 1000.0
    got = _snapshot(R, grads)
    for k in ("image", "final_T", "n_contrib", "ranges", "list"):
        assert torch.equal(got[k], ref[k]), k
    for k in ("dmean", "dscale", "dquat", "dopacity", "dfeat"):
        a, b = got[k].cpu().numpy(), ref[k].cpu().numpy()
        scale = np.abs(b).max()
        assert np.abs(a - b).max() <= 1e-4 * scale + 1e-7, k


def test_pipeline_with_two_steps_in_flight(dev):
    """StepPipeline: five steps on different targets, each submitted before
    the previous step's loss is read, give every step's loss as a lone graph
    replay on that target does, and the last step's outputs bit for bit."""
    scene = S.gmm_scene(6, 40_000, components=8)
    cam = S.front_camera(512, 384)
    sc, grads, target, R = _setup(dev, scene, cam)
    hosts = [torch.from_numpy(S.target_image(20 + i, cam.width, cam.height)).pin_memory() for i in range(5)]
    pipe = pipeline.StepPipeline(R, sc, (0.0, 0.0, 0.0), grads)
    losses, prev = [], None
    for h in hosts:
        k = pipe.submit(h)
        if prev is not None:
            losses.append(pipe.result(prev))
        prev = k
    losses.append(pipe.result(prev))
    torch.cuda.synchronize()
    assert pipe.ok()
    last = _snapshot(R, grads)
    g = pipeline.StepGraph(R, sc, target, (0.0, 0.0, 0.0), grads, accumulate=False)
    for h, loss in zip(hosts, losses):
        target.copy_(h)
        g.replay()
        torch.cuda.synchronize()
        assert float(R.loss.item()) == pytest.approx(loss, rel=1e-5)
    _assert_same(_snapshot(R, grads), last)
