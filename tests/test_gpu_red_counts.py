"""Traversal statistics and the global red traffic of each accumulation tier.

* gsr_backward_stats against the oracle: active (pixel, splat) pairs equal
  the oracle's per-pixel contributor counts summed (Sec. III-A: one atomic
  per parameter per such pair in the baseline), and the examined pairs the
  oracle's last-contributor positions summed, except where an FP32-ambiguous
  decision may flip a pair.
* gsr_backward_red_counts against the active-lanes histogram of the same
  traversal: PLAIN sends 9 adds per active pair; WARP one 9-lane red per
  warp step with an active lane; HYBRID with threshold t the WARP form for
  steps with >= t active lanes and two v4 reds plus one scalar red per
  active lane otherwise (Sec. IV-B).  Integer identities, exact.
"""
import numpy as np
import pytest
import torch

from _helpers import pack_records, records_f64
from paper_2401_05345_gb300 import gsr
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


@pytest.fixture(scope="module")
def view(dev, orc):
    scene, cam = S.gmm_scene(3, 20000, 32, (-3.2, 0.4), 1), S.front_camera(200, 150)
    pp = orc.preprocess(scene, cam)
    rec, radius = pack_records(pp)
    r64 = records_f64(rec)
    W, H = cam.width, cam.height
    keys, pl, ranges = orc.bin_sort(r64["uv"], r64["depth"], radius, W, H)
    out = orc.render(W, H, ranges, pl, r64["uv"], r64["conic"], r64["opacity"], r64["rgb"], np.zeros(3))
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    image = torch.zeros((3, H, W), device=dev)
    fT = torch.zeros((H, W), device=dev)
    nc = torch.zeros((H, W), dtype=torch.int32, device=dev)
    v = dict(W=W, H=H, ranges=T(ranges.view(np.int32)), pl=T(np.concatenate([pl, [0]]).astype(np.uint32).view(np.int32)),
             splat=T(rec), fT=fT, nc=nc, out=out)
    gsr.gsr_forward(W, H, 16, 16, v["ranges"], v["pl"], v["splat"], (0.0, 0.0, 0.0), image, fT, nc)
    torch.cuda.synchronize()
    return v


def _hist(v, layout):
    h = torch.zeros(38, dtype=torch.int64, device=v["splat"].device)
    gsr.gsr_backward_stats(v["W"], v["H"], 16, 16, v["ranges"], v["pl"], v["splat"], v["nc"], h, layout)
    return h.cpu().numpy().astype(np.int64)


def _counts(v, opts):
    c = torch.zeros(39, dtype=torch.int64, device=v["splat"].device)
    gsr.gsr_backward_red_counts(v["W"], v["H"], 16, 16, v["ranges"], v["pl"], v["splat"], v["fT"], v["nc"], opts, c)
    c = c.cpu().numpy().astype(np.int64)
    out = dict(zip(gsr.RED_COUNT_NAMES, c.tolist()))
    out["hist"] = c[6:]
    return out


@pytest.mark.parametrize("layout", [0, 1])
def test_stats_match_oracle_pair_counts(view, layout):
    h = _hist(view, layout)
    out = view["out"]
    amb = int((out["pix_ambig"] > 0).sum())
    assert abs(int(h[33]) - int(out["n_active"].sum())) <= amb
    assert int(h[34]) == int(view["nc"].cpu().numpy().sum())
    assert abs(int(h[34]) - int(out["n_contrib"].sum())) <= int(np.abs(out["nc_alt"] - out["n_contrib"])[
        out["pix_ambig"] > 0].sum())
    assert int((np.arange(33) * h[:33]).sum()) == int(h[33])  # active lanes per step add up to the pairs
    assert h[33] > 100_000


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("tier", [("plain", 0), ("warp", 0), ("hybrid", 1), ("hybrid", 8), ("hybrid", 24),
                                  ("hybrid", 33)])
def test_red_counts_follow_the_active_lane_histogram(view, tier, layout):
    h = _hist(view, layout)
    act = np.arange(33)
    steps = int(h[1:33].sum())  # warp steps with at least one active lane
    c = _counts(view, gsr.backward_opts(tier[0], tier[1], layout))
    assert c["warp_steps_active"] == steps
    assert c["warp_steps"] >= steps
    # the same traversal: steps with a >= 1 active lanes as the statistics
    # kernel counts them (it also counts the steps the cull skips, all at 0)
    np.testing.assert_array_equal(c["hist"][1:], h[1:33])
    assert c["hist"].sum() == c["warp_steps"]
    if tier[0] == "plain":
        assert c["adds"] == c["lane_reds"] == 9 * int(h[33])
        assert c["red_instructions"] == 9 * steps and c["red_v4_instructions"] == 0
        return
    t = 0 if tier[0] == "warp" else tier[1]
    dense = int(h[max(t, 1):33].sum())
    sparse_steps = int(h[1:max(t, 1)].sum())
    sparse_lanes = int((act[1:max(t, 1)] * h[1:max(t, 1)]).sum())
    assert c["adds"] == 9 * dense + 9 * sparse_lanes
    assert c["lane_reds"] == 9 * dense + 3 * sparse_lanes
    assert c["red_instructions"] == dense + sparse_steps
    assert c["red_v4_instructions"] == 2 * sparse_steps


def test_red_counts_two_pixels_per_thread(view):
    """Two pixels per thread: one step serves 64 pixels, so a warp with any
    active pixel reduces once; the adds still cover every parameter of every
    warp step with an active lane."""
    c1 = _counts(view, gsr.backward_opts("warp", 0, 1, True, 1))
    c2 = _counts(view, gsr.backward_opts("warp", 0, 1, True, 2))
    assert c2["adds"] == 9 * c2["warp_steps_active"] and c2["red_v4_instructions"] == 0
    assert int((np.arange(33) * c2["hist"]).sum()) <= int((np.arange(33) * c1["hist"]).sum())
    assert c2["warp_steps_active"] < c1["warp_steps_active"] < 2 * c2["warp_steps_active"] + 1
