"""torch.autograd.Function over the CUDA rasterizer.

* On a 200-Gaussian 64x64 crop of the large-scene camera (SH degree 3): the
  image and the gradients of the raw parameters against the FP64 oracle
  (oracle projection -> binning -> render -> backward projection, chained
  through the activations), with T stored and recomputed.  The stages are held
  to 1e-5 in isolation (test_gpu_parity); end to end the FP32 rounding of the
  projection feeds the blend, so this check is held to 1e-3 of the same
  scales: a wiring check (argument order, activations, zeroing).
* Central differences (eps 1e-3, an absolute step as in torch's gradcheck;
  FP32 forward, loss summed in FP64) against the analytic gradient: the
  spread between the quotients at eps and eps/2 measures the FD's own FP32
  noise and the analytic value must lie in that band (plus 1 %); steps that
  cross a discrete decision of the forward are skipped.
* T stored vs recomputed: same image bit for bit, same gradients up to the
  float summation order of the accumulation, 8 bytes per pixel less kept
  between passes.
* The large scene (3M Gaussians, 1920x1080) through the Function.
"""
import numpy as np
import pytest
import torch

from _helpers import check_scaled
from paper_2401_05345_gb300 import autograd as AG
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


def crop_workload():
    """200 Gaussians (mixture generator, SH3) seen by the central 64x64 crop
    of the 1920x1080 camera of the large scene."""
    full = S.front_camera(1920, 1080)
    x0, y0 = 928, 508
    cam = S.Camera(64, 64, full.view, full.fx, full.fy, full.cx - x0, full.cy - y0, full.tan_fovx,
                   full.tan_fovy, full.campos, full.znear)
    scene = S.gmm_scene(5, 200, 6, (-4.0, 0.5), 3, center_box=0.04, comp_std=(0.01, 0.04))
    return scene, cam


def weights(H, W, seed=3):
    return np.random.default_rng(seed).normal(size=(3, H, W)).astype(np.float32)


def run_model(dev, scene, cam, w, store_T, opts=None, deterministic=False):
    model = AG.GaussianModel(scene, dev)
    st = AG.RasterSettings(cam, (0.1, 0.2, 0.3), opts, store_T, deterministic=deterministic)
    img = model(st)
    loss = (img * torch.from_numpy(w).to(dev)).sum()
    loss.backward()
    grads = {k: p.grad.detach().cpu().numpy() for k, p in model.named_parameters()}
    return img.detach().cpu().numpy(), grads


@pytest.mark.parametrize("store_T", [True, False])
def test_autograd_matches_oracle(dev, orc, store_T):
    scene, cam = crop_workload()
    w = weights(cam.height, cam.width)
    img, g = run_model(dev, scene, cam, w, store_T, gsr.backward_opts("hybrid", 8, 1, store_T))
    pp = orc.preprocess(scene, cam)
    assert pp["pp_ambig"].sum() == 0 and (pp["radius"] > 0).sum() > 150
    ref = orc.render_scene(scene, cam, (0.1, 0.2, 0.3), w, extras=True)
    check_scaled("image", img, ref["image"], 100 * np.abs(ref["image"]), ref["iallow"])
    bp = orc.backproject(scene, cam, ref["grad2d"])
    mag = orc.backproject(scene, cam, ref["gscale"] + ref["gallow"])
    s64, o64 = scene.scale.astype(np.float64), scene.opacity.astype(np.float64)
    n = scene.n
    expect = {
        "mean": (bp["dmean"], mag["dmean_mag"]),
        "log_scale": (bp["dscale"] * s64, mag["dscale_mag"] * s64),
        "quat": (bp["dquat"], mag["dquat_mag"]),
        "opacity_logit": (bp["dopacity"] * o64 * (1 - o64), np.abs(ref["gscale"][:, 5] + ref["gallow"][:, 5]) * o64 * (1 - o64)),
        "feat": (bp["dfeat"].reshape(n, -1), mag["dfeat_mag"].reshape(n, -1)),
    }
    ok = pp["bp_ambig"] == 0
    for k, (r, m) in expect.items():
        check_scaled(f"d{k}", g[k][ok], r[ok], m[ok], rtol=1e-3, atol=1e-6)


def test_store_vs_recompute(dev):
    scene, cam = crop_workload()
    w = weights(cam.height, cam.width)
    img1, g1 = run_model(dev, scene, cam, w, True)
    img0, g0 = run_model(dev, scene, cam, w, False)
    np.testing.assert_array_equal(img1, img0)
    for k in g1:
        scale = np.abs(g1[k]).max()
        assert np.abs(g1[k] - g0[k]).max() <= 1e-5 * scale + 1e-7, k


def _decisions(model, cam, dev):
    """Discrete state of the forward at the model's current parameters: the
    sorted tile lists, every pixel's last contributor and the number of
    active (pixel, splat) pairs.  A central difference is only a derivative
    where this does not change inside the step."""
    from paper_2401_05345_gb300 import pipeline
    with torch.no_grad():
        sc = pipeline.SceneTensors(model.mean.detach(), torch.exp(model.log_scale).detach(), model.quat.detach(),
                                   torch.sigmoid(model.opacity_logit).detach(), model.feat.detach(), model.sh_degree)
        vb = pipeline.ViewBuffers(sc.n, cam, dev, 64 * sc.n)
        vb.preprocess(sc)
        vb.bin()
        vb.forward((0.1, 0.2, 0.3))
        hist = torch.zeros(38, dtype=torch.int64, device=dev)
        gsr.gsr_backward_stats(vb.W, vb.H, 16, 16, vb.tile_ranges, vb.point_list, vb.splat2d, vb.n_contrib, hist)
        return (vb.point_list[:vb.n_keys].cpu().numpy().tobytes(), vb.tile_ranges.cpu().numpy().tobytes(),
                vb.n_contrib.cpu().numpy().tobytes(), int(hist[33]))


def test_autograd_central_differences(dev, orc):
    """Central differences of the FP32 forward at eps = 1e-3 (absolute, as in
    gradcheck) and at eps/2; their spread measures the FD's own FP32 noise,
    and the analytic gradient must lie within that band plus 1 % plus the
    quotient's FP32 rounding floor (3 eps32 times the weighted norm of the
    pixels the step changes, over 2h).
    Entries are drawn from the top quarter of |gradient| of each parameter
    group over the visible Gaussians.  Steps in which a discrete decision
    of the forward changes (list order, last contributor, active pairs) are
    not derivatives and are skipped, and so are steps that change no pixel
    at all (the quotient is then 0 whatever the derivative); at least 25
    entries must have an
    informative band (band plus floor narrower than 20 % of the value)."""
    scene, cam = crop_workload()
    vis = np.nonzero(orc.preprocess(scene, cam)["radius"] > 0)[0]
    w = torch.from_numpy(weights(cam.height, cam.width)).to(dev).double()
    model = AG.GaussianModel(scene, dev)
    st = AG.RasterSettings(cam, (0.1, 0.2, 0.3), None, True)
    img0 = model(st)
    (img0.double() * w).sum().backward()
    base = _decisions(model, cam, dev)

    def rounding_floor(ip, im, h):
        # the forward is deterministic: pixels the step does not change round
        # identically and cancel; each changed pixel carries independent FP32
        # rounding (unit roundoff 2^-24) in both evaluations -> 3 sigma of the
        # central quotient's noise
        ch = ip != im
        nrm = float(torch.linalg.norm((ip.double() * w)[ch])) + float(torch.linalg.norm((im.double() * w)[ch]))
        return 3 * 2.0 ** -24 * nrm / (2 * h)
    rng = np.random.default_rng(0)
    informative, checked, crossings, unresolved = 0, 0, 0, 0
    with torch.no_grad():
        for name, p in model.named_parameters():
            g = p.grad.detach().cpu().numpy()
            per = p.data[0].numel()
            flat = p.data.view(-1)
            # entries a difference quotient can resolve: random ones among the
            # top quarter of |gradient| over the visible Gaussians' entries
            cand = (vis[:, None] * per + np.arange(per)[None, :]).reshape(-1)
            mag = np.abs(g.reshape(-1)[cand])
            cand = cand[mag >= np.quantile(mag, 0.75)]
            for idx in rng.choice(cand, 30, replace=False):
                idx = int(idx)
                x0 = float(flat[idx])
                fds, crossed, floor, changed = [], False, 0.0, False
                for h in (1e-3, 5e-4):
                    flat[idx] = x0 + h
                    ip = model(st).detach()
                    crossed |= _decisions(model, cam, dev) != base
                    flat[idx] = x0 - h
                    im = model(st).detach()
                    crossed |= _decisions(model, cam, dev) != base
                    flat[idx] = x0
                    fds.append(float(((ip.double() - im.double()) * w).sum()) / (2 * h))
                    changed |= bool((ip != im).any())
                    if h == 1e-3:
                        floor = rounding_floor(ip, im, h)
                if crossed:
                    crossings += 1
                    continue
                if not changed:
                    # no pixel moved by a rounding step: the quotient is 0
                    # whatever the derivative, it measures nothing
                    unresolved += 1
                    continue
                an = float(g.reshape(-1)[idx])
                band = abs(fds[0] - fds[1])
                checked += 1
                if band + floor < 0.2 * abs(an):
                    informative += 1
                assert abs(fds[0] - an) <= 2 * band + 1e-2 * abs(an) + floor, (name, idx, fds, an, floor)
    assert informative >= 25, (informative, checked, crossings, unresolved)


def test_large_scene_through_autograd(dev):
    """3M Gaussians at 1080p through the autograd Function.  With the
    atomic-free backward every stage is bitwise repeatable, and recomputing T
    in the backward reproduces the forward's T bit for bit, so stored and
    recomputed T give the same gradient bits.  The atomic HYBRID tier on the
    same scene gives finite gradients within float summation-order noise of
    those (its exact sums are checked against the oracle at small sizes)."""
    scene, cam = S.large_workload(0)
    w = np.where(np.random.default_rng(1).uniform(size=(3, cam.height, cam.width)) < 0.5, -1.0, 1.0).astype(np.float32)
    res = {}
    for key, store_T in (("store", True), ("store_again", True), ("recompute", False)):
        torch.cuda.synchronize()
        img, g = run_model(dev, scene, cam, w, store_T, gsr.backward_opts("warp", 0, 1, store_T, 2),
                           deterministic=True)
        res[key] = (img, g)
    np.testing.assert_array_equal(res["store"][0], res["recompute"][0])
    np.testing.assert_array_equal(res["store"][0], res["store_again"][0])
    for k in res["store"][1]:
        a = res["store"][1][k]
        assert np.isfinite(a).all()
        np.testing.assert_array_equal(a, res["store_again"][1][k])
        np.testing.assert_array_equal(a, res["recompute"][1][k])
    assert np.abs(res["store"][1]["mean"]).max() > 0
    img, ga = run_model(dev, scene, cam, w, True, gsr.backward_opts("hybrid", 12, 1, True))
    np.testing.assert_array_equal(img, res["store"][0])
    for k, ref in res["store"][1].items():
        a = ga[k]
        assert np.isfinite(a).all()
        # two atomic runs differ by about 5e-5 of the norm (summation order)
        assert np.linalg.norm(a - ref) <= 1e-3 * np.linalg.norm(ref), (k, np.linalg.norm(a - ref))


def test_recompute_keeps_less_state(dev):
    from paper_2401_05345_gb300.pipeline import ViewBuffers
    cam = S.front_camera(1920, 1080)
    a = ViewBuffers(1000, cam, dev, 1024, store_T=True)
    b = ViewBuffers(1000, cam, dev, 1024, store_T=False)
    assert a.device_bytes() - b.device_bytes() == 8 * 1920 * 1080
