"""torch.autograd.Function over the CUDA rasterizer.

* On a 200-Gaussian 64x64 crop of the large-scene camera (SH degree 3): the
  image and the gradients of the raw parameters against the FP64 oracle
  (oracle projection -> binning -> render -> backward projection, chained
  through the activations), with T stored and recomputed, at 1e-5 of the
  same scales as the stage tests.  End to end, the FP32 projection's error
  feeds the blend; the oracle bounds what it can do to first order (each
  splat's record components moved one at a time by the projection's own
  tolerance, the absolute changes of the image and 2D gradients summed) and
  that bound joins the allowances, as do depth ties within FP32 rounding
  (both draw orders are valid).
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


EPS32 = 2.0 ** -24
_crop_ref = {}


def crop_reference(orc, scene, cam, w, bg):
    """The oracle's image and 2D gradients of the crop, with the allowances
    of an end-to-end comparison: ``pimg`` / ``pgrad`` bound (to first order)
    what an FP32 projection within its tested tolerance (1e-5 of the scale of
    each record component, plus 1e-7) changes, and ``timg`` / ``tgrad`` are
    the changes from swapping co-listed splats whose depths lie within FP32
    rounding of each other (32 ulp)."""
    key = (id(scene), cam.width)
    if key in _crop_ref:
        return _crop_ref[key]
    W, H = cam.width, cam.height
    pp = orc.preprocess(scene, cam)
    keys, pl, ranges = orc.bin_sort(pp["uv"], pp["depth"], pp["radius"], W, H)
    bg = np.asarray(bg, np.float64)
    rec = [pp["uv"].copy(), pp["conic"].copy(), pp["opacity"].copy(), pp["rgb"].copy()]
    render = lambda pl_, r_, extras=False: orc.render(W, H, ranges, pl_, r_[0], r_[1], r_[2], r_[3], bg, w,
                                                      extras=extras)
    ref = render(pl, rec, extras=True)
    # the projection's tested tolerance per record component (test_gpu_parity)
    A, B, C = pp["conic"][:, 0], pp["conic"][:, 1], pp["conic"][:, 2]
    kap = np.maximum((np.abs(A * C) + B * B) / (A * C - B * B + 1e-300), 1.0)
    feat = np.abs(scene.feat.astype(np.float64)).reshape(scene.n, -1, 3).sum(1) + 0.5
    E = [np.stack([np.abs(pp["uv"][:, 0] - cam.cx) + abs(cam.cx), np.abs(pp["uv"][:, 1] - cam.cy) + abs(cam.cy)], 1),
         ((np.abs(A) + np.abs(B) + np.abs(C)) * kap)[:, None].repeat(3, 1), np.abs(pp["opacity"]), feat]
    E = [1e-5 * e + 1e-7 for e in E]
    pimg, pgrad = np.zeros_like(ref["image"]), np.zeros_like(ref["grad2d"])
    for j in np.nonzero(pp["radius"] > 0)[0]:
        for a, arr in enumerate(rec):
            for c in range(1 if arr.ndim == 1 else arr.shape[1]):
                idx = (j,) if arr.ndim == 1 else (j, c)
                keep = arr[idx]
                arr[idx] = keep + E[a][idx]
                o = render(pl, rec)
                arr[idx] = keep
                pimg += np.abs(o["image"] - ref["image"])
                pgrad += np.abs(o["grad2d"] - ref["grad2d"])
    # depth ties within FP32 rounding: the pair swapped in every list
    timg, tgrad = np.zeros_like(pimg), np.zeros_like(pgrad)
    d = pp["depth"]
    pairs = set()
    for t in range(len(ranges)):
        ids = pl[ranges[t, 0]:ranges[t, 1]]
        for a, b in zip(ids[:-1], ids[1:]):
            if d[b] - d[a] <= 32 * EPS32 * abs(d[b]):
                pairs.add((int(a), int(b)))
    for a, b in pairs:
        pl2 = pl.copy()
        for t in range(len(ranges)):
            seg = pl2[ranges[t, 0]:ranges[t, 1]]
            ia, ib = np.nonzero(seg == a)[0], np.nonzero(seg == b)[0]
            if len(ia) and len(ib):
                seg[ia[0]], seg[ib[0]] = b, a
        o = render(pl2, rec)
        timg += np.abs(o["image"] - ref["image"])
        tgrad += np.abs(o["grad2d"] - ref["grad2d"])
    res = dict(pp=pp, ref=ref, pimg=pimg, pgrad=pgrad, timg=timg, tgrad=tgrad, ties=len(pairs))
    _crop_ref[key] = res
    return res


_crop_scene = {}


@pytest.mark.parametrize("store_T", [True, False])
def test_autograd_matches_oracle(dev, orc, store_T):
    if "s" not in _crop_scene:
        _crop_scene["s"] = crop_workload()
    scene, cam = _crop_scene["s"]
    w = weights(cam.height, cam.width)
    bg = (0.1, 0.2, 0.3)
    img, g = run_model(dev, scene, cam, w, store_T, gsr.backward_opts("hybrid", 8, 1, store_T))
    cr = crop_reference(orc, scene, cam, w, bg)
    pp, ref = cr["pp"], cr["ref"]
    assert pp["pp_ambig"].sum() == 0 and (pp["radius"] > 0).sum() > 150
    check_scaled("autograd image", img, ref["image"], np.abs(ref["image"]) * ref["pix_widen"][None],
                 ref["iallow"] + cr["pimg"] + cr["timg"], lit=np.abs(ref["image"]))
    # 3D: 1e-5 of the chain of magnitudes of |grad2d| and of the 2D scale,
    # plus every 2D allowance carried through the same (linear) chain
    bp = orc.backproject(scene, cam, ref["grad2d"])
    mag = lambda x: orc.backproject(scene, cam, x)
    m_g, m_s, m_l = mag(np.abs(ref["grad2d"])), mag(ref["gscale"]), mag(ref["glit"])
    a2 = ref["gallow"] + cr["pgrad"] + cr["tgrad"] + 1e-7
    m_a = mag(a2)
    s64, o64 = scene.scale.astype(np.float64), scene.opacity.astype(np.float64)
    n = scene.n
    do = o64 * (1 - o64)
    expect = {  # name: (reference, scale, allowance, literal scale)
        "mean": (bp["dmean"], m_g["dmean_mag"] + m_s["dmean_mag"], m_a["dmean_mag"],
                 m_g["dmean_mag"] + m_l["dmean_mag"]),
        "log_scale": (bp["dscale"] * s64, (m_g["dscale_mag"] + m_s["dscale_mag"]) * s64, m_a["dscale_mag"] * s64,
                      (m_g["dscale_mag"] + m_l["dscale_mag"]) * s64),
        "quat": (bp["dquat"], m_g["dquat_mag"] + m_s["dquat_mag"], m_a["dquat_mag"],
                 m_g["dquat_mag"] + m_l["dquat_mag"]),
        "opacity_logit": (bp["dopacity"] * do, (np.abs(ref["grad2d"][:, 5]) + ref["gscale"][:, 5]) * do,
                          a2[:, 5] * do, (np.abs(ref["grad2d"][:, 5]) + ref["glit"][:, 5]) * do),
        "feat": (bp["dfeat"].reshape(n, -1), (m_g["dfeat_mag"] + m_s["dfeat_mag"]).reshape(n, -1),
                 m_a["dfeat_mag"].reshape(n, -1), (m_g["dfeat_mag"] + m_l["dfeat_mag"]).reshape(n, -1)),
    }
    ok = pp["bp_ambig"] == 0
    for k, (r, sc, al, lit) in expect.items():
        check_scaled(f"autograd d{k}", g[k][ok], r[ok], sc[ok], al[ok], lit=lit[ok])


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


def test_view_buffers_are_reused_between_steps(dev):
    """The Function takes its view buffers from the settings' pool and gives
    them back in the backward: a training loop allocates them once, and two
    views rendered before one backward keep separate buffers."""
    scene, cam = crop_workload()
    w = torch.from_numpy(weights(cam.height, cam.width)).to(dev)
    model = AG.GaussianModel(scene, dev)
    st = AG.RasterSettings(cam, (0.1, 0.2, 0.3), gsr.backward_opts("warp", 0, 1, True, 2), True, deterministic=True)
    grads = []
    for _ in range(2):
        model.zero_grad(set_to_none=True)
        (model(st) * w).sum().backward()
        grads.append([p.grad.clone() for p in model.parameters()])
    (pool,) = st.pool.values()
    assert len(pool) == 1
    first = pool[0]
    for a, b in zip(*grads):
        assert torch.equal(a, b)
    model.zero_grad(set_to_none=True)
    img1 = model(st)
    img2 = model(st)
    assert len(pool) == 0
    ((img1 + img2) * w).sum().backward()
    assert len(pool) == 2 and any(vb is first for vb in pool)
    torch.testing.assert_close(img1, img2, rtol=0, atol=0)
    for a, p in zip(grads[0], model.parameters()):
        assert torch.equal(p.grad, 2 * a)
