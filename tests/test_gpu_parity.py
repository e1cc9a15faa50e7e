"""CUDA path against the FP64 oracle, stage by stage, element by element.

Each stage of the CUDA library is fed the oracle's own stage inputs (the
oracle's projection rounded to the FP32 record format), so a mismatch points
at exactly one kernel.  Integer and index outputs must agree bit for bit,
except where the oracle shows that FP32 may legitimately decide a comparison
the other way (then the result must be one of the two valid outcomes).
Floating-point outputs: |gpu - oracle| <= 1e-5 * scale + 1e-7 + allowance,
scale = sum of the absolute values of the terms summed (widened where FP32
evaluation of alpha near 1 is ill-conditioned), allowance = difference
between the two valid outcomes of an FP32-ambiguous decision.
"""
import numpy as np
import pytest
import torch

from _helpers import check_scaled, pack_records, records_f64
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


def T(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def N(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


# ----------------------------------------------------------------------------
# workloads (seeded, small enough for the full oracle, several tiles and a
# ragged tail; "dense" has lists longer than one 256-entry batch)
# ----------------------------------------------------------------------------

def workload(name, seed=0):
    if name == "tiny":
        return S.tiny_workload(seed)
    if name == "ragged_sh3":
        return S.gmm_scene(seed, 3000, 16, (-3.5, 0.5), 3), S.front_camera(77, 53)
    if name == "dense_sh1":
        return S.gmm_scene(seed, 20000, 32, (-3.2, 0.4), 1), S.front_camera(200, 150)
    if name == "offaxis_sh2":
        cam = S.look_at_camera((1.5, -1.0, -3.2), (0.1, 0.0, 0.2), 143, 97)
        return S.gmm_scene(seed, 8000, 24, (-3.4, 0.5), 2), cam
    raise KeyError(name)


WORKLOADS = ["tiny", "ragged_sh3", "dense_sh1", "offaxis_sh2"]
_cache = {}


def oracle_stage(orc, name, bg=(0.0, 0.0, 0.0)):
    key = (name, tuple(bg))
    if key in _cache:
        return _cache[key]
    scene, cam = workload(name)
    pp = orc.preprocess(scene, cam)
    rec, radius = pack_records(pp)
    r64 = records_f64(rec)
    keys, pl, ranges = orc.bin_sort(r64["uv"], r64["depth"], radius, cam.width, cam.height)
    g = S.upstream_grad(7, cam.width, cam.height)
    out = orc.render(cam.width, cam.height, ranges, pl, r64["uv"], r64["conic"], r64["opacity"], r64["rgb"],
                     np.asarray(bg, np.float64), g)
    res = dict(scene=scene, cam=cam, pp=pp, rec=rec, radius=radius, keys=keys, pl=pl, ranges=ranges, g=g,
               out=out, bg=np.asarray(bg, np.float32))
    _cache[key] = res
    return res


# ----------------------------------------------------------------------------
# a1: projection
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("name", WORKLOADS)
def test_preprocess_matches_oracle(dev, orc, name):
    scene, cam = workload(name)
    pp = orc.preprocess(scene, cam)
    n = scene.n
    splat = torch.zeros((n, 12), device=dev)
    radius = torch.zeros(n, dtype=torch.int32, device=dev)
    gz = torch.full((n, 12), 7.0, device=dev)
    feat = T(scene.feat.reshape(n, -1))
    gsr.gsr_preprocess(n, scene.sh_degree, T(scene.mean), T(scene.scale), T(scene.quat), T(scene.opacity),
                       feat, cam, 16, 16, splat, radius, gz)
    rec, rad = N(splat), N(radius)
    assert np.all(N(gz) == 0.0)
    amb = pp["pp_ambig"] != 0
    exact = ~amb
    np.testing.assert_array_equal(rad[exact], pp["radius"][exact])
    # ambiguous ones: either the same, a neighbouring ceiling, or the cull flipped
    d = np.abs(rad[amb].astype(np.int64) - pp["radius"][amb])
    assert np.all((d <= 1) | (rad[amb] == 0) | (pp["radius"][amb] == 0))
    vis = (rad > 0) & (pp["radius"] > 0)
    assert vis.sum() > 0.5 * n or name == "offaxis_sh2"
    # u, v: scale = |fx x / z| + |cx|
    for c, cc in ((0, cam.cx), (1, cam.cy)):
        ref = pp["uv"][:, c]
        check_scaled(f"{name} uv{c}", rec[vis, c], ref[vis], np.abs(ref[vis] - cc) + abs(cc))
    # conic: relative to |A|+|B|+|C| times the conditioning of the 2x2 inverse
    A, B, C = pp["conic"][:, 0], pp["conic"][:, 1], pp["conic"][:, 2]
    kap = (np.abs(A * C) + B * B) / (A * C - B * B + 1e-300)
    sc = (np.abs(A) + np.abs(B) + np.abs(C)) * np.maximum(kap, 1.0)
    for j in range(3):
        check_scaled(f"{name} conic{j}", rec[vis, 2 + j], pp["conic"][vis, j], sc[vis])
    np.testing.assert_array_equal(rec[vis, 5], scene.opacity[vis])
    # colour: scale = sum of |SH coefficients| + 0.5 (|Y_lm| <= 1 for degree <= 3)
    f = np.abs(scene.feat.astype(np.float64)).reshape(n, -1, 3).sum(1) + 0.5
    check_scaled(f"{name} rgb", rec[vis, 6:9], pp["rgb"][vis], f[vis])
    # depth: scale = sum |R_z . mean| + |t_z|
    V = cam.view.astype(np.float64)
    zs = np.abs(scene.mean.astype(np.float64)) @ np.abs(V[2, :3]) + abs(V[2, 3])
    check_scaled(f"{name} depth", rec[vis, 9], pp["depth"][vis], zs[vis])
    culled = rad == 0
    assert np.all(rec[culled] == 0.0)


# ----------------------------------------------------------------------------
# a2: binning -- bit-exact
# ----------------------------------------------------------------------------

def gpu_bin(dev, rec, radius, W, H, cap):
    n = len(rec)
    splat, rad = T(rec), T(radius)
    sb = gsr.gsr_bin_scratch_bytes(n, W, H, 16, 16, cap)
    scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
    pl = torch.zeros(max(cap, 1), dtype=torch.int32, device=dev)
    gx, gy = (W + 15) // 16, (H + 15) // 16
    ranges = torch.full((gx * gy, 2), -1, dtype=torch.int32, device=dev)
    keys = torch.zeros(max(cap, 1), dtype=torch.int64, device=dev)
    st, nk = gsr.gsr_bin_sort(n, W, H, 16, 16, splat, rad, cap, scratch, pl, ranges, keys)
    return st, nk, pl, ranges, keys


@pytest.mark.parametrize("name", WORKLOADS)
def test_bin_sort_bit_exact(dev, orc, name):
    st_ = oracle_stage(orc, name)
    cam = st_["cam"]
    nref = len(st_["pl"])
    st, nk, pl, ranges, keys = gpu_bin(dev, st_["rec"], st_["radius"], cam.width, cam.height, nref + 100)
    assert st == gsr.GSR_OK and nk == nref
    np.testing.assert_array_equal(N(keys)[:nk].view(np.uint64), st_["keys"])
    np.testing.assert_array_equal(N(pl)[:nk].view(np.uint32), st_["pl"])
    np.testing.assert_array_equal(N(ranges).view(np.uint32), st_["ranges"])


def test_bin_sort_capacity_overflow_then_regrow(dev, orc):
    st_ = oracle_stage(orc, "tiny")
    cam = st_["cam"]
    nref = len(st_["pl"])
    st, nk, pl, ranges, keys = gpu_bin(dev, st_["rec"], st_["radius"], cam.width, cam.height, nref - 1)
    assert st == gsr.GSR_ECAPACITY and nk == nref
    st, nk, pl, ranges, keys = gpu_bin(dev, st_["rec"], st_["radius"], cam.width, cam.height, nref)
    assert st == gsr.GSR_OK
    np.testing.assert_array_equal(N(pl)[:nk].view(np.uint32), st_["pl"])


# ----------------------------------------------------------------------------
# a3: forward blend
# ----------------------------------------------------------------------------

def gpu_forward(dev, st_):
    cam = st_["cam"]
    W, H = cam.width, cam.height
    image = torch.zeros((3, H, W), device=dev)
    fT = torch.zeros((H, W), device=dev)
    nc = torch.zeros((H, W), dtype=torch.int32, device=dev)
    ranges = T(st_["ranges"].view(np.int32))
    pl = T(np.concatenate([st_["pl"], [0]]).astype(np.uint32).view(np.int32))
    splat = T(st_["rec"])
    gsr.gsr_forward(W, H, 16, 16, ranges, pl, splat, st_["bg"], image, fT, nc)
    return dict(image=image, final_T=fT, n_contrib=nc, ranges=ranges, pl=pl, splat=splat)


def check_forward(name, got, out):
    check_scaled(f"{name} image", got["image"], out["image"], np.abs(out["image"]) * out["pix_widen"][None],
                 out["iallow"], lit=np.abs(out["image"]))
    check_scaled(f"{name} final_T", got["final_T"], out["final_T"],
                 out["final_T"] * np.maximum(1.0, 8 * out["terr"] / 1e-5), out["tallow"], lit=out["final_T"])
    nc = got["n_contrib"]
    ok = (nc == out["n_contrib"]) | ((out["pix_ambig"] > 0) & (nc == out["nc_alt"]))
    assert ok.all(), f"{name} n_contrib: {(~ok).sum()} pixels differ"


@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.3, 0.7, 0.1)])
@pytest.mark.parametrize("name", WORKLOADS)
def test_forward_matches_oracle(dev, orc, name, bg):
    st_ = oracle_stage(orc, name, bg)
    r = gpu_forward(dev, st_)
    got = {k: N(r[k]) for k in ("image", "final_T", "n_contrib")}
    check_forward(name, got, st_["out"])


# ----------------------------------------------------------------------------
# a4-a6: backward blend + gradient accumulation, every tier
# ----------------------------------------------------------------------------

TIERS = [("plain", 0, 0, 1), ("warp", 0, 0, 1), ("warp", 0, 1, 1), ("hybrid", 8, 0, 1), ("hybrid", 16, 1, 1),
         ("hybrid", 33, 0, 1), ("block", 0, 0, 1), ("block", 12, 1, 1),
         ("warp", 0, 0, 2), ("hybrid", 8, 1, 2), ("hybrid", 33, 1, 2), ("block", 0, 1, 2), ("block", 12, 0, 2),
         ("cluster", 0, 0, 1), ("cluster", 12, 1, 1), ("cluster", 0, 1, 2), ("cluster", 8, 0, 2)]


@pytest.mark.parametrize("store_T", [True, False])
@pytest.mark.parametrize("tier", TIERS, ids=lambda t: f"{t[0]}-thr{t[1]}-lay{t[2]}-ppt{t[3]}")
@pytest.mark.parametrize("name", WORKLOADS)
def test_backward_matches_oracle(dev, orc, name, tier, store_T):
    st_ = oracle_stage(orc, name, (0.3, 0.7, 0.1))
    cam = st_["cam"]
    W, H = cam.width, cam.height
    f = gpu_forward(dev, st_)
    n = len(st_["rec"])
    grad = torch.zeros((n, 12), device=dev)
    opts = gsr.backward_opts(tier[0], tier[1], tier[2], store_T, tier[3])
    gsr.gsr_backward(W, H, 16, 16, f["ranges"], f["pl"], f["splat"], st_["bg"],
                     f["final_T"] if store_T else None, f["n_contrib"] if store_T else None,
                     T(st_["g"]), grad, opts)
    got = N(grad)
    out = st_["out"]
    # at most 0.5 % of the elements may need an allowance or the widening
    worst = check_scaled(f"{name} {tier} grad2d", got[:, :9], out["grad2d"], out["gscale"], out["gallow"],
                         lit=out["glit"])
    assert np.all(got[:, 9:] == 0.0)
    print(f"{name} {tier} store_T={store_T}: worst/bound {worst:.3f}")


def test_backward_accumulates_into_existing_values(dev, orc):
    st_ = oracle_stage(orc, "tiny", (0.3, 0.7, 0.1))
    cam = st_["cam"]
    f = gpu_forward(dev, st_)
    n = len(st_["rec"])
    base = torch.randn((n, 12), device=dev)
    grad = base.clone()
    gsr.gsr_backward(cam.width, cam.height, 16, 16, f["ranges"], f["pl"], f["splat"], st_["bg"],
                     f["final_T"], f["n_contrib"], T(st_["g"]), grad, gsr.backward_opts("block", 0))
    out = st_["out"]
    check_scaled("accumulate", N(grad)[:, :9] - N(base)[:, :9], out["grad2d"], out["gscale"] + 10 * np.abs(N(base)[:, :9]),
                 out["gallow"])
    np.testing.assert_array_equal(N(grad)[:, 9:], N(base)[:, 9:])


# ----------------------------------------------------------------------------
# a8: backward projection
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("name", WORKLOADS)
def test_backward_project_matches_oracle(dev, orc, name):
    st_ = oracle_stage(orc, name, (0.3, 0.7, 0.1))
    scene, cam, pp = st_["scene"], st_["cam"], st_["pp"]
    n = scene.n
    g9 = st_["out"]["grad2d"].astype(np.float32)
    g12 = np.zeros((n, 12), np.float32)
    g12[:, :9] = g9
    ref = orc.backproject(scene, cam, g9.astype(np.float64))
    k = scene.feat.reshape(n, -1).shape[1]
    dm, ds, dq = (torch.zeros((n, c), device=dev) for c in (3, 3, 4))
    do = torch.zeros(n, device=dev)
    df = torch.zeros((n, k), device=dev)
    gsr.gsr_backward_project(n, scene.sh_degree, T(scene.mean), T(scene.scale), T(scene.quat),
                             T(scene.opacity), T(scene.feat.reshape(n, -1)), cam, T(st_["radius"]), T(g12),
                             dm, ds, dq, do, df)
    ok = (pp["bp_ambig"] == 0) & (pp["pp_ambig"] == 0)
    vis = (st_["radius"] > 0) & ok
    for key, got, mag in (("dmean", dm, "dmean_mag"), ("dscale", ds, "dscale_mag"), ("dquat", dq, "dquat_mag"),
                          ("dfeat", df, "dfeat_mag")):
        r = ref[key].reshape(n, -1)
        m = ref[mag].reshape(n, -1)
        check_scaled(f"{name} {key}", N(got)[vis], r[vis], m[vis])
    np.testing.assert_allclose(N(do)[vis], g9[vis, 5], rtol=0, atol=0)
    assert np.all(N(dm)[st_["radius"] == 0] == 0)


@pytest.mark.parametrize("name", WORKLOADS)
def test_backward_project_store_overwrites(dev, orc, name):
    """The store variant writes every output (old contents irrelevant): equal
    to the accumulating call on zeroed buffers, zero for culled Gaussians."""
    st_ = oracle_stage(orc, name, (0.3, 0.7, 0.1))
    scene, cam = st_["scene"], st_["cam"]
    n = scene.n
    g12 = np.zeros((n, 12), np.float32)
    g12[:, :9] = st_["out"]["grad2d"].astype(np.float32)
    k = scene.feat.reshape(n, -1).shape[1]
    args = (n, scene.sh_degree, T(scene.mean), T(scene.scale), T(scene.quat), T(scene.opacity),
            T(scene.feat.reshape(n, -1)), cam, T(st_["radius"]), T(g12))
    acc = [torch.zeros((n, c), device=dev) for c in (3, 3, 4)] + [torch.zeros(n, device=dev),
                                                                 torch.zeros((n, k), device=dev)]
    sto = [torch.full_like(t, 7.25) for t in acc]
    gsr.gsr_backward_project(*args, *acc)
    gsr.gsr_backward_project(*args, *sto, accumulate=False)
    for a, b in zip(acc, sto):
        np.testing.assert_array_equal(N(a), N(b))
    assert np.all(N(sto[4])[st_["radius"] == 0] == 0.0)


# ----------------------------------------------------------------------------
# edge cases
# ----------------------------------------------------------------------------

def _run_all(dev, scene, cam, bg=(0.2, 0.4, 0.6)):
    from paper_2401_05345_gb300 import pipeline
    sc = pipeline.SceneTensors.from_scene(scene, dev)
    vb = pipeline.ViewBuffers(scene.n, cam, dev, key_capacity=16)
    vb.preprocess(sc)
    vb.bin()
    vb.forward(bg)
    g = T(S.upstream_grad(1, cam.width, cam.height))
    vb.backward(bg, g, gsr.backward_opts("hybrid", 8))
    grads = sc.zeros_like_params()
    vb.backward_project(sc, grads)
    torch.cuda.synchronize()
    return vb, grads


def test_empty_scene_renders_background(dev):
    cam = S.front_camera(40, 24)
    scene = S.uniform_scene(0, 1).subset(slice(0, 0))
    vb, grads = _run_all(dev, scene, cam)
    assert vb.n_keys == 0
    img = N(vb.image)
    np.testing.assert_array_equal(img, np.broadcast_to(np.float32([0.2, 0.4, 0.6])[:, None, None], img.shape))
    assert np.all(N(vb.final_T) == 1.0) and np.all(N(vb.n_contrib) == 0)


def test_everything_behind_the_camera(dev):
    cam = S.front_camera(48, 48)
    scene = S.uniform_scene(1, 200)
    scene.mean[:, 2] = -6.0  # z_cam = -2
    vb, grads = _run_all(dev, scene, cam)
    assert vb.n_keys == 0 and np.all(N(vb.radius) == 0)
    assert np.all(N(vb.grad2d)[:, :9] == 0) and np.all(N(grads.mean) == 0)


def test_splat_covering_every_tile(dev, orc):
    cam = S.front_camera(100, 70)
    scene = S.uniform_scene(2, 3)
    scene.mean[:] = [[0.0, 0.0, 0.0], [0.05, 0.02, -0.5], [0.3, -0.2, 1.0]]
    scene.scale[:] = [[1.5, 1.2, 1.0], [0.05, 0.05, 0.05], [0.4, 0.9, 0.2]]
    vb, _ = _run_all(dev, scene, cam)
    pp = orc.preprocess(scene, cam)
    assert vb.n_keys >= vb.gx * vb.gy
    assert pp["radius"][0] > 50


def test_capacity_growth_in_pipeline(dev):
    scene, cam = S.tiny_workload(3)
    vb, _ = _run_all(dev, scene, cam)
    assert vb.key_capacity >= vb.n_keys > 16


def test_invalid_arguments_raise(dev):
    cam = S.front_camera(32, 32)
    x = torch.zeros(16, device=dev)
    with pytest.raises(gsr.GsrError, match="invalid"):
        gsr.gsr_forward(32, 32, 16, 8, x, x, x, (0, 0, 0), x)
    with pytest.raises(gsr.GsrError, match="invalid"):
        gsr.gsr_preprocess(4, 5, x, x, x, x, x, cam, 16, 16, x, x)


def test_unaligned_features_take_the_scalar_path(dev):
    """Feature and quaternion arrays at any 4-byte offset (e.g. segments of a
    packed parameter buffer) give the same projection and backward
    projection, bit for bit.  Features 32-byte aligned take the projection's
    32-byte register loads, 16-byte aligned its 16-byte ones, others the
    scalar staging; quaternions 16-byte aligned take one 16-byte load, others
    four scalar ones (1001 Gaussians: the last chunk is ragged)."""
    scene = S.gmm_scene(9, 1001, 8, (-3.3, 0.4), 3)
    cam = S.front_camera(96, 80)
    n = scene.n
    feat = scene.feat.reshape(n, -1)

    def at_offset(a, off):  # a copy of a starting `off` floats into a fresh (256-byte aligned) buffer
        buf = torch.zeros(a.size + off, device=dev)
        buf[off:] = torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to(dev)
        return buf[off:]

    outs = []
    for foff, qoff in ((0, 0), (4, 0), (1, 1), (0, 1)):
        f = at_offset(feat, foff).view(n, -1)
        q = at_offset(scene.quat, qoff).view(n, 4)
        assert (f.data_ptr() % 32 == 0) == (foff == 0) and (f.data_ptr() % 16 == 0) == (foff % 4 == 0)
        splat = torch.zeros((n, 12), device=dev)
        radius = torch.zeros(n, dtype=torch.int32, device=dev)
        gsr.gsr_preprocess(n, 3, T(scene.mean), T(scene.scale), q, T(scene.opacity), f, cam, 16, 16, splat, radius)
        g12 = torch.ones((n, 12), device=dev)
        df = at_offset(np.zeros(feat.size, np.float32), foff)
        z = lambda c: torch.zeros((n, c), device=dev)
        dm, ds, dq, do = z(3), z(3), z(4), torch.zeros(n, device=dev)
        gsr.gsr_backward_project(n, 3, T(scene.mean), T(scene.scale), q, T(scene.opacity), f, cam, radius, g12, dm,
                                 ds, dq, do, df)
        outs.append((N(splat), N(radius), N(df), N(dm), N(dq)))
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("ppt,layout", [(1, 0), (1, 1), (2, 0), (2, 1)])
@pytest.mark.parametrize("name", WORKLOADS)
def test_deterministic_backward_matches_oracle_and_repeats_bitwise(dev, orc, name, ppt, layout):
    """The atomic-free tier: oracle parity, and the same bits on every run and
    whether T is stored or recomputed."""
    st_ = oracle_stage(orc, name, (0.3, 0.7, 0.1))
    cam = st_["cam"]
    W, H = cam.width, cam.height
    f = gpu_forward(dev, st_)
    n = len(st_["rec"])
    radius = T(st_["radius"])
    off = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    scr = torch.empty(gsr.gsr_entry_offsets_scratch_bytes(n), dtype=torch.uint8, device=dev)
    gsr.gsr_entry_offsets(n, W, H, 16, 16, f["splat"], radius, scr, off)
    nk = int(off[n])
    assert nk == len(st_["pl"])
    partial = torch.full((9 * nk + 9,), float("nan"), device=dev)   # every slot must be written
    outs = []
    for store_T in (True, True, False):
        grad = torch.zeros((n, 12), device=dev)
        gsr.gsr_backward_deterministic(W, H, 16, 16, f["ranges"], f["pl"], f["splat"], radius, n, off, st_["bg"],
                                       f["final_T"] if store_T else None, f["n_contrib"] if store_T else None,
                                       T(st_["g"]), partial, grad, gsr.backward_opts("warp", 0, layout, store_T, ppt))
        outs.append(N(grad))
    out = st_["out"]
    check_scaled(f"{name} deterministic", outs[0][:, :9], out["grad2d"], out["gscale"], out["gallow"])
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])


def test_deterministic_backward_leaves_everything_when_partial_is_too_small(dev, orc):
    """A partial buffer one entry short of the view's entry count: neither
    kernel writes (grad2d keeps its values, partial its contents)."""
    st_ = oracle_stage(orc, "tiny", (0.3, 0.7, 0.1))
    cam = st_["cam"]
    f = gpu_forward(dev, st_)
    n = len(st_["rec"])
    radius = T(st_["radius"])
    off = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    scr = torch.empty(gsr.gsr_entry_offsets_scratch_bytes(n), dtype=torch.uint8, device=dev)
    gsr.gsr_entry_offsets(n, cam.width, cam.height, 16, 16, f["splat"], radius, scr, off)
    nk = int(off[n])
    partial = torch.full((9 * (nk - 1),), 7.0, device=dev)
    grad = torch.full((n, 12), 3.0, device=dev)
    gsr.gsr_backward_deterministic(cam.width, cam.height, 16, 16, f["ranges"], f["pl"], f["splat"], radius, n, off,
                                   st_["bg"], f["final_T"], f["n_contrib"], T(st_["g"]), partial, grad)
    torch.cuda.synchronize()
    assert bool((grad == 3.0).all()) and bool((partial == 7.0).all())
    assert not np.isnan(N(partial)[:9 * nk]).any()


def _order_bucket(lens):
    """Bucket of gsr_tile_order, written from its definition: floor(log2 len)
    and the next two bits below the leading one (0 for an empty list)."""
    out = np.zeros(len(lens), np.int64)
    for i, n in enumerate(int(x) for x in lens):
        if n == 0:
            continue
        l2 = n.bit_length() - 1
        out[i] = 1 + l2 if l2 < 2 else 4 * l2 + ((n >> (l2 - 2)) & 3)
    return out


@pytest.mark.parametrize("name", WORKLOADS)
def test_tile_order_changes_no_result(dev, orc, name):
    """gsr_tile_order gives a permutation of the tiles with non-increasing
    list-length buckets; the forward taking tiles in that order writes the
    same bits, the atomic backward stays within the oracle tolerance and the
    deterministic backward writes the same bits."""
    st_ = oracle_stage(orc, name, (0.3, 0.7, 0.1))
    cam = st_["cam"]
    W, H = cam.width, cam.height
    tiles = ((W + 15) // 16) * ((H + 15) // 16)
    f = gpu_forward(dev, st_)
    order = torch.full((tiles,), -1, dtype=torch.int32, device=dev)
    gsr.gsr_tile_order(W, H, 16, 16, f["ranges"], order)
    o = N(order)
    assert sorted(o.tolist()) == list(range(tiles))
    rg = st_["ranges"].astype(np.int64).reshape(-1, 2)
    b = _order_bucket(rg[o, 1] - rg[o, 0])
    assert np.all(np.diff(b) <= 0)
    # forward: bit for bit
    image = torch.zeros_like(f["image"])
    fT = torch.zeros_like(f["final_T"])
    nc = torch.zeros_like(f["n_contrib"])
    gsr.gsr_forward(W, H, 16, 16, f["ranges"], f["pl"], f["splat"], st_["bg"], image, fT, nc, tile_order=order)
    for a, c in ((image, f["image"]), (fT, f["final_T"]), (nc, f["n_contrib"])):
        assert torch.equal(a, c)
    # atomic backward: oracle tolerance
    n = len(st_["rec"])
    out = st_["out"]
    for opts in (gsr.backward_opts("hybrid", 12, 1, True, 2), gsr.backward_opts("plain", 0, 1, True, 1)):
        grad = torch.zeros((n, 12), device=dev)
        gsr.gsr_backward(W, H, 16, 16, f["ranges"], f["pl"], f["splat"], st_["bg"], f["final_T"], f["n_contrib"],
                         T(st_["g"]), grad, opts, tile_order=order)
        check_scaled(f"{name} ordered backward", N(grad)[:, :9], out["grad2d"], out["gscale"], out["gallow"])
    # deterministic backward: the same bits in either order
    radius = T(st_["radius"])
    off = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    scr = torch.empty(gsr.gsr_entry_offsets_scratch_bytes(n), dtype=torch.uint8, device=dev)
    gsr.gsr_entry_offsets(n, W, H, 16, 16, f["splat"], radius, scr, off)
    partial = torch.empty(9 * int(off[n]) + 9, device=dev)
    res = []
    for tord in (None, order):
        grad = torch.zeros((n, 12), device=dev)
        gsr.gsr_backward_deterministic(W, H, 16, 16, f["ranges"], f["pl"], f["splat"], radius, n, off, st_["bg"],
                                       f["final_T"], f["n_contrib"], T(st_["g"]), partial, grad, tile_order=tord)
        res.append(N(grad))
    np.testing.assert_array_equal(res[0], res[1])


@pytest.mark.parametrize("name", ["tiny", "dense_sh1", "offaxis_sh2"])
def test_forward_block_masks(dev, orc, name):
    """Block masks written by the forward: every entry the forward reads
    (at least every list position up to the tile's furthest last
    contributor) gets a mask with bits 4..7 clear, and a clear bit is a
    correct cull: in FP64 on the oracle's records, no pixel of that 8x8
    block reaches alpha >= 1/255.  Backward results with the masks: the
    deterministic tier gives the same bits as without them (stored and
    recomputed transmittance), the hybrid tier matches the oracle."""
    st_ = oracle_stage(orc, name, (0.3, 0.7, 0.1))
    cam = st_["cam"]
    W, H = cam.width, cam.height
    gx, gy = (W + 15) // 16, (H + 15) // 16
    f = gpu_forward(dev, st_)
    nk = len(st_["pl"])
    mask = torch.full((nk + 1,), 0xAA, dtype=torch.uint8, device=dev)  # 0xAA: bits 5 and 7 mark "not written"
    image = torch.zeros_like(f["image"])
    fT = torch.zeros_like(f["final_T"])
    nc = torch.zeros_like(f["n_contrib"])
    gsr.gsr_forward(W, H, 16, 16, f["ranges"], f["pl"], f["splat"], st_["bg"], image, fT, nc, block_mask=mask)
    for a, c in ((image, f["image"]), (fT, f["final_T"]), (nc, f["n_contrib"])):
        assert torch.equal(a, c)  # writing the masks changes no output
    m = N(mask)[:nk].astype(np.int64)
    ncn = N(f["n_contrib"])
    rec = st_["rec"].astype(np.float64)
    pl = st_["pl"].astype(np.int64)
    rg = st_["ranges"].astype(np.int64).reshape(-1, 2)
    culled = 0
    for t in range(gx * gy):
        s0, s1 = rg[t]
        if s1 == s0:
            continue
        tx, ty = t % gx, t // gx
        reach = int(ncn[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16].max())
        written = m[s0:s1] & 0xF0 == 0
        assert written[:reach].all(), f"tile {t}: an entry before the last contributor has no mask"
        for b in range(4):
            x0, y0 = tx * 16 + 8 * (b & 1), ty * 16 + 8 * (b >> 1)
            xs = np.arange(x0, min(x0 + 8, W), dtype=np.float64)
            ys = np.arange(y0, min(y0 + 8, H), dtype=np.float64)
            if len(xs) == 0 or len(ys) == 0:
                continue
            sel = np.nonzero(written & ((m[s0:s1] >> b) & 1 == 0))[0]
            if len(sel) == 0:
                continue
            r = rec[pl[s0 + sel]]
            dx = r[:, 0, None, None] - xs[None, None, :]
            dy = r[:, 1, None, None] - ys[None, :, None]
            sig = 0.5 * (r[:, 2, None, None] * dx * dx + r[:, 4, None, None] * dy * dy) + r[:, 3, None, None] * dx * dy
            alpha = np.minimum(0.99, r[:, 5, None, None] * np.exp(-sig))
            passes = (sig >= 0) & (alpha >= 1.0 / 255.0)
            assert not passes.any(), f"tile {t} block {b}: a culled entry reaches alpha >= 1/255"
            culled += len(sel)
    assert culled > 0
    n = len(st_["rec"])
    out = st_["out"]
    grad = torch.zeros((n, 12), device=dev)
    gsr.gsr_backward(W, H, 16, 16, f["ranges"], f["pl"], f["splat"], st_["bg"], f["final_T"], f["n_contrib"],
                     T(st_["g"]), grad, gsr.backward_opts("hybrid", 12, 1, True, 2), block_mask=mask)
    check_scaled(f"{name} backward with block masks", N(grad)[:, :9], out["grad2d"], out["gscale"], out["gallow"])
    radius = T(st_["radius"])
    off = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    scr = torch.empty(gsr.gsr_entry_offsets_scratch_bytes(n), dtype=torch.uint8, device=dev)
    gsr.gsr_entry_offsets(n, W, H, 16, 16, f["splat"], radius, scr, off)
    partial = torch.empty(9 * int(off[n]) + 9, device=dev)
    for store_T in (True, False):
        opts = gsr.backward_opts("warp", 0, 1, store_T, 2)
        res = []
        for bm in (None, mask):
            grad = torch.zeros((n, 12), device=dev)
            gsr.gsr_backward_deterministic(W, H, 16, 16, f["ranges"], f["pl"], f["splat"], radius, n, off, st_["bg"],
                                           f["final_T"], f["n_contrib"], T(st_["g"]), partial, grad, opts,
                                           block_mask=bm)
            res.append(N(grad))
        np.testing.assert_array_equal(res[0], res[1])


def test_tile_ids_outside_the_grid_are_skipped(dev, orc):
    """An order whose entries are all past the last tile renders nothing:
    the outputs keep their values (no access outside the grid)."""
    st_ = oracle_stage(orc, "tiny", (0.3, 0.7, 0.1))
    cam = st_["cam"]
    W, H = cam.width, cam.height
    tiles = ((W + 15) // 16) * ((H + 15) // 16)
    f = gpu_forward(dev, st_)
    bad = torch.arange(tiles, 2 * tiles, dtype=torch.int32, device=dev)
    image = torch.full_like(f["image"], 5.0)
    gsr.gsr_forward(W, H, 16, 16, f["ranges"], f["pl"], f["splat"], st_["bg"], image, None, None, tile_order=bad)
    n = len(st_["rec"])
    grad = torch.full((n, 12), 3.0, device=dev)
    gsr.gsr_backward(W, H, 16, 16, f["ranges"], f["pl"], f["splat"], st_["bg"], f["final_T"], f["n_contrib"],
                     T(st_["g"]), grad, gsr.backward_opts("hybrid", 12, 1, True, 2), tile_order=bad)
    torch.cuda.synchronize()
    assert bool((image == 5.0).all()) and bool((grad == 3.0).all())


@pytest.mark.parametrize("name", ["tiny", "ragged_sh3", "dense_sh1"])
def test_forward_with_l1_equals_forward_then_l1(dev, orc, name):
    """gsr_forward_l1 writes the image, transmittance, contributor counts
    and loss gradient of gsr_forward followed by gsr_l1_loss bit for bit,
    and the same loss within the 1e-5 relative tolerance of float sums in
    another order; without an image buffer it writes the same gradient."""
    st_ = oracle_stage(orc, name, (0.3, 0.7, 0.1))
    cam = st_["cam"]
    W, H = cam.width, cam.height
    f = gpu_forward(dev, st_)
    tiles = ((W + 15) // 16) * ((H + 15) // 16)
    order = torch.empty(tiles, dtype=torch.int32, device=dev)
    gsr.gsr_tile_order(W, H, 16, 16, f["ranges"], order)
    target = T(S.target_image(3, W, H))
    dref = torch.empty_like(f["image"])
    lref = torch.zeros(1, device=dev)
    gsr.gsr_l1_loss(dref.numel(), f["image"], target, dref, lref)
    image = torch.zeros_like(f["image"])
    fT = torch.zeros_like(f["final_T"])
    nc = torch.zeros_like(f["n_contrib"])
    dimg = torch.full_like(f["image"], 7.0)
    loss = torch.zeros(1, device=dev)
    gsr.gsr_forward_l1(W, H, 16, 16, f["ranges"], f["pl"], f["splat"], st_["bg"], target, image, fT, nc, dimg, loss,
                       tile_order=order)
    for a, b in ((image, f["image"]), (fT, f["final_T"]), (nc, f["n_contrib"]), (dimg, dref)):
        assert torch.equal(a, b)
    assert float(loss) == pytest.approx(float(lref), rel=1e-5)
    dimg2 = torch.full_like(f["image"], 7.0)
    gsr.gsr_forward_l1(W, H, 16, 16, f["ranges"], f["pl"], f["splat"], st_["bg"], target, None, None, None, dimg2)
    assert torch.equal(dimg2, dref)
