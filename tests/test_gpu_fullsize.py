"""Parity at the benchmark's full size (500k Gaussians, SH degree 3, 1297x840)
in the launch configurations the benchmark times, on sampled outputs.

Every stage gets the oracle's own stage inputs (as in test_gpu_parity): the
projection is compared for all 500k Gaussians, the binning bit for bit over
all 5.8M keys, the forward on 40 random tiles, the backward on 300 random
visible splats -- the oracle renders exactly the tiles those splats touch, so
their gradients are complete -- and the backward projection for all
Gaussians on the oracle's (partial) gradient records.
"""
import numpy as np
import pytest
import torch

from _helpers import check_scaled, pack_records, records_f64
from paper_2401_05345_gb300 import gsr
from paper_2401_05345_gb300 import scenes as S

pytestmark = pytest.mark.gpu

TIERS = [("plain", 0, 1, 1), ("warp", 0, 1, 1), ("hybrid", 12, 1, 1), ("hybrid", 8, 0, 1), ("block", 0, 1, 1),
         ("hybrid", 12, 1, 2), ("warp", 0, 0, 2), ("block", 0, 1, 2), ("cluster", 12, 1, 2), ("cluster", 0, 0, 1)]
BG = (0.0, 0.0, 0.0)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_05345_gb300 import build
    build.build()
    gsr.lib()
    return torch.device("cuda")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def N(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def full(orc):
    scene, cam = S.single_view_workload(0)
    W, H = cam.width, cam.height
    pp = orc.preprocess(scene, cam)
    rec, radius = pack_records(pp)
    r64 = records_f64(rec)
    keys, pl, ranges = orc.bin_sort(r64["uv"], r64["depth"], radius, W, H)
    rng = np.random.default_rng(123)
    gx, gy = (W + 15) // 16, (H + 15) // 16
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    # sampled splats and every tile they touch; plus sampled tiles
    vis = np.nonzero(radius > 0)[0]
    splats = np.sort(rng.choice(vis, 300, replace=False))
    mask = np.zeros(gx * gy, np.uint8)
    mask[np.unique(tiles[np.isin(pl, splats)])] = 1
    tile_sample = rng.choice(gx * gy, 40, replace=False)
    mask[tile_sample] = 1
    g = S.upstream_grad(11, W, H)
    out = orc.render(W, H, ranges, pl, r64["uv"], r64["conic"], r64["opacity"], r64["rgb"],
                     np.asarray(BG, np.float64), g, tile_mask=mask)
    return dict(scene=scene, cam=cam, pp=pp, rec=rec, radius=radius, keys=keys, pl=pl, ranges=ranges,
                splats=splats, tile_sample=tile_sample, g=g, out=out, gx=gx)


def test_fullsize_projection_all_gaussians(dev, full):
    scene, cam, pp = full["scene"], full["cam"], full["pp"]
    n = scene.n
    splat = torch.zeros((n, 12), device=dev)
    radius = torch.zeros(n, dtype=torch.int32, device=dev)
    gsr.gsr_preprocess(n, 3, T(scene.mean), T(scene.scale), T(scene.quat), T(scene.opacity),
                       T(scene.feat.reshape(n, -1)), cam, 16, 16, splat, radius)
    rec, rad = N(splat), N(radius)
    exact = pp["pp_ambig"] == 0
    assert exact.mean() > 0.999
    np.testing.assert_array_equal(rad[exact], pp["radius"][exact])
    vis = (rad > 0) & (pp["radius"] > 0)
    for c, cc in ((0, cam.cx), (1, cam.cy)):
        ref = pp["uv"][:, c]
        check_scaled(f"uv{c}", rec[vis, c], ref[vis], np.abs(ref[vis] - cc) + abs(cc))
    A, B, C = pp["conic"][:, 0], pp["conic"][:, 1], pp["conic"][:, 2]
    kap = np.maximum((np.abs(A * C) + B * B) / (A * C - B * B + 1e-300), 1.0)
    sc = (np.abs(A) + np.abs(B) + np.abs(C)) * kap
    for j in range(3):
        check_scaled(f"conic{j}", rec[vis, 2 + j], pp["conic"][vis, j], sc[vis])
    f = np.abs(scene.feat.astype(np.float64)).reshape(n, -1, 3).sum(1) + 0.5
    check_scaled("rgb", rec[vis, 6:9], pp["rgb"][vis], f[vis])


def test_fullsize_binning_bit_exact(dev, full):
    cam = full["cam"]
    n = full["scene"].n
    cap = len(full["pl"]) + 1024
    sb = gsr.gsr_bin_scratch_bytes(n, cam.width, cam.height, 16, 16, cap)
    scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
    pl = torch.zeros(cap, dtype=torch.int32, device=dev)
    ranges = torch.zeros((full["gx"] * ((cam.height + 15) // 16), 2), dtype=torch.int32, device=dev)
    keys = torch.zeros(cap, dtype=torch.int64, device=dev)
    st, nk = gsr.gsr_bin_sort(n, cam.width, cam.height, 16, 16, T(full["rec"]), T(full["radius"]), cap, scratch,
                              pl, ranges, keys)
    assert st == gsr.GSR_OK and nk == len(full["pl"]) > 5_000_000
    np.testing.assert_array_equal(N(keys)[:nk].view(np.uint64), full["keys"])
    np.testing.assert_array_equal(N(pl)[:nk].view(np.uint32), full["pl"])
    np.testing.assert_array_equal(N(ranges).view(np.uint32), full["ranges"])


def _forward(dev, full):
    cam = full["cam"]
    W, H = cam.width, cam.height
    image = torch.zeros((3, H, W), device=dev)
    fT = torch.zeros((H, W), device=dev)
    nc = torch.zeros((H, W), dtype=torch.int32, device=dev)
    ranges = T(full["ranges"].view(np.int32))
    pl = T(full["pl"].view(np.int32))
    splat = T(full["rec"])
    gsr.gsr_forward(W, H, 16, 16, ranges, pl, splat, BG, image, fT, nc)
    return image, fT, nc, ranges, pl, splat


def _tile_pixels(full, t):
    W, H = full["cam"].width, full["cam"].height
    tx, ty = t % full["gx"], t // full["gx"]
    return slice(ty * 16, min(H, ty * 16 + 16)), slice(tx * 16, min(W, tx * 16 + 16))


def test_fullsize_forward_on_sampled_tiles(dev, full):
    image, fT, nc, *_ = _forward(dev, full)
    img, ft, ncn = N(image), N(fT), N(nc)
    out = full["out"]
    for t in full["tile_sample"]:
        ys, xs = _tile_pixels(full, t)
        check_scaled(f"image tile {t}", img[:, ys, xs], out["image"][:, ys, xs],
                     np.abs(out["image"][:, ys, xs]) * out["pix_widen"][None, ys, xs], out["iallow"][:, ys, xs],
                     lit=np.abs(out["image"][:, ys, xs]))
        check_scaled(f"final_T tile {t}", ft[ys, xs], out["final_T"][ys, xs],
                     out["final_T"][ys, xs] * np.maximum(1.0, 8 * out["terr"][ys, xs] / 1e-5),
                     out["tallow"][ys, xs], lit=out["final_T"][ys, xs])
        ok = (ncn[ys, xs] == out["n_contrib"][ys, xs]) | (
            (out["pix_ambig"][ys, xs] > 0) & (ncn[ys, xs] == out["nc_alt"][ys, xs]))
        assert ok.all(), f"n_contrib differs in tile {t}"


@pytest.mark.parametrize("tier", TIERS, ids=lambda t: f"{t[0]}-thr{t[1]}-lay{t[2]}-ppt{t[3]}")
def test_fullsize_backward_on_sampled_splats(dev, full, tier):
    cam = full["cam"]
    image, fT, nc, ranges, pl, splat = _forward(dev, full)
    n = full["scene"].n
    grad = torch.zeros((n, 12), device=dev)
    gsr.gsr_backward(cam.width, cam.height, 16, 16, ranges, pl, splat, BG, fT, nc, T(full["g"]), grad,
                     gsr.backward_opts(*tier))
    got = N(grad)[:, :9]
    s = full["splats"]
    out = full["out"]
    assert np.abs(out["grad2d"][s]).max() > 0
    check_scaled(f"grad2d {tier}", got[s], out["grad2d"][s], out["gscale"][s], out["gallow"][s],
                 lit=out["glit"][s])


def test_fullsize_backward_projection(dev, orc, full):
    scene, cam = full["scene"], full["cam"]
    n = scene.n
    g9 = full["out"]["grad2d"].astype(np.float32)   # complete for the sampled splats, partial elsewhere
    g12 = np.zeros((n, 12), np.float32)
    g12[:, :9] = g9
    ref = orc.backproject(scene, cam, g9.astype(np.float64))
    dm, ds, dq = (torch.zeros((n, c), device=dev) for c in (3, 3, 4))
    do = torch.zeros(n, device=dev)
    df = torch.zeros((n, 48), device=dev)
    gsr.gsr_backward_project(n, 3, T(scene.mean), T(scene.scale), T(scene.quat), T(scene.opacity),
                             T(scene.feat.reshape(n, -1)), cam, T(full["radius"]), T(g12), dm, ds, dq, do, df)
    pp = full["pp"]
    ok = (full["radius"] > 0) & (pp["bp_ambig"] == 0) & (pp["pp_ambig"] == 0)
    for key, got, mag in (("dmean", dm, "dmean_mag"), ("dscale", ds, "dscale_mag"), ("dquat", dq, "dquat_mag"),
                          ("dfeat", df, "dfeat_mag")):
        check_scaled(key, N(got)[ok], ref[key].reshape(n, -1)[ok], ref[mag].reshape(n, -1)[ok])


def test_fullsize_deterministic_backward(dev, full):
    cam = full["cam"]
    image, fT, nc, ranges, pl, splat = _forward(dev, full)
    n = full["scene"].n
    radius = T(full["radius"])
    off = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    scr = torch.empty(gsr.gsr_entry_offsets_scratch_bytes(n), dtype=torch.uint8, device=dev)
    gsr.gsr_entry_offsets(n, cam.width, cam.height, 16, 16, splat, radius, scr, off)
    nk = int(off[n])
    partial = torch.empty(9 * nk, device=dev)
    res = []
    for _ in range(2):
        grad = torch.zeros((n, 12), device=dev)
        gsr.gsr_backward_deterministic(cam.width, cam.height, 16, 16, ranges, pl, splat, radius, n, off, BG, fT, nc,
                                       T(full["g"]), partial, grad, gsr.backward_opts("warp", 0, 1, True, 2))
        res.append(N(grad))
    np.testing.assert_array_equal(res[0], res[1])
    s = full["splats"]
    out = full["out"]
    check_scaled("grad2d deterministic", res[0][s, :9], out["grad2d"][s], out["gscale"][s], out["gallow"][s],
                 lit=out["glit"][s])
