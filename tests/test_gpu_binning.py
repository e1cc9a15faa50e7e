"""The hand-written binning (depth radix sort + tile counting sort) against
the oracle's key sort, bit for bit, on synthetic splat records that stress
what a sort can get wrong: equal depths (stability, id order), culled and
off-screen splats, ragged sizes around the sort's 2048-key tiles, tile
grids larger than one window of the counting sort (8x8 tiles at
4000x840: 500 x 105 tiles, seven row windows of the counts and seven
placement windows; at 70000x16 a tile row of 8750 tiles is longer than a
window), non-square tiles,
splats larger than the image.  The CUB-based
comparison entry point must give the same bytes."""
import numpy as np
import pytest
import torch

from paper_2401_05345_gb300 import gsr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_05345_gb300 import build
    build.build()
    gsr.lib()
    return torch.device("cuda")


def records(seed, n, W, H, depth_levels=0, culled=0.1, rmax=40, big=0):
    """FP32 splat records (only u, v and depth matter to binning) and radii."""
    rng = np.random.default_rng(seed)
    rec = np.zeros((n, 12), np.float32)
    rec[:, 0] = rng.uniform(-60, W + 60, n)
    rec[:, 1] = rng.uniform(-60, H + 60, n)
    if depth_levels:
        rec[:, 9] = rng.integers(0, depth_levels, n).astype(np.float32) * 0.25 + 2.0
    else:
        rec[:, 9] = rng.uniform(0.3, 12.0, n).astype(np.float32)
    radius = rng.integers(1, rmax + 1, n).astype(np.int32)
    if big:
        radius[rng.choice(n, big, replace=False)] = max(W, H)
    radius[rng.random(n) < culled] = 0
    rec[radius == 0] = 0.0
    return rec, radius


def run_bin(dev, rec, radius, W, H, tw, th, library=False, cap=None):
    n = len(radius)
    gx, gy = (W + tw - 1) // tw, (H + th - 1) // th
    if cap is None:
        cap = 1 << 16
    splat = torch.from_numpy(np.ascontiguousarray(rec)).to(dev)
    rad = torch.from_numpy(radius).to(dev)
    while True:
        sb = gsr.gsr_bin_scratch_bytes(n, W, H, tw, th, cap, library=library)
        scratch = torch.empty(max(sb, 1), dtype=torch.uint8, device=dev)
        pl = torch.zeros(max(cap, 1), dtype=torch.int32, device=dev)
        ranges = torch.full((gx * gy, 2), -1, dtype=torch.int32, device=dev)
        keys = torch.zeros(max(cap, 1), dtype=torch.int64, device=dev)
        st, nk = gsr.gsr_bin_sort(n, W, H, tw, th, splat, rad, cap, scratch, pl, ranges, keys, library=library)
        if st == gsr.GSR_ECAPACITY:
            cap = nk
            continue
        torch.cuda.synchronize()
        return (nk, pl.cpu().numpy()[:nk].view(np.uint32), ranges.cpu().numpy().view(np.uint32),
                keys.cpu().numpy()[:nk].view(np.uint64))


def oracle_bin(orc, rec, radius, W, H, tw, th):
    r = rec.astype(np.float64)
    return orc.bin_sort(r[:, 0:2].copy(), r[:, 9].copy(), radius, W, H, (tw, th))


CASES = [
    # name, seed, n, W, H, tile, depth levels, culled fraction, big splats
    ("ties_ragged", 0, 9_000, 300, 200, (16, 16), 5, 0.1, 0),
    ("one_key_tile", 1, 4096, 128, 96, (16, 16), 0, 0.0, 0),
    ("one_over_tile", 2, 4097, 128, 96, (16, 16), 3, 0.2, 0),
    ("single", 6, 1, 64, 64, (16, 16), 0, 0.0, 0),
    ("row_windows_8x8", 4, 60_000, 4000, 840, (8, 8), 0, 0.1, 3),
    ("row_windows_ties", 5, 30_000, 4000, 840, (8, 8), 2, 0.05, 0),
    ("tiles_32x16", 6, 20_000, 500, 333, (32, 16), 7, 0.1, 2),
    ("tiles_8x32", 7, 20_000, 333, 500, (8, 32), 0, 0.1, 1),
    ("many_radix_tiles", 8, 150_000, 800, 800, (16, 16), 40, 0.3, 0),
    ("row_longer_than_a_window", 9, 20_000, 70_000, 16, (8, 8), 0, 0.1, 2),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_own_binning_matches_oracle_bit_for_bit(dev, orc, case):
    name, seed, n, W, H, (tw, th), levels, culled, big = case
    rec, radius = records(seed, n, W, H, levels, culled, big=big)
    keys_ref, pl_ref, ranges_ref = oracle_bin(orc, rec, radius, W, H, tw, th)
    nk, pl, ranges, keys = run_bin(dev, rec, radius, W, H, tw, th)
    assert nk == len(pl_ref)
    np.testing.assert_array_equal(keys, keys_ref[:nk])
    np.testing.assert_array_equal(pl, pl_ref)
    np.testing.assert_array_equal(ranges, ranges_ref)


@pytest.mark.parametrize("case", CASES[:5], ids=lambda c: c[0])
def test_library_binning_gives_the_same_bytes(dev, case):
    name, seed, n, W, H, (tw, th), levels, culled, big = case
    rec, radius = records(seed, n, W, H, levels, culled, big=big)
    own = run_bin(dev, rec, radius, W, H, tw, th)
    lib = run_bin(dev, rec, radius, W, H, tw, th, library=True)
    assert own[0] == lib[0]
    for a, b in zip(own[1:], lib[1:]):
        np.testing.assert_array_equal(a, b)


def test_all_culled_and_empty(dev):
    W, H = 100, 60
    rec, radius = records(9, 5000, W, H, culled=1.0)
    nk, pl, ranges, keys = run_bin(dev, rec, radius, W, H, 16, 16)
    assert nk == 0 and np.all(ranges == 0)
    nk, pl, ranges, keys = run_bin(dev, rec[:0], radius[:0], W, H, 16, 16)
    assert nk == 0 and np.all(ranges == 0)


def test_capacity_error_then_exact_fit(dev, orc):
    W, H = 200, 120
    rec, radius = records(10, 3000, W, H, 4)
    keys_ref, pl_ref, ranges_ref = oracle_bin(orc, rec, radius, W, H, 16, 16)
    n = len(radius)
    cap = len(pl_ref) - 1
    sb = gsr.gsr_bin_scratch_bytes(n, W, H, 16, 16, cap)
    scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
    pl = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    ranges = torch.zeros((((W + 15) // 16) * ((H + 15) // 16), 2), dtype=torch.int32, device=dev)
    st, nk = gsr.gsr_bin_sort(n, W, H, 16, 16, torch.from_numpy(rec).to(dev), torch.from_numpy(radius).to(dev),
                              cap, scratch, pl, ranges)
    assert st == gsr.GSR_ECAPACITY and nk == len(pl_ref)
    assert np.all(pl.cpu().numpy() == -7)  # nothing written past the count check
    out = run_bin(dev, rec, radius, W, H, 16, 16, cap=len(pl_ref))
    np.testing.assert_array_equal(out[1], pl_ref)


def test_repeated_calls_reuse_scratch(dev, orc):
    """Scratch contents left by one call (count matrices, done counter) must
    not leak into the next, with a different scene in the same buffers."""
    W, H = 300, 200
    n = 12_000
    sb = gsr.gsr_bin_scratch_bytes(n, W, H, 16, 16, 1 << 18)
    scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
    pl = torch.zeros(1 << 18, dtype=torch.int32, device=dev)
    ranges = torch.zeros((19 * 13, 2), dtype=torch.int32, device=dev)
    for seed in (11, 12, 11):
        rec, radius = records(seed, n, W, H, 6)
        keys_ref, pl_ref, ranges_ref = oracle_bin(orc, rec, radius, W, H, 16, 16)
        st, nk = gsr.gsr_bin_sort(n, W, H, 16, 16, torch.from_numpy(rec).to(dev), torch.from_numpy(radius).to(dev),
                                  1 << 18, scratch, pl, ranges)
        assert st == gsr.GSR_OK and nk == len(pl_ref)
        np.testing.assert_array_equal(pl.cpu().numpy()[:nk].view(np.uint32), pl_ref)
        np.testing.assert_array_equal(ranges.cpu().numpy().view(np.uint32), ranges_ref)


@pytest.mark.parametrize("case", CASES[:6], ids=lambda c: c[0])
def test_async_binning_matches_sync(dev, case):
    name, seed, n, W, H, (tw, th), levels, culled, big = case
    rec, radius = records(seed, n, W, H, levels, culled, big=big)
    nk, pl, ranges, keys = run_bin(dev, rec, radius, W, H, tw, th)
    cap = max(nk, 1)
    sb = gsr.gsr_bin_scratch_bytes(n, W, H, tw, th, cap)
    scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
    gx, gy = (W + tw - 1) // tw, (H + th - 1) // th
    apl = torch.zeros(cap, dtype=torch.int32, device=dev)
    arg = torch.full((gx * gy, 2), -1, dtype=torch.int32, device=dev)
    akeys = torch.zeros(cap, dtype=torch.int64, device=dev)
    cnt = torch.full((2,), -1, dtype=torch.int32, device=dev)
    gsr.gsr_bin_sort_async(n, W, H, tw, th, torch.from_numpy(rec).to(dev), torch.from_numpy(radius).to(dev), cap,
                           scratch, apl, arg, cnt, akeys)
    torch.cuda.synchronize()
    assert cnt.cpu().tolist() == [nk, 0]
    np.testing.assert_array_equal(apl.cpu().numpy()[:nk].view(np.uint32), pl)
    np.testing.assert_array_equal(arg.cpu().numpy().view(np.uint32), ranges)
    np.testing.assert_array_equal(akeys.cpu().numpy()[:nk].view(np.uint64), keys)


def test_async_binning_over_capacity_leaves_empty_lists(dev):
    W, H = 300, 200
    rec, radius = records(21, 9000, W, H, 3)
    nk = run_bin(dev, rec, radius, W, H, 16, 16)[0]
    cap = nk - 5
    n = len(radius)
    sb = gsr.gsr_bin_scratch_bytes(n, W, H, 16, 16, cap)
    scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
    pl = torch.full((cap,), -3, dtype=torch.int32, device=dev)
    ranges = torch.full((19 * 13, 2), 7, dtype=torch.int32, device=dev)
    cnt = torch.zeros(2, dtype=torch.int32, device=dev)
    gsr.gsr_bin_sort_async(n, W, H, 16, 16, torch.from_numpy(rec).to(dev), torch.from_numpy(radius).to(dev), cap,
                           scratch, pl, ranges, cnt)
    torch.cuda.synchronize()
    assert cnt.cpu().tolist() == [nk, 1]
    assert np.all(ranges.cpu().numpy() == 0)
    assert np.all(pl.cpu().numpy() == -3)


def test_renderer_step_with_async_binning(dev):
    """A whole step with asynchronous binning equals the synchronous one, and
    an undersized key buffer is reported and grown by check_bin."""
    from paper_2401_05345_gb300 import pipeline
    from paper_2401_05345_gb300 import scenes as S
    scene, cam = S.tiny_workload(4)
    sc = pipeline.SceneTensors.from_scene(scene, dev)
    target = torch.from_numpy(S.target_image(4, cam.width, cam.height)).to(dev)
    out = []
    for sync in (True, False):
        R = pipeline.Renderer(scene.n, cam, dev, key_capacity=64)
        grads = sc.zeros_like_params()
        if not sync:
            R.step(sc, target, (0.1, 0.2, 0.3), grads, sync_bin=False)
            torch.cuda.synchronize()
            assert not R.vb.check_bin()      # 64 keys are too few: reported, buffers grown
            grads = sc.zeros_like_params()
            R.step(sc, target, (0.1, 0.2, 0.3), grads, sync_bin=False)
            torch.cuda.synchronize()
            assert R.vb.check_bin()
        else:
            R.step(sc, target, (0.1, 0.2, 0.3), grads)
        torch.cuda.synchronize()
        out.append((R.vb.image.cpu().numpy(), [t.cpu().numpy() for t in grads.tensors()]))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):  # float atomics: only the summation order differs
        assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max() + 1e-7
