"""Longest-first tile order on a grid of more than 65,536 tiles (4112 x 4112
pixels, 257 x 257 tiles): the order is a permutation of the tile ids with
non-increasing list-length buckets, and the forward and the deterministic
backward give the same bits whichever order the CTAs take tiles in."""
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


def _bucket(n):
    """Bucket of gsr_tile_order, from its definition: floor(log2 n) and the
    next two bits below the leading one (0 for an empty list)."""
    if n == 0:
        return 0
    l2 = n.bit_length() - 1
    return 1 + l2 if l2 < 2 else 4 * l2 + ((n >> (l2 - 2)) & 3)


def test_order_on_a_grid_of_66049_tiles(dev):
    scene = S.gmm_scene(11, 40_000, 32, (-3.5, 0.5), 1)
    cam = S.front_camera(4112, 4112)
    tiles = 257 * 257
    sc = pipeline.SceneTensors.from_scene(scene, dev)
    vb = pipeline.ViewBuffers(scene.n, cam, dev)
    vb.preprocess(sc)
    vb.bin()
    torch.cuda.synchronize()
    assert vb.n_keys > 0
    o = vb.tile_order.cpu().numpy()
    assert sorted(o.tolist()) == list(range(tiles))
    rg = vb.tile_ranges.cpu().numpy().astype(np.int64)
    lens = rg[o, 1] - rg[o, 0]
    b = np.array([_bucket(int(n)) for n in lens])
    assert np.all(np.diff(b) <= 0) and b[0] == _bucket(int(lens.max()))  # order inside a bucket is free

    bg = (0.2, 0.4, 0.6)
    ref = {}
    for name, order in (("rows", None), ("ordered", vb.tile_order)):
        image = torch.zeros_like(vb.image)
        fT = torch.zeros_like(vb.final_T)
        nc = torch.zeros_like(vb.n_contrib)
        gsr.gsr_forward(vb.W, vb.H, 16, 16, vb.tile_ranges, vb.point_list, vb.splat2d, bg, image, fT, nc,
                        tile_order=order)
        ref[name] = (image, fT, nc)
    for a, c in zip(ref["rows"], ref["ordered"]):
        assert torch.equal(a, c)

    image, fT, nc = ref["ordered"]
    g = torch.from_numpy(S.upstream_grad(3, vb.W, vb.H)).to(dev)
    n = scene.n
    off = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    scr = torch.empty(gsr.gsr_entry_offsets_scratch_bytes(n), dtype=torch.uint8, device=dev)
    gsr.gsr_entry_offsets(n, vb.W, vb.H, 16, 16, vb.splat2d, vb.radius, scr, off)
    partial = torch.empty(9 * vb.n_keys + 9, device=dev)
    res = []
    for order in (None, vb.tile_order):
        grad = torch.zeros((n, 12), device=dev)
        gsr.gsr_backward_deterministic(vb.W, vb.H, 16, 16, vb.tile_ranges, vb.point_list, vb.splat2d, vb.radius,
                                       n, off, bg, fT, nc, g, partial, grad, tile_order=order)
        res.append(grad.cpu().numpy())
    np.testing.assert_array_equal(res[0], res[1])
    assert np.abs(res[0]).max() > 0


@pytest.mark.parametrize("size,n", [((4112, 4112), 30_000), ((300, 200), 3_000), ((64, 48), 0)])
def test_async_binning_leaves_the_tile_order(dev, size, n):
    """gsr_bin_sort_async with a tile_order output (the last block of its
    column scan forms the order): a permutation with non-increasing buckets,
    the same bucket sequence as gsr_tile_order; a view without Gaussians
    gets one too."""
    W, H = size
    cam = S.front_camera(W, H)
    vb = pipeline.ViewBuffers(n, cam, dev)
    if n:
        vb.preprocess(pipeline.SceneTensors.from_scene(S.gmm_scene(12, n, 32, (-3.5, 0.5), 1), dev))
    for attempt in range(2):  # an overflow grows the key buffers: bin again
        vb.tile_order.fill_(-1)
        vb.bin_async()
        torch.cuda.synchronize()
        if vb.check_bin():
            break
    else:
        raise AssertionError("binning did not fit the grown key buffers")
    tiles = vb.gx * vb.gy
    o = vb.tile_order.cpu().numpy()
    assert sorted(o.tolist()) == list(range(tiles))
    rg = vb.tile_ranges.cpu().numpy().astype(np.int64)
    b = np.array([_bucket(int(x)) for x in rg[o, 1] - rg[o, 0]])
    assert np.all(np.diff(b) <= 0)
    o2 = torch.empty_like(vb.tile_order)
    gsr.gsr_tile_order(W, H, 16, 16, vb.tile_ranges, o2)
    torch.cuda.synchronize()
    b2 = np.array([_bucket(int(x)) for x in rg[o2.cpu().numpy(), 1] - rg[o2.cpu().numpy(), 0]])
    np.testing.assert_array_equal(b, b2)
    if n:
        assert vb.n_keys > 0 and b[0] > 0
