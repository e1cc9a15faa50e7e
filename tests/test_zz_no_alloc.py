"""The allocation-free binning entry point against the regular one.

gsr_bin_sort_static is for callers that cannot allocate device memory: code
whose process has given the GPU's memory to another allocator or a fixed
budget, and loops that cannot afford cudaMalloc's latency and implicit
synchronisation.  It keeps its scratch in a static device array inside libgsr
instead of a caller-provided buffer.  Through the C ABI it must give exactly
what gsr_bin_sort gives -- bit-identical keys, point list and tile ranges, as
every binning test requires -- on two calls in a row (on different scenes, so
anything the first call left in the shared array would show in the second),
and it must refuse sizes beyond its fixed limits with GSR_ELIMIT.
"""
import numpy as np
import pytest
import torch

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


def _splats(dev, scene, cam):
    n = scene.n
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev)
    splat = torch.zeros((n, 12), device=dev)
    radius = torch.zeros(n, dtype=torch.int32, device=dev)
    gsr.gsr_preprocess(n, scene.sh_degree, t(scene.mean), t(scene.scale), t(scene.quat), t(scene.opacity),
                       t(scene.feat.reshape(n, -1)), cam, 16, 16, splat, radius)
    return splat, radius


def _outputs(dev, cam, cap):
    tiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    pl = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    ranges = torch.full((tiles, 2), -7, dtype=torch.int32, device=dev)
    keys = torch.full((cap,), -7, dtype=torch.int64, device=dev)
    return pl, ranges, keys


def _regular(dev, scene, cam, splat, radius, cap):
    sb = gsr.gsr_bin_scratch_bytes(scene.n, cam.width, cam.height, 16, 16, cap)
    scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
    pl, ranges, keys = _outputs(dev, cam, cap)
    st, nk = gsr.gsr_bin_sort(scene.n, cam.width, cam.height, 16, 16, splat, radius, cap, scratch, pl,
                              ranges, keys)
    return st, nk, pl, ranges, keys


def _static(dev, scene, cam, splat, radius, cap):
    pl, ranges, keys = _outputs(dev, cam, cap)
    st, nk = gsr.gsr_bin_sort_static(scene.n, cam.width, cam.height, 16, 16, splat, radius, cap, pl,
                                     ranges, keys)
    return st, nk, pl, ranges, keys


def test_static_binning_matches_regular_on_two_calls_in_a_row(dev):
    cases = [(S.gmm_scene(1, 30000, 32, (-3.5, 0.5), 2), S.front_camera(640, 400)),
             S.tiny_workload(2)]
    for scene, cam in cases:
        splat, radius = _splats(dev, scene, cam)
        cap = 16 * scene.n + 1024
        st_r, nk_r, pl_r, rg_r, k_r = _regular(dev, scene, cam, splat, radius, cap)
        st_s, nk_s, pl_s, rg_s, k_s = _static(dev, scene, cam, splat, radius, cap)
        torch.cuda.synchronize()
        assert st_r == gsr.GSR_OK and st_s == gsr.GSR_OK
        assert nk_s == nk_r > 0
        assert torch.equal(k_s[:nk_s], k_r[:nk_r])
        assert torch.equal(pl_s[:nk_s], pl_r[:nk_r])
        assert torch.equal(rg_s, rg_r)


def test_static_binning_refuses_sizes_beyond_its_limits(dev):
    cam = S.front_camera(1920, 1080)
    # more Gaussians than the static scratch holds: refused before any work
    x = torch.zeros(16, device=dev)
    xi = torch.zeros(16, dtype=torch.int32, device=dev)
    st, _ = gsr.gsr_bin_sort_static(gsr.STATIC_BIN_MAX_GAUSSIANS + 1, cam.width, cam.height, 16, 16, x, xi,
                                    16, xi, xi, x)
    assert st == gsr.GSR_ELIMIT
    # 520 splats covering every one of the 8160 tiles: 4.24M keys > 2^22
    scene = S.uniform_scene(5, 520)
    scene.mean[:] = 0.0
    scene.scale[:] = 2.0
    splat, radius = _splats(dev, scene, cam)
    cap = 5_000_000
    pl, ranges, keys = _outputs(dev, cam, cap)
    st, nk = gsr.gsr_bin_sort_static(scene.n, cam.width, cam.height, 16, 16, splat, radius, cap, pl, ranges,
                                     keys)
    assert nk == 520 * 8160 > gsr.STATIC_BIN_MAX_KEYS
    assert st == gsr.GSR_ELIMIT
    # and the regular entry point still bins the same scene
    st_r, nk_r, *_ = _regular(dev, scene, cam, splat, radius, cap)
    assert st_r == gsr.GSR_OK and nk_r == nk
