"""Cube-map texture workload (the NvDiffRec environment-map learning of
Sec. VI) against the FP64 oracle: the bilinear sample of every pixel and the
texture gradient of every texel, for every accumulation tier.  Texel
choices are FP32 decisions taken with the same operations on both sides, so
the tap texels agree exactly; values agree within 1e-5 x (sum of the
absolute terms) + 1e-7."""
import numpy as np
import pytest
import torch

from _helpers import check_scaled
from paper_2401_05345_gb300 import gsr
from paper_2401_05345_gb300 import scenes as S

pytestmark = pytest.mark.gpu

METHODS = [("plain", 0), ("plain_v4", 0), ("serial", 0), ("serial", 2), ("serial", 16), ("serial", 33),
           ("sorted", 0), ("block", 0)]
CASES = [(96, 80, 8), (96, 80, 32), (64, 48, 1), (77, 53, 16)]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_05345_gb300 import build
    build.build()
    gsr.lib()
    return torch.device("cuda")


def _case(W, H, R, seed=0):
    dirs, tex, dL = S.cubemap_workload(seed, W, H, R, bumps=6)
    return dirs, tex, dL


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}-R{c[2]}")
def test_cube_forward_matches_oracle(dev, orc, case):
    W, H, R = case
    dirs, tex, dL = _case(W, H, R)
    out = torch.zeros((H, W, 3), device=dev)
    gsr.gsr_cube_forward(W, H, torch.from_numpy(dirs).to(dev), R, torch.from_numpy(tex).to(dev), out)
    ref, sc = orc.cube_forward(dirs.reshape(-1, 3), R, tex)
    check_scaled("cube forward", out.cpu().numpy().reshape(-1, 3), ref, sc)


@pytest.mark.parametrize("method", METHODS, ids=lambda m: f"{m[0]}-thr{m[1]}")
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}-R{c[2]}")
def test_cube_backward_matches_oracle(dev, orc, case, method):
    W, H, R = case
    dirs, tex, dL = _case(W, H, R, 1)
    grad = torch.zeros((6, R, R, 4), device=dev)
    gsr.gsr_cube_backward(W, H, torch.from_numpy(dirs).to(dev), torch.from_numpy(dL).to(dev), R, grad, *method)
    g = grad.cpu().numpy()
    ref, sc = orc.cube_backward(dirs.reshape(-1, 3), dL.reshape(-1, 3), R)
    assert np.abs(ref).max() > 0
    check_scaled(f"cube grad {method}", g[..., :3], ref, sc)
    assert np.all(g[..., 3] == 0.0)


def test_cube_backward_accumulates(dev, orc):
    W, H, R = 64, 64, 8
    dirs, tex, dL = _case(W, H, R, 2)
    init = np.random.default_rng(3).normal(size=(6, R, R, 4)).astype(np.float32)
    grad = torch.from_numpy(init.copy()).to(dev)
    gsr.gsr_cube_backward(W, H, torch.from_numpy(dirs).to(dev), torch.from_numpy(dL).to(dev), R, grad, "sorted")
    ref, sc = orc.cube_backward(dirs.reshape(-1, 3), dL.reshape(-1, 3), R)
    check_scaled("accumulate", grad.cpu().numpy()[..., :3], ref + init[..., :3], sc + np.abs(init[..., :3]))


@pytest.mark.parametrize("method", ["plain", "plain_v4", "serial", "sorted", "block"])
def test_cube_backward_full_size(dev, orc, method):
    """The benchmark workload: 1024 x 1024 mirror sphere, R = 128 (27 taps per
    texel on average, up to about 1300): every texel of the gradient."""
    dirs, tex, dL = S.cubemap_workload(0)
    H, W = dirs.shape[:2]
    R = tex.shape[1]
    grad = torch.zeros((6, R, R, 4), device=dev)
    gsr.gsr_cube_backward(W, H, torch.from_numpy(dirs).to(dev), torch.from_numpy(dL).to(dev), R, grad, method, 2)
    ref, sc = orc.cube_backward(dirs.reshape(-1, 3), dL.reshape(-1, 3), R)
    check_scaled(f"full-size cube grad {method}", grad.cpu().numpy()[..., :3], ref, sc)


def test_cube_invalid_arguments(dev):
    d = torch.zeros((4, 4, 3), device=dev)
    g = torch.zeros(6 * 4 * 4 * 4 + 1, device=dev)
    with pytest.raises(gsr.GsrError):
        gsr.gsr_cube_backward(4, 4, d, d, 4, g[1:], "plain")  # grad not 16-byte aligned
    with pytest.raises(gsr.GsrError):
        gsr.gsr_cube_backward(4, 4, d, d, 4, g[:-1], 9)
    with pytest.raises(gsr.GsrError):
        gsr.gsr_cube_forward(4, 4, d, 0, g[:-1], d)
