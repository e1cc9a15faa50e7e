"""Divergent-destination accumulation (Sec. V-A1, SW-S): every method of
gsr_scatter_add9 against the FP64 oracle's plain scatter-add, for warps whose
lanes hit 1, 2, 3, 8 or 32 distinct destinations, ragged sizes and every
threshold regime."""
import numpy as np
import pytest
import torch

from _helpers import check_scaled
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


def divergent_indices(rng, n, distinct_per_warp, rows):
    """Each warp of 32 consecutive items draws from its own set of
    ``distinct_per_warp`` destinations (lanes shuffled)."""
    idx = np.empty(n, np.uint32)
    for w0 in range(0, n, 32):
        k = min(32, n - w0)
        pool = rng.choice(rows, distinct_per_warp, replace=False)
        idx[w0:w0 + k] = rng.choice(pool, k)
    return idx


@pytest.mark.parametrize("stride", [12, 9])  # 12: rows 16-byte aligned (vector reds); 9: scalar reds
@pytest.mark.parametrize("distinct", [1, 2, 3, 8, 32])
@pytest.mark.parametrize("method,threshold", [("plain", 0), ("serial", 0), ("serial", 4), ("serial", 33),
                                              ("sorted", 0)])
def test_scatter_add9_matches_oracle(dev, orc, distinct, method, threshold, stride):
    rng = np.random.default_rng(distinct * 7 + threshold)
    n, rows = 10_000 + 13, 500
    idx = divergent_indices(rng, n, distinct, rows)
    vals = rng.normal(size=(n, 9)).astype(np.float32)
    out = torch.zeros((rows, stride), device=dev)
    gsr.gsr_scatter_add9(n, torch.from_numpy(idx.view(np.int32)).to(dev), torch.from_numpy(vals).to(dev), out,
                         stride, method, threshold)
    got = out.cpu().numpy()
    ref = orc.scatter_add9(idx, vals.astype(np.float64), rows)
    scale = orc.scatter_add9(idx, np.abs(vals.astype(np.float64)), rows)
    check_scaled(f"{method}-{threshold}-{distinct}", got[:, :9], ref, scale)
    assert np.all(got[:, 9:] == 0)
