"""Host logic of ViewBuffers' block masks, with the libgsr calls replaced by
stand-ins that record their arguments: the forward always receives the mask
buffer to fill, and a backward receives it only while it belongs to the
current projection and binning (a mask of other lists or splats would cull
wrong pairs)."""
import types

import pytest
import torch

from paper_2401_05345_gb300 import gsr, pipeline
from paper_2401_05345_gb300 import scenes as S


@pytest.fixture
def vb(monkeypatch):
    calls = []

    def rec(name):
        def f(*a, **k):
            calls.append((name, k.get("block_mask")))
        return f

    for name in ("gsr_preprocess", "gsr_tile_order", "gsr_bin_sort_async", "gsr_entry_offsets",
                 "gsr_forward", "gsr_forward_l1", "gsr_backward", "gsr_backward_deterministic"):
        monkeypatch.setattr(gsr, name, rec(name))
    monkeypatch.setattr(gsr, "gsr_bin_scratch_bytes", lambda *a, **k: 256)
    monkeypatch.setattr(gsr, "gsr_entry_offsets_scratch_bytes", lambda n: 256)
    status = {"st": gsr.GSR_OK}
    monkeypatch.setattr(gsr, "gsr_bin_sort", lambda *a, **k: (status["st"], 5000))
    v = pipeline.ViewBuffers(100, S.front_camera(64, 48), device="cpu")
    v.calls = calls
    v.status = status
    return v


def last(vb, name):
    return [m for n, m in vb.calls if n == name][-1]


def test_forward_always_writes_the_masks(vb):
    bg = (0.0, 0.0, 0.0)
    vb.forward(bg)
    assert last(vb, "gsr_forward") is vb.block_mask
    vb.forward_l1(bg, None, None)
    assert last(vb, "gsr_forward_l1") is vb.block_mask
    assert vb.block_mask.dtype == torch.uint8 and vb.block_mask.numel() >= vb.key_capacity


def test_backward_reads_masks_only_after_a_forward_of_the_current_lists(vb):
    bg, g = (0.0, 0.0, 0.0), None
    vb.backward(bg, g)
    assert last(vb, "gsr_backward") is None  # no forward yet
    vb.forward(bg)
    vb.backward(bg, g)
    assert last(vb, "gsr_backward") is vb.block_mask
    vb.backward_deterministic(bg, g)
    assert last(vb, "gsr_backward_deterministic") is vb.block_mask
    scene = types.SimpleNamespace(sh_degree=3, mean=None, scale=None, quat=None, opacity=None, feat=None)
    vb.preprocess(scene)  # new splats: the masks are stale
    vb.backward(bg, g)
    assert last(vb, "gsr_backward") is None
    vb.forward_l1(bg, None, None)
    vb.bin()  # new lists
    vb.backward(bg, g)
    assert last(vb, "gsr_backward") is None
    vb.forward(bg)
    vb.bin_async()
    vb.backward_deterministic(bg, g)
    assert last(vb, "gsr_backward_deterministic") is None


def test_regrown_key_buffers_start_without_valid_masks(vb):
    bg = (0.0, 0.0, 0.0)
    vb.forward(bg)
    cap = vb.key_capacity
    assert not vb.apply_bin_status(cap + 10_000, 1)  # overflow: buffers grown for the next attempt
    assert vb.key_capacity > cap and vb.block_mask.numel() >= vb.key_capacity
    vb.backward(bg, None)
    assert last(vb, "gsr_backward") is None
