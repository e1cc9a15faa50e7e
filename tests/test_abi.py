"""The C-ABI library builds, loads and exports every entry point that
include/gsr.h declares; host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gsr_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_05345_gb300 import build, gsr
    if not os.path.exists(gsr.LIB_PATH):
        try:
            build.build()
        except RuntimeError as e:  # no toolkit on this host
            pytest.skip(str(e))
    return gsr.lib()


def test_header_declares_the_boundary():
    fns = declared_functions()
    for f in ("gsr_preprocess", "gsr_bin_scratch_bytes", "gsr_bin_sort", "gsr_forward", "gsr_backward",
              "gsr_backward_project", "gsr_l1_loss", "gsr_adam_step", "gsr_status_string"):
        assert f in fns


def test_every_declared_symbol_is_exported(lib):
    for f in declared_functions():
        assert hasattr(lib, f), f"libgsr.so does not export {f}"


def test_status_strings(lib):
    from paper_2401_05345_gb300 import gsr
    for code in (gsr.GSR_OK, gsr.GSR_EINVAL, gsr.GSR_ECAPACITY, gsr.GSR_ECUDA, gsr.GSR_ETIMEOUT,
                 gsr.GSR_ESCRATCH):
        s = lib.gsr_status_string(code).decode()
        assert s and s != "unknown status"
    assert lib.gsr_version() >= 100


def test_argument_errors_are_reported_before_any_launch(lib):
    from paper_2401_05345_gb300 import gsr
    bg = (ctypes.c_float * 3)(0, 0, 0)
    # zero-sized image, unsupported tile, bad reduce mode: all rejected on the host
    assert lib.gsr_forward(0, 16, 16, 16, None, None, None, bg, None, None, None, None, None, None) == gsr.GSR_EINVAL
    opts = gsr.backward_opts("warp")
    opts.reduce_mode = 7
    p = ctypes.c_void_p(16)

    def bwd(*head, opts_ref=None, final=(p, p)):
        """gsr_backward with the given leading arguments, NULL tile order,
        block mask and stream."""
        return lib.gsr_backward(*head, *final, p, p, opts_ref, None, None, None)

    assert bwd(32, 32, 16, 16, p, p, p, bg, opts_ref=ctypes.byref(opts)) == gsr.GSR_EINVAL
    opts = gsr.backward_opts("hybrid", threshold=40)
    assert bwd(32, 32, 16, 16, p, p, p, bg, opts_ref=ctypes.byref(opts)) == gsr.GSR_EINVAL
    opts = gsr.backward_opts("plain", pixels_per_thread=2)   # the plain baseline keeps one pixel per thread
    assert bwd(32, 32, 16, 16, p, p, p, bg, opts_ref=ctypes.byref(opts)) == gsr.GSR_EINVAL
    opts = gsr.backward_opts("warp", pixels_per_thread=3)
    assert bwd(32, 32, 16, 16, p, p, p, bg, opts_ref=ctypes.byref(opts)) == gsr.GSR_EINVAL
    opts = gsr.backward_opts("warp", store_T=True)
    assert bwd(32, 32, 16, 16, p, p, p, bg, opts_ref=ctypes.byref(opts), final=(None, None)) == gsr.GSR_EINVAL
    assert bwd(32, 32, 12, 16, p, p, p, bg) == gsr.GSR_EINVAL
    # records must be 16-byte aligned, ranges 8-byte aligned
    p8 = ctypes.c_void_p(24)
    assert bwd(32, 32, 16, 16, p, p, p8, bg) == gsr.GSR_EINVAL
    assert bwd(32, 32, 16, 16, ctypes.c_void_p(20), p, p, bg) == gsr.GSR_EINVAL
    assert lib.gsr_forward(32, 32, 16, 16, p, p, p8, bg, p, None, None, None, None, None) == gsr.GSR_EINVAL
    # tile order: empty image, unsupported tile, missing output
    assert lib.gsr_tile_order(0, 16, 16, 16, p, p, None) == gsr.GSR_EINVAL
    assert lib.gsr_tile_order(32, 32, 8, 16, p, p, None) == gsr.GSR_EINVAL
    assert lib.gsr_tile_order(32, 32, 16, 16, p, None, None) == gsr.GSR_EINVAL
    # forward + L1: the target and the loss gradient are required
    assert lib.gsr_forward_l1(32, 32, 16, 16, p, p, p, bg, None, p, None, None, p,
                              None, None, None, None) == gsr.GSR_EINVAL
    assert lib.gsr_forward_l1(32, 32, 16, 16, p, p, p, bg, p, p, None, None, None,
                              None, None, None, None) == gsr.GSR_EINVAL
    cam = gsr.Camera()
    assert lib.gsr_preprocess(10, 4, p, p, p, p, p, ctypes.byref(cam), 16, 16, p, p, None, None) == gsr.GSR_EINVAL
    out = ctypes.c_size_t(0)
    assert lib.gsr_bin_scratch_bytes(10, 64, 64, 16, 16, -1, ctypes.byref(out)) == gsr.GSR_EINVAL
    assert lib.gsr_adam_step(10, p, p, p, p, 1e-3, 0.9, 0.999, 1e-8, 0, None) == gsr.GSR_EINVAL
    n = ctypes.c_int64(0)
    assert lib.gsr_bench_red(9, 32, 1, 1, p, 1024, ctypes.byref(n), None) == gsr.GSR_EINVAL
    assert lib.gsr_bench_red(7, 32, 1, 1, p, 1024, ctypes.byref(n), None) == gsr.GSR_EINVAL
    assert lib.gsr_bench_red(4, 32, 1, 1, ctypes.c_void_p(20), 1024, ctypes.byref(n), None) == gsr.GSR_EINVAL
    for lanes in (0, 33):
        assert lib.gsr_bench_red(3, lanes, 1, 1, p, 1024, ctypes.byref(n), None) == gsr.GSR_EINVAL


def test_grad2d_alignment_is_checked(lib):
    """grad2d takes 16-byte vector reds: a record buffer that starts off a
    16-byte boundary is refused on the host (not a misaligned access on the
    device)."""
    from paper_2401_05345_gb300 import gsr
    bg = (ctypes.c_float * 3)(0, 0, 0)
    p = ctypes.c_void_p(16)
    opts = gsr.backward_opts("hybrid", 24, 1, True, 2)
    for off in (4, 8, 12):
        g = ctypes.c_void_p(16 + off)
        assert lib.gsr_backward(32, 32, 16, 16, p, p, p, bg, p, p, p, g, ctypes.byref(opts), None, None,
                                None) == gsr.GSR_EINVAL
        assert lib.gsr_backward_deterministic(32, 32, 16, 16, p, p, p, p, 10, p, bg, p, p, p, p, 100, g,
                                              ctypes.byref(opts), None, None, None) == gsr.GSR_EINVAL


def test_red_counts_argument_errors(lib):
    from paper_2401_05345_gb300 import gsr
    p = ctypes.c_void_p(16)

    def rc(opts, counts=p, final=(p, p)):
        return lib.gsr_backward_red_counts(32, 32, 16, 16, p, p, p, *final, ctypes.byref(opts), None, None, counts,
                                           None)
    for bad in (gsr.backward_opts("block"), gsr.backward_opts("cluster"), gsr.backward_opts("warp", store_T=False),
                gsr.backward_opts("plain", pixels_per_thread=2)):
        assert rc(bad) == gsr.GSR_EINVAL
    good = gsr.backward_opts("hybrid", 24, 1, True, 2)
    assert rc(good, counts=None) == gsr.GSR_EINVAL
    assert rc(good, counts=ctypes.c_void_p(20)) == gsr.GSR_EINVAL
    assert rc(good, final=(None, p)) == gsr.GSR_EINVAL


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2401_05345_gb300 import gsr
    monkeypatch.setattr(gsr, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gsr, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        gsr.lib()
