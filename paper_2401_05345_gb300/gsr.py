"""Python binding of libgsr (include/gsr.h): the same entry points, argument
marshalling only.  Device buffers are torch tensors (their data_ptr() is
passed); the CUDA stream defaults to torch's current stream.  Every compute
step runs in the library's kernels; there is no fallback: if libgsr.so is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_float, c_int, c_int32, c_int64, c_size_t, c_void_p

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsr.so")

GSR_OK, GSR_EINVAL, GSR_ECAPACITY, GSR_ECUDA, GSR_ETIMEOUT, GSR_ESCRATCH, GSR_ELIMIT = 0, -1, -2, -3, -4, -5, -6
STATIC_BIN_MAX_GAUSSIANS, STATIC_BIN_MAX_KEYS = 1 << 20, 1 << 22
GSR_REC = 12
REDUCE_PLAIN, REDUCE_WARP, REDUCE_HYBRID, REDUCE_BLOCK, REDUCE_CLUSTER = 0, 1, 2, 3, 4
REDUCE_NAMES = {"plain": REDUCE_PLAIN, "warp": REDUCE_WARP, "hybrid": REDUCE_HYBRID, "block": REDUCE_BLOCK,
                "cluster": REDUCE_CLUSTER}


class GsrError(RuntimeError):
    def __init__(self, fn, status, lib):
        self.status = status
        msg = lib.gsr_status_string(status).decode()
        if status == GSR_ECUDA:
            msg += " (" + lib.gsr_last_cuda_error().decode() + ")"
        super().__init__(f"{fn}: {msg} [{status}]")


class Camera(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("view", c_float * 12),
                ("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float),
                ("tan_fovx", c_float), ("tan_fovy", c_float), ("campos", c_float * 3),
                ("znear", c_float)]


class BackwardOpts(ctypes.Structure):
    _fields_ = [("reduce_mode", c_int32), ("threshold", c_int32), ("lane_layout", c_int32),
                ("store_T", c_int32), ("pixels_per_thread", c_int32), ("reserved", c_int32 * 3)]


def backward_opts(reduce="warp", threshold=0, lane_layout=0, store_T=True, pixels_per_thread=1) -> BackwardOpts:
    o = BackwardOpts()
    o.reduce_mode = REDUCE_NAMES[reduce] if isinstance(reduce, str) else int(reduce)
    o.threshold = int(threshold)
    o.lane_layout = int(lane_layout)
    o.store_T = 1 if store_T else 0
    o.pixels_per_thread = int(pixels_per_thread)
    return o


def default_backward_opts(store_T=True) -> BackwardOpts:
    """The tier the autotuner picks on a GB300 for the 500k single-view
    workload: HYBRID with threshold 24, 8x8 pixel blocks per warp, two pixels
    per thread.  autotune.tune measures the candidates for a given view."""
    return backward_opts("hybrid", 24, 1, store_T, 2)


def camera(cam) -> Camera:
    """ctypes camera from an object with the fields of ``scenes.Camera``."""
    c = Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    for i, x in enumerate(list(map(float, cam.view.reshape(-1)))):
        c.view[i] = x
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.tan_fovx, c.tan_fovy = float(cam.tan_fovx), float(cam.tan_fovy)
    for i in range(3):
        c.campos[i] = float(cam.campos[i])
    c.znear = float(cam.znear)
    return c


_lib = None


def lib():
    """Loads libgsr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2401_05345_gb300.build` (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    L.gsr_status_string.restype = c_char_p
    L.gsr_status_string.argtypes = [c_int]
    L.gsr_last_cuda_error.restype = c_char_p
    L.gsr_version.restype = c_int
    L.gsr_preprocess.argtypes = [c_int32, c_int32, P, P, P, P, P, POINTER(Camera), c_int32, c_int32,
                                 P, P, P, P]
    L.gsr_bin_scratch_bytes.argtypes = [c_int32, c_int32, c_int32, c_int32, c_int32, c_int64,
                                        POINTER(c_size_t)]
    L.gsr_bin_sort.argtypes = [c_int32, c_int32, c_int32, c_int32, c_int32, P, P, c_int64, P, c_size_t,
                               P, P, P, POINTER(c_int64), P]
    L.gsr_bin_scratch_bytes_library.argtypes = L.gsr_bin_scratch_bytes.argtypes
    L.gsr_bin_sort_library.argtypes = L.gsr_bin_sort.argtypes
    L.gsr_bin_sort_async.argtypes = [c_int32, c_int32, c_int32, c_int32, c_int32, P, P, c_int64, P, c_size_t,
                                     P, P, P, P, P, P]
    L.gsr_bin_sort_static.argtypes = [c_int32, c_int32, c_int32, c_int32, c_int32, P, P, c_int64, P, P, P,
                                      POINTER(c_int64), P]
    L.gsr_tile_order.argtypes = [c_int32, c_int32, c_int32, c_int32, P, P, P]
    L.gsr_forward_l1.argtypes = [c_int32, c_int32, c_int32, c_int32, P, P, P, POINTER(c_float), P, P, P, P, P, P,
                                 P, P, P]
    L.gsr_forward.argtypes = [c_int32, c_int32, c_int32, c_int32, P, P, P, POINTER(c_float), P, P, P, P, P, P]
    L.gsr_backward.argtypes = [c_int32, c_int32, c_int32, c_int32, P, P, P, POINTER(c_float), P, P, P, P,
                               POINTER(BackwardOpts), P, P, P]
    L.gsr_backward_stats.argtypes = [c_int32, c_int32, c_int32, c_int32, P, P, P, P, c_int32, P, P]
    L.gsr_backward_red_counts.argtypes = [c_int32, c_int32, c_int32, c_int32, P, P, P, P, P,
                                          POINTER(BackwardOpts), P, P, P, P]
    L.gsr_backward_project.argtypes = [c_int32, c_int32, P, P, P, P, P, POINTER(Camera), P, P, P, P, P,
                                       P, P, P]
    L.gsr_backward_project_store.argtypes = L.gsr_backward_project.argtypes
    L.gsr_l1_loss.argtypes = [c_int64, P, P, P, P, P]
    L.gsr_activate.argtypes = [c_int64, P, P, P, P, P]
    L.gsr_activate_backward.argtypes = [c_int64, P, P, P, P, P, P, P]
    L.gsr_adam_step.argtypes = [c_int64, P, P, P, P, c_float, c_float, c_float, c_float, c_int32, P]
    L.gsr_entry_offsets_scratch_bytes.argtypes = [c_int32, POINTER(c_size_t)]
    L.gsr_entry_offsets.argtypes = [c_int32, c_int32, c_int32, c_int32, c_int32, P, P, P, c_size_t, P, P]
    L.gsr_backward_deterministic.argtypes = [c_int32, c_int32, c_int32, c_int32, P, P, P, P, c_int32, P,
                                             POINTER(c_float), P, P, P, P, c_int64, P, POINTER(BackwardOpts), P, P,
                                             P]
    L.gsr_scatter_add9.argtypes = [c_int64, P, P, P, c_int32, c_int32, c_int32, P]
    L.gsr_bench_red.argtypes = [c_int32, c_int32, c_int32, c_int32, P, c_int64, POINTER(c_int64), P]
    L.gsr_cube_forward.argtypes = [c_int32, c_int32, P, c_int32, P, P, P]
    L.gsr_cube_backward.argtypes = [c_int32, c_int32, P, P, c_int32, P, c_int32, c_int32, P]
    for name in ("gsr_preprocess", "gsr_bin_scratch_bytes", "gsr_bin_sort", "gsr_bin_sort_static",
                 "gsr_bin_scratch_bytes_library", "gsr_bin_sort_library",
                 "gsr_tile_order", "gsr_forward", "gsr_forward_l1", "gsr_backward",
                 "gsr_backward_stats", "gsr_backward_project", "gsr_l1_loss", "gsr_adam_step", "gsr_bench_red",
                 "gsr_activate", "gsr_activate_backward", "gsr_scatter_add9", "gsr_entry_offsets_scratch_bytes",
                 "gsr_entry_offsets", "gsr_backward_deterministic", "gsr_cube_forward", "gsr_cube_backward",
                 "gsr_backward_project_store", "gsr_bin_sort_async"):
        getattr(L, name).restype = c_int
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _check(fn, status):
    if status != GSR_OK:
        raise GsrError(fn, status, lib())


def _f3(x):
    return (c_float * 3)(*[float(v) for v in x])


def gsr_version() -> int:
    return lib().gsr_version()


def gsr_preprocess(n, sh_degree, mean, scale, quat, opacity, feat, cam, tile_w, tile_h, splat2d, radius,
                   grad2d_to_zero=None, stream=None):
    c = cam if isinstance(cam, Camera) else camera(cam)
    _check("gsr_preprocess", lib().gsr_preprocess(n, sh_degree, _ptr(mean), _ptr(scale), _ptr(quat),
                                                  _ptr(opacity), _ptr(feat), ctypes.byref(c), tile_w,
                                                  tile_h, _ptr(splat2d), _ptr(radius),
                                                  _ptr(grad2d_to_zero), _stream(stream)))


def gsr_bin_scratch_bytes(n, width, height, tile_w, tile_h, key_capacity, library=False) -> int:
    name = "gsr_bin_scratch_bytes_library" if library else "gsr_bin_scratch_bytes"
    out = c_size_t(0)
    _check(name, getattr(lib(), name)(n, width, height, tile_w, tile_h, key_capacity, ctypes.byref(out)))
    return int(out.value)


def gsr_bin_sort(n, width, height, tile_w, tile_h, splat2d, radius, key_capacity, scratch, point_list,
                 tile_ranges, keys_out=None, stream=None, library=False):
    """Returns (status, n_keys); status is GSR_OK or GSR_ECAPACITY.  With
    library=True the same binning runs through CUB's radix sort
    (gsr_bin_sort_library, the measured comparison)."""
    name = "gsr_bin_sort_library" if library else "gsr_bin_sort"
    nk = c_int64(0)
    st = getattr(lib(), name)(n, width, height, tile_w, tile_h, _ptr(splat2d), _ptr(radius), key_capacity,
                              _ptr(scratch), scratch.numel() * scratch.element_size(), _ptr(point_list),
                              _ptr(tile_ranges), _ptr(keys_out), ctypes.byref(nk), _stream(stream))
    if st not in (GSR_OK, GSR_ECAPACITY):
        _check(name, st)
    return st, int(nk.value)


def gsr_bin_sort_async(n, width, height, tile_w, tile_h, splat2d, radius, key_capacity, scratch, point_list,
                       tile_ranges, count_dev, keys_out=None, stream=None, tile_order=None):
    """Binning without a host sync; count_dev (int32 [2] on the device)
    receives (key count, status 0 ok / 1 over capacity / 2 inconsistent);
    tile_order (optional, int32 [tiles]) the longest-first tile order."""
    _check("gsr_bin_sort_async", lib().gsr_bin_sort_async(
        n, width, height, tile_w, tile_h, _ptr(splat2d), _ptr(radius), key_capacity, _ptr(scratch),
        scratch.numel() * scratch.element_size(), _ptr(point_list), _ptr(tile_ranges), _ptr(keys_out),
        _ptr(count_dev), _ptr(tile_order), _stream(stream)))


def gsr_bin_sort_static(n, width, height, tile_w, tile_h, splat2d, radius, key_capacity, point_list,
                        tile_ranges, keys_out, stream=None):
    """Allocation-free binning (scratch in a static device array of libgsr).
    Returns (status, n_keys); status is GSR_OK, GSR_ECAPACITY or GSR_ELIMIT."""
    nk = c_int64(0)
    st = lib().gsr_bin_sort_static(n, width, height, tile_w, tile_h, _ptr(splat2d), _ptr(radius), key_capacity,
                                   _ptr(point_list), _ptr(tile_ranges), _ptr(keys_out), ctypes.byref(nk),
                                   _stream(stream))
    if st not in (GSR_OK, GSR_ECAPACITY, GSR_ELIMIT):
        _check("gsr_bin_sort_static", st)
    return st, int(nk.value)


def gsr_tile_order(width, height, tile_w, tile_h, tile_ranges, order, stream=None):
    """order: int32 tensor [tiles] (out): tile ids, longest lists first."""
    _check("gsr_tile_order", lib().gsr_tile_order(width, height, tile_w, tile_h, _ptr(tile_ranges), _ptr(order),
                                                  _stream(stream)))


def gsr_forward(width, height, tile_w, tile_h, tile_ranges, point_list, splat2d, bg, image, final_T=None,
                n_contrib=None, stream=None, tile_order=None, block_mask=None):
    _check("gsr_forward", lib().gsr_forward(width, height, tile_w, tile_h, _ptr(tile_ranges),
                                            _ptr(point_list), _ptr(splat2d), _f3(bg), _ptr(image),
                                            _ptr(final_T), _ptr(n_contrib), _ptr(block_mask), _ptr(tile_order),
                                            _stream(stream)))


def gsr_forward_l1(width, height, tile_w, tile_h, tile_ranges, point_list, splat2d, bg, target, image, final_T,
                   n_contrib, dL_dimage, loss_sum=None, stream=None, tile_order=None, block_mask=None):
    _check("gsr_forward_l1", lib().gsr_forward_l1(width, height, tile_w, tile_h, _ptr(tile_ranges),
                                                  _ptr(point_list), _ptr(splat2d), _f3(bg), _ptr(target),
                                                  _ptr(image), _ptr(final_T), _ptr(n_contrib), _ptr(dL_dimage),
                                                  _ptr(loss_sum), _ptr(block_mask), _ptr(tile_order),
                                                  _stream(stream)))


def gsr_backward(width, height, tile_w, tile_h, tile_ranges, point_list, splat2d, bg, final_T, n_contrib,
                 dL_dimage, grad2d, opts=None, stream=None, tile_order=None, block_mask=None):
    o = opts if opts is not None else backward_opts()
    _check("gsr_backward", lib().gsr_backward(width, height, tile_w, tile_h, _ptr(tile_ranges),
                                              _ptr(point_list), _ptr(splat2d), _f3(bg), _ptr(final_T),
                                              _ptr(n_contrib), _ptr(dL_dimage), _ptr(grad2d),
                                              ctypes.byref(o), _ptr(block_mask), _ptr(tile_order),
                                              _stream(stream)))


def gsr_entry_offsets_scratch_bytes(n) -> int:
    out = c_size_t(0)
    _check("gsr_entry_offsets_scratch_bytes", lib().gsr_entry_offsets_scratch_bytes(n, ctypes.byref(out)))
    return int(out.value)


def gsr_entry_offsets(n, width, height, tile_w, tile_h, splat2d, radius, scratch, offsets, stream=None):
    _check("gsr_entry_offsets", lib().gsr_entry_offsets(n, width, height, tile_w, tile_h, _ptr(splat2d), _ptr(radius),
                                                        _ptr(scratch), scratch.numel() * scratch.element_size(),
                                                        _ptr(offsets), _stream(stream)))


def gsr_backward_deterministic(width, height, tile_w, tile_h, tile_ranges, point_list, splat2d, radius, n,
                               entry_offsets, bg, final_T, n_contrib, dL_dimage, partial, grad2d, opts=None,
                               stream=None, tile_order=None, block_mask=None):
    """partial: float tensor; its size / 9 is the entry capacity passed on."""
    o = opts if opts is not None else backward_opts("warp", 0, 1, True, 2)
    _check("gsr_backward_deterministic", lib().gsr_backward_deterministic(
        width, height, tile_w, tile_h, _ptr(tile_ranges), _ptr(point_list), _ptr(splat2d), _ptr(radius), n,
        _ptr(entry_offsets), _f3(bg), _ptr(final_T), _ptr(n_contrib), _ptr(dL_dimage), _ptr(partial),
        partial.numel() // 9, _ptr(grad2d), ctypes.byref(o), _ptr(block_mask), _ptr(tile_order), _stream(stream)))


def gsr_backward_stats(width, height, tile_w, tile_h, tile_ranges, point_list, splat2d, n_contrib, hist,
                       lane_layout=0, stream=None):
    """hist: int64 tensor [38] (uint64 counts, see include/gsr.h)."""
    _check("gsr_backward_stats", lib().gsr_backward_stats(width, height, tile_w, tile_h, _ptr(tile_ranges),
                                                          _ptr(point_list), _ptr(splat2d), _ptr(n_contrib),
                                                          lane_layout, _ptr(hist), _stream(stream)))


RED_COUNT_NAMES = ("red_instructions", "red_v4_instructions", "adds", "lane_reds", "warp_steps",
                   "warp_steps_active")


def gsr_backward_red_counts(width, height, tile_w, tile_h, tile_ranges, point_list, splat2d, final_T, n_contrib,
                            opts, counts, stream=None, tile_order=None, block_mask=None):
    """counts: int64 tensor [39]: the totals named by RED_COUNT_NAMES, then
    the steps with 0..32 active lanes."""
    _check("gsr_backward_red_counts",
           lib().gsr_backward_red_counts(width, height, tile_w, tile_h, _ptr(tile_ranges), _ptr(point_list),
                                         _ptr(splat2d), _ptr(final_T), _ptr(n_contrib), ctypes.byref(opts),
                                         _ptr(block_mask), _ptr(tile_order), _ptr(counts), _stream(stream)))


def gsr_backward_project(n, sh_degree, mean, scale, quat, opacity, feat, cam, radius, grad2d, dmean,
                         dscale, dquat, dopacity, dfeat, stream=None, accumulate=True):
    """accumulate=False calls gsr_backward_project_store (outputs written,
    zero for culled Gaussians)."""
    c = cam if isinstance(cam, Camera) else camera(cam)
    name = "gsr_backward_project" if accumulate else "gsr_backward_project_store"
    _check(name, getattr(lib(), name)(
        n, sh_degree, _ptr(mean), _ptr(scale), _ptr(quat), _ptr(opacity), _ptr(feat), ctypes.byref(c),
        _ptr(radius), _ptr(grad2d), _ptr(dmean), _ptr(dscale), _ptr(dquat), _ptr(dopacity), _ptr(dfeat),
        _stream(stream)))


def gsr_l1_loss(count, image, target, dL_dimage, loss_sum=None, stream=None):
    _check("gsr_l1_loss", lib().gsr_l1_loss(count, _ptr(image), _ptr(target), _ptr(dL_dimage),
                                            _ptr(loss_sum), _stream(stream)))


def gsr_activate(n, log_scale, opacity_logit, scale, opacity, stream=None):
    _check("gsr_activate", lib().gsr_activate(n, _ptr(log_scale), _ptr(opacity_logit), _ptr(scale), _ptr(opacity),
                                              _stream(stream)))


def gsr_activate_backward(n, scale, opacity, dscale, dopacity, dlog_scale, dopacity_logit, stream=None):
    _check("gsr_activate_backward", lib().gsr_activate_backward(
        n, _ptr(scale), _ptr(opacity), _ptr(dscale), _ptr(dopacity), _ptr(dlog_scale), _ptr(dopacity_logit),
        _stream(stream)))


def gsr_adam_step(n, param, grad, m, v, lr, beta1, beta2, eps, step, stream=None):
    _check("gsr_adam_step", lib().gsr_adam_step(n, _ptr(param), _ptr(grad), _ptr(m), _ptr(v), lr, beta1,
                                                beta2, eps, step, _stream(stream)))


SCATTER_METHODS = {"plain": 0, "serial": 1, "sorted": 2}


def gsr_scatter_add9(n, idx, vals, out, stride=GSR_REC, method="serial", threshold=2, stream=None):
    m = SCATTER_METHODS[method] if isinstance(method, str) else int(method)
    _check("gsr_scatter_add9", lib().gsr_scatter_add9(n, _ptr(idx), _ptr(vals), _ptr(out), stride, m, threshold,
                                                      _stream(stream)))


def gsr_bench_red(pattern, blocks, iters, buffer, stream=None, active_lanes=32) -> int:
    adds = c_int64(0)
    _check("gsr_bench_red", lib().gsr_bench_red(pattern, active_lanes, blocks, iters, _ptr(buffer), buffer.numel(),
                                                ctypes.byref(adds), _stream(stream)))
    return int(adds.value)


TEX_METHODS = {"plain": 0, "plain_v4": 1, "serial": 2, "sorted": 3, "block": 4}


def gsr_cube_forward(width, height, dirs, R, tex, out, stream=None):
    _check("gsr_cube_forward", lib().gsr_cube_forward(width, height, _ptr(dirs), R, _ptr(tex), _ptr(out),
                                                      _stream(stream)))


def gsr_cube_backward(width, height, dirs, dL_dout, R, grad_tex, method="sorted", threshold=0, stream=None):
    m = TEX_METHODS[method] if isinstance(method, str) else int(method)
    _check("gsr_cube_backward", lib().gsr_cube_backward(width, height, _ptr(dirs), _ptr(dL_dout), R, _ptr(grad_tex),
                                                        m, threshold, _stream(stream)))
