"""Shared test plumbing: packing oracle outputs into the FP32 records the CUDA
path consumes, and the scaled tolerance check used by every parity test."""
import numpy as np

RTOL = 1e-5   # relative tolerance for FP32 images and gradients
ATOL = 1e-7   # absolute floor


def pack_records(pp):
    """Oracle preprocess outputs -> FP32 splat2d [N,12] (u, v, A, B, C, o,
    r, g, b, depth, 0, 0) and int32 radius."""
    n = len(pp["radius"])
    rec = np.zeros((n, 12), np.float32)
    rec[:, 0:2] = pp["uv"]
    rec[:, 2:5] = pp["conic"]
    rec[:, 5] = pp["opacity"]
    rec[:, 6:9] = pp["rgb"]
    rec[:, 9] = pp["depth"]
    rec[pp["radius"] <= 0] = 0.0
    return rec, pp["radius"].astype(np.int32)


def records_f64(rec):
    """Columns of the FP32 records as float64 arrays for the oracle."""
    r = rec.astype(np.float64)
    return dict(uv=r[:, 0:2].copy(), conic=r[:, 2:5].copy(), opacity=r[:, 5].copy(),
                rgb=r[:, 6:9].copy(), depth=r[:, 9].copy())


def check_scaled(name, got, ref, scale, allow=None, rtol=RTOL, atol=ATOL, mask=None):
    """|got - ref| <= rtol*scale + atol + allow elementwise (where mask).
    Returns the worst ratio |err| / bound; raises AssertionError on failure."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    bound = rtol * np.asarray(scale, np.float64) + atol
    if allow is not None:
        bound = bound + np.asarray(allow, np.float64)
    err = np.abs(got - ref)
    if mask is not None:
        err = np.where(mask, err, 0.0)
    ratio = err / bound
    worst = float(ratio.max()) if ratio.size else 0.0
    if not worst <= 1.0:
        idx = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
        n_bad = int((ratio > 1.0).sum())
        raise AssertionError(f"{name}: {n_bad}/{ratio.size} elements out of tolerance; worst at {idx}: "
                             f"got {got[idx]!r} ref {ref[idx]!r} bound {bound[idx]!r}")
    return worst
