"""Shared test plumbing: packing oracle outputs into the FP32 records the CUDA
path consumes, and the scaled tolerance check used by every parity test."""
import json
import os

import numpy as np

RTOL = 1e-5   # relative tolerance for FP32 images and gradients
ATOL = 1e-7   # absolute floor
# Largest share of elements that may pass only through an FP32-ambiguity
# allowance or the per-pixel widening of the scale (not the literal bound).
MAX_EXTRA = 0.005

# One entry per check_scaled call: what the parity tests report at the end of
# the session (tests/conftest.py prints it; GSR_PARITY_REPORT=path writes it).
REPORT = []


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


def check_scaled(name, got, ref, scale, allow=None, rtol=RTOL, atol=ATOL, mask=None, lit=None,
                 max_extra=MAX_EXTRA):
    """|got - ref| <= rtol*scale + atol + allow elementwise (where mask).

    ``lit`` is the literal scale before any widening (default: ``scale``).
    Elements that fail rtol*lit + atol but pass the full bound pass only
    through an FP32-ambiguity allowance or the widening; their share must not
    exceed ``max_extra``.  Also recorded: the share meeting the plain bound
    rtol*|ref| + atol.  Returns the worst ratio |err| / bound; raises
    AssertionError on failure."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    bound = rtol * np.asarray(scale, np.float64) + atol
    if allow is not None:
        bound = bound + np.asarray(allow, np.float64)
    err = np.abs(got - ref)
    sel = np.ones(err.shape, bool) if mask is None else np.broadcast_to(np.asarray(mask, bool), err.shape)
    err = np.where(sel, err, 0.0)
    ratio = err / bound
    worst = float(ratio.max()) if ratio.size else 0.0
    lit_bound = rtol * (np.asarray(scale if lit is None else lit, np.float64)) + atol
    n_sel = int(sel.sum())
    lit_fail = sel & (err > lit_bound)
    extra = float((lit_fail & (ratio <= 1.0)).sum()) / max(1, n_sel)
    plain = float((sel & (err <= rtol * np.abs(ref) + atol)).sum()) / max(1, n_sel)
    REPORT.append({"check": name, "elements": n_sel, "worst_ratio": worst, "extra_share": extra,
                   "plain_bound_share": plain, "literal_share": 1.0 - float(lit_fail.sum()) / max(1, n_sel)})
    if not worst <= 1.0:
        idx = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
        n_bad = int((ratio > 1.0).sum())
        raise AssertionError(f"{name}: {n_bad}/{ratio.size} elements out of tolerance; worst at {idx}: "
                             f"got {got[idx]!r} ref {ref[idx]!r} bound {bound[idx]!r}")
    if extra > max_extra:
        raise AssertionError(f"{name}: {extra:.4%} of the elements pass only through an allowance or the "
                             f"widening (at most {max_extra:.2%} allowed)")
    return worst


def write_report(path):
    with open(path, "w") as f:
        json.dump(REPORT, f, indent=0)


def report_lines():
    """Summary of the recorded checks, worst first."""
    if not REPORT:
        return []
    rows = sorted(REPORT, key=lambda r: -r["extra_share"])
    tot = sum(r["elements"] for r in REPORT)
    ext = sum(r["extra_share"] * r["elements"] for r in REPORT)
    pla = sum(r["plain_bound_share"] * r["elements"] for r in REPORT)
    out = [f"{len(REPORT)} scaled checks over {tot} elements: {ext / max(1, tot):.5%} pass only through an "
           f"allowance or the widening; {pla / max(1, tot):.4%} meet 1e-5*|oracle| + 1e-7"]
    for r in rows[:8]:
        out.append(f"  {r['check'][:70]:70s} n={r['elements']:8d} worst={r['worst_ratio']:.3f} "
                   f"extra={r['extra_share']:.4%} plain={r['plain_bound_share']:.4%}")
    return out
