"""ctypes wrapper of the FP64 CPU oracle (``gsr_oracle.c``: the splat
rasterizer; ``cube_oracle.c``: cube-map texture sampling and its gradient).

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the
benchmark's CPU-baseline leg.  It shares no code with the CUDA library or its
Python binding; only the seeded input generators (``scenes``) serve both.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from ctypes import POINTER, c_double, c_float, c_int, c_longlong, c_uint32, c_uint64

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsr_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "cube_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, no FMA contraction, no fast-math, so
    x86 and Arm hosts evaluate the same IEEE operations."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp] + _SRCS + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrcCamera(ctypes.Structure):
    _fields_ = [("width", c_int), ("height", c_int), ("view", c_double * 12),
                ("fx", c_double), ("fy", c_double), ("cx", c_double), ("cy", c_double),
                ("tan_fovx", c_double), ("tan_fovy", c_double), ("campos", c_double * 3),
                ("znear", c_double)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    F = POINTER(c_float)
    lib.orc_cube_taps.argtypes = [c_longlong, F, c_int, POINTER(c_int), POINTER(c_longlong), POINTER(c_double)]
    lib.orc_cube_taps.restype = None
    lib.orc_cube_forward.argtypes = [c_longlong, F, c_int, F, POINTER(c_double), POINTER(c_double)]
    lib.orc_cube_forward.restype = None
    lib.orc_cube_backward.argtypes = [c_longlong, F, F, c_int, POINTER(c_double), POINTER(c_double)]
    lib.orc_cube_backward.restype = None
    D = POINTER(c_double)
    I = POINTER(c_int)
    U32 = POINTER(c_uint32)
    lib.orc_preprocess.argtypes = [c_int, c_int, D, D, D, D, D, POINTER(OrcCamera), c_int, c_int,
                                   D, D, D, D, I, I, I]
    lib.orc_preprocess.restype = c_int
    lib.orc_bin_count.argtypes = [c_int, D, I, c_int, c_int, c_int, c_int]
    lib.orc_bin_count.restype = c_longlong
    lib.orc_bin.argtypes = [c_int, D, D, I, c_int, c_int, c_int, c_int, POINTER(c_uint64), U32, U32]
    lib.orc_bin.restype = c_int
    lib.orc_render.argtypes = [c_int, c_int, c_int, c_int, U32, U32, c_int, D, D, D, D, D,
                               POINTER(c_float), POINTER(ctypes.c_uint8), D, D, I, D, D, D, D, D, D,
                               I, I, D, D, I]
    lib.orc_render.restype = c_int
    lib.orc_backproject.argtypes = [c_int, c_int, D, D, D, D, D, POINTER(OrcCamera), c_int, c_int,
                                    D, D, D, D, D, D, D, D, D, D]
    lib.orc_backproject.restype = c_int
    lib.orc_sh_basis.argtypes = [c_int, D, D]
    lib.orc_sh_basis_grad.argtypes = [c_int, D, D]
    lib.orc_adam.argtypes = [c_longlong, D, D, D, D, c_double, c_double, c_double, c_double, c_int]
    _lib = lib
    return lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a, t=c_double):
    return a.ctypes.data_as(POINTER(t)) if a is not None else None


def camera(cam) -> OrcCamera:
    c = OrcCamera()
    c.width, c.height = int(cam.width), int(cam.height)
    for i, x in enumerate(np.asarray(cam.view, np.float64).reshape(-1)):
        c.view[i] = float(x)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.tan_fovx, c.tan_fovy = float(cam.tan_fovx), float(cam.tan_fovy)
    for i in range(3):
        c.campos[i] = float(cam.campos[i])
    c.znear = float(cam.znear)
    return c


def _feat(scene):
    return _d(scene.feat).reshape(scene.n, -1)


def preprocess(scene, cam, tile=(16, 16)):
    lib = _load()
    n = scene.n
    out = dict(uv=np.zeros((n, 2)), conic=np.zeros((n, 3)), rgb=np.zeros((n, 3)),
               depth=np.zeros(n), radius=np.zeros(n, np.int32),
               pp_ambig=np.zeros(n, np.int32), bp_ambig=np.zeros(n, np.int32))
    m, s, q, o, f = _d(scene.mean), _d(scene.scale), _d(scene.quat), _d(scene.opacity), _feat(scene)
    oc = camera(cam)
    out["visible"] = lib.orc_preprocess(n, scene.sh_degree, _p(m), _p(s), _p(q), _p(o), _p(f),
                                        ctypes.byref(oc), tile[0], tile[1], _p(out["uv"]),
                                        _p(out["conic"]), _p(out["rgb"]), _p(out["depth"]),
                                        _p(out["radius"], c_int), _p(out["pp_ambig"], c_int),
                                        _p(out["bp_ambig"], c_int))
    out["opacity"] = o.copy()
    return out


def bin_count(uv, radius, W, H, tile=(16, 16)):
    lib = _load()
    uv, radius = _d(uv), np.ascontiguousarray(radius, np.int32)
    return int(lib.orc_bin_count(len(radius), _p(uv), _p(radius, c_int), W, H, tile[0], tile[1]))


def bin_sort(uv, depth, radius, W, H, tile=(16, 16)):
    """Returns (keys uint64 [P], point_list uint32 [P], ranges uint32 [tiles,2])."""
    lib = _load()
    uv, depth, radius = _d(uv), _d(depth), np.ascontiguousarray(radius, np.int32)
    n = bin_count(uv, radius, W, H, tile)
    gx, gy = (W + tile[0] - 1) // tile[0], (H + tile[1] - 1) // tile[1]
    keys = np.zeros(max(n, 1), np.uint64)
    vals = np.zeros(max(n, 1), np.uint32)
    ranges = np.zeros((gx * gy, 2), np.uint32)
    rc = lib.orc_bin(len(radius), _p(uv), _p(depth), _p(radius, c_int), W, H, tile[0], tile[1],
                     _p(keys, c_uint64), _p(vals, c_uint32), _p(ranges, c_uint32))
    if rc != 0:
        raise MemoryError("oracle bin_sort")
    return keys[:n], vals[:n], ranges


def render(W, H, ranges, point_list, uv, conic, opacity, rgb, bg, dL_dimage=None, tile=(16, 16),
           extras=True, tile_mask=None):
    """Forward image and (if dL_dimage is given) exact FP64 grad2d [N,9].
    ``tile_mask`` (bool per tile) restricts the evaluation to those tiles."""
    lib = _load()
    n = len(opacity)
    uv, conic, opacity, rgb, bg = _d(uv), _d(conic), _d(opacity), _d(rgb), _d(bg)
    ranges = np.ascontiguousarray(ranges, np.uint32)
    pl = np.ascontiguousarray(point_list, np.uint32)
    if pl.size == 0:
        pl = np.zeros(1, np.uint32)
    hw = W * H
    out = dict(image=np.zeros((3, H, W)), final_T=np.zeros((H, W)),
               n_contrib=np.zeros((H, W), np.int32), n_active=np.zeros((H, W), np.int32))
    g = None
    if dL_dimage is not None:
        g = np.ascontiguousarray(dL_dimage, np.float32)
        out["grad2d"] = np.zeros((n, 9))
        if extras:
            out["gscale"] = np.zeros((n, 9))
            out["glit"] = np.zeros((n, 9))
            out["gallow"] = np.zeros((n, 9))
    if extras:
        out["iallow"] = np.zeros((3, H, W))
        out["tallow"] = np.zeros((H, W))
        out["nc_alt"] = np.zeros((H, W), np.int32)
        out["pix_ambig"] = np.zeros((H, W), np.int32)
        out["pix_widen"] = np.ones((H, W))
        out["terr"] = np.zeros((H, W))
    tm = None
    if tile_mask is not None:
        tm = np.ascontiguousarray(tile_mask, np.uint8)
    gp = lambda k, t=c_double: _p(out[k], t) if k in out else None
    rc = lib.orc_render(W, H, tile[0], tile[1], _p(ranges, c_uint32), _p(pl, c_uint32), n,
                        _p(uv), _p(conic), _p(opacity), _p(rgb), _p(bg),
                        _p(g, c_float) if g is not None else None,
                        _p(tm, ctypes.c_uint8) if tm is not None else None,
                        gp("image"), gp("final_T"), gp("n_contrib", c_int), gp("grad2d"),
                        gp("gscale"), gp("glit"), gp("gallow"), gp("iallow"), gp("tallow"),
                        gp("nc_alt", c_int), gp("pix_ambig", c_int), gp("pix_widen"), gp("terr"),
                        gp("n_active", c_int))
    if rc != 0:
        raise MemoryError("oracle render")
    return out


def backproject(scene, cam, grad2d, tile=(16, 16), mags=True):
    lib = _load()
    n = scene.n
    k = 1 if scene.sh_degree < 0 else (scene.sh_degree + 1) ** 2
    m, s, q, o, f = _d(scene.mean), _d(scene.scale), _d(scene.quat), _d(scene.opacity), _feat(scene)
    g = _d(grad2d)
    out = dict(dmean=np.zeros((n, 3)), dscale=np.zeros((n, 3)), dquat=np.zeros((n, 4)),
               dopacity=np.zeros(n), dfeat=np.zeros((n, k, 3)) if scene.sh_degree >= 0 else np.zeros((n, 3)))
    if mags:
        out.update(dmean_mag=np.zeros((n, 3)), dscale_mag=np.zeros((n, 3)),
                   dquat_mag=np.zeros((n, 4)), dfeat_mag=np.zeros_like(out["dfeat"]))
    gp = lambda key: _p(out[key]) if key in out else None
    oc = camera(cam)
    lib.orc_backproject(n, scene.sh_degree, _p(m), _p(s), _p(q), _p(o), _p(f), ctypes.byref(oc),
                        tile[0], tile[1], _p(g), gp("dmean"), gp("dscale"), gp("dquat"),
                        gp("dopacity"), gp("dfeat"), gp("dmean_mag"), gp("dscale_mag"),
                        gp("dquat_mag"), gp("dfeat_mag"))
    return out


def sh_basis(deg, direction):
    lib = _load()
    d = _d(direction)
    out = np.zeros((deg + 1) ** 2)
    lib.orc_sh_basis(deg, _p(d), _p(out))
    return out


def sh_basis_grad(deg, direction):
    lib = _load()
    d = _d(direction)
    out = np.zeros(((deg + 1) ** 2, 3))
    lib.orc_sh_basis_grad(deg, _p(d), _p(out))
    return out


def adam(param, grad, m, v, lr, beta1, beta2, eps, step):
    """In-place FP64 Adam step on float64 arrays."""
    lib = _load()
    for a in (param, grad, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib.orc_adam(param.size, _p(param), _p(grad), _p(m), _p(v), lr, beta1, beta2, eps, step)


# --- conveniences used by tests and the CPU baseline -------------------

def render_scene(scene, cam, bg=(0.0, 0.0, 0.0), dL_dimage=None, tile=(16, 16), extras=False,
                 round_f32=False):
    """Whole oracle pipeline: preprocess -> bin -> render.  ``round_f32``
    rounds the 2D splat parameters to FP32 first (the storage format of the
    CUDA path); otherwise everything stays FP64 (finite-difference tests)."""
    pp = preprocess(scene, cam, tile)
    uv, conic, rgb, depth = pp["uv"], pp["conic"], pp["rgb"], pp["depth"]
    op = pp["opacity"]
    if round_f32:
        f = lambda a: a.astype(np.float32).astype(np.float64)
        uv, conic, rgb, depth, op = f(uv), f(conic), f(rgb), f(depth), f(op)
    keys, pl, ranges = bin_sort(uv, depth, pp["radius"], cam.width, cam.height, tile)
    out = render(cam.width, cam.height, ranges, pl, uv, conic, op, rgb, np.asarray(bg, np.float64),
                 dL_dimage, tile, extras)
    out.update(pp=pp, keys=keys, point_list=pl, ranges=ranges)
    return out


def scatter_add9(idx, vals, rows):
    """FP64 scatter-add of 9-value records: out[idx[i]] += vals[i] (the plain
    definition of the gradient accumulation with arbitrary destinations)."""
    out = np.zeros((rows, 9))
    np.add.at(out, np.asarray(idx, np.int64), np.asarray(vals, np.float64))
    return out


# ----------------------------------------------------------------------------
# cube-map texture sampling (cube_oracle.c)
# ----------------------------------------------------------------------------
def _f32(a):
    return np.ascontiguousarray(a, np.float32)


def cube_taps(dirs, R):
    """Per direction [n,3] (FP32): face (-1 = no sample), linear tap texels
    [n,4] (face*R*R + row*R + column) and tap weights [n,4] (FP64)."""
    lib = _load()
    d = _f32(dirs).reshape(-1, 3)
    n = len(d)
    face = np.zeros(max(n, 1), np.int32)
    texel = np.zeros((max(n, 1), 4), np.int64)
    w = np.zeros((max(n, 1), 4), np.float64)
    lib.orc_cube_taps(n, _p(d, c_float), R, _p(face, c_int), _p(texel, c_longlong), _p(w))
    return face[:n], texel[:n], w[:n]


def cube_forward(dirs, R, tex):
    """Bilinear cube-map samples [n,3] (FP64) and their scales (sum of the
    absolute terms).  tex: [6,R,R,4] FP32."""
    lib = _load()
    d = _f32(dirs).reshape(-1, 3)
    t = _f32(tex)
    assert t.shape == (6, R, R, 4)
    n = len(d)
    out = np.zeros((max(n, 1), 3))
    sc = np.zeros((max(n, 1), 3))
    lib.orc_cube_forward(n, _p(d, c_float), R, _p(t, c_float), _p(out), _p(sc))
    return out[:n], sc[:n]


def cube_backward(dirs, dL, R):
    """Texture gradient [6,R,R,3] (FP64) of sum(dL * sample) and its scale."""
    lib = _load()
    d = _f32(dirs).reshape(-1, 3)
    g = _f32(dL).reshape(-1, 3)
    grad = np.zeros((6, R, R, 3))
    sc = np.zeros((6, R, R, 3))
    lib.orc_cube_backward(len(d), _p(d, c_float), _p(g, c_float), R, _p(grad), _p(sc))
    return grad, sc
