"""Seeded synthetic scenes and cameras.

This module is the only code shared by the CPU oracle and the CUDA path.  It
draws random inputs (Gaussian parameters, cameras, target images, upstream
gradients) and builds pinhole cameras; it holds none of the rasterizer's own
arithmetic (no projection, covariance, colour or compositing).

The paper evaluates 3DGS on captured datasets (Table I) that are not available
here; the generators below stand in for them with point clouds of the same
kind: Gaussian means from a uniform box or from an anisotropic Gaussian
mixture, log-normal scales, uniformly random rotations, sigmoid-normal
opacities and SH colour coefficients.

Conventions (shared by both sides, documented in the C header):
  * ``mean`` float32 [N,3] world position.
  * ``scale`` float32 [N,3] activated (positive) per-axis standard deviations.
  * ``quat`` float32 [N,4] (w, x, y, z), NOT normalised (the rasterizer
    normalises and differentiates through the normalisation).
  * ``opacity`` float32 [N] in (0, 1).
  * ``sh`` float32 [N, (deg+1)^2, 3] SH coefficients, or ``colors`` float32
    [N,3] precomputed RGB when ``sh_degree == -1``.
  * cameras: ``view`` float32 [3,4] row-major world->camera [R | t], the camera
    looks down +z, pixel centres at integer coordinates.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    view: np.ndarray        # float32 [3,4] world -> camera, row-major
    fx: float
    fy: float
    cx: float
    cy: float
    tan_fovx: float
    tan_fovy: float
    campos: np.ndarray      # float32 [3]
    znear: float = 0.2

    def as_f32(self) -> "Camera":
        f = lambda x: float(np.float32(x))
        return Camera(self.width, self.height, self.view.astype(np.float32),
                      f(self.fx), f(self.fy), f(self.cx), f(self.cy),
                      f(self.tan_fovx), f(self.tan_fovy),
                      self.campos.astype(np.float32), f(self.znear))


@dataclasses.dataclass
class Scene:
    mean: np.ndarray
    scale: np.ndarray
    quat: np.ndarray
    opacity: np.ndarray
    sh_degree: int            # -1 => ``feat`` holds RGB colours
    feat: np.ndarray          # [N, K, 3] SH coefficients or [N, 3] colours

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.mean[idx].copy(), self.scale[idx].copy(), self.quat[idx].copy(),
                     self.opacity[idx].copy(), self.sh_degree, self.feat[idx].copy())


def look_at_camera(eye, target, width, height, fov_x_deg=60.0, up=(0.0, 1.0, 0.0),
                   znear=0.2) -> Camera:
    """Pinhole camera at ``eye`` looking at ``target``; horizontal field of view
    ``fov_x_deg``, vertical one from the aspect ratio (square pixels)."""
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    upv = np.asarray(up, np.float64)
    if abs(float(np.dot(fwd, upv))) > 0.999:
        upv = np.array([0.0, 0.0, 1.0])
    right = np.cross(upv, fwd)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)        # camera y points down the image
    R = np.stack([right, down, fwd])   # rows: camera axes in world coordinates
    t = -R @ eye
    view = np.concatenate([R, t[:, None]], axis=1)
    tan_fovx = math.tan(math.radians(fov_x_deg) / 2.0)
    tan_fovy = tan_fovx * height / width
    fx = width / (2.0 * tan_fovx)
    fy = height / (2.0 * tan_fovy)
    return Camera(width, height, view.astype(np.float32), fx, fy,
                  (width - 1) / 2.0, (height - 1) / 2.0, tan_fovx, tan_fovy,
                  eye.astype(np.float32), znear).as_f32()


def front_camera(width, height, distance=4.0, fov_x_deg=60.0) -> Camera:
    """Camera on the -z axis at ``distance`` looking at the origin (+z)."""
    return look_at_camera((0.0, 0.0, -distance), (0.0, 0.0, 0.0), width, height, fov_x_deg)


def sphere_cameras(rng, n, center, radius, resolutions, fov_x_deg=60.0):
    """``n`` cameras on a sphere of ``radius`` around ``center`` looking at it."""
    cams = []
    for i in range(n):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        w, h = resolutions[i % len(resolutions)]
        cams.append(look_at_camera(np.asarray(center) + radius * d, center, w, h, fov_x_deg))
    return cams


def _random_rotations(rng, k):
    """Uniform random rotation matrices via QR of Gaussian matrices."""
    out = np.empty((k, 3, 3))
    for i in range(k):
        q, r = np.linalg.qr(rng.normal(size=(3, 3)))
        q = q * np.sign(np.diag(r))
        if np.linalg.det(q) < 0:
            q[:, 0] = -q[:, 0]
        out[i] = q
    return out


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _common(rng, n, log_scale_mu, log_scale_sd):
    scale = np.exp(rng.normal(log_scale_mu, log_scale_sd, size=(n, 3)))
    quat = rng.normal(size=(n, 4))
    opacity = _sigmoid(rng.normal(size=n))
    return scale.astype(np.float32), quat.astype(np.float32), opacity.astype(np.float32)


def uniform_scene(seed, n=1000, log_scale=(-3.0, 0.5), sh_degree=-1) -> Scene:
    """Means uniform in [-1,1]^3, log-scales N(mu, sd), random rotations,
    opacity sigmoid(N(0,1)).  ``sh_degree=-1``: RGB colours U[0,1]; otherwise
    SH coefficients with DC ~ U[0,1] and higher bands N(0, 0.05)."""
    rng = np.random.default_rng(seed)
    mean = rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
    scale, quat, opacity = _common(rng, n, *log_scale)
    return Scene(mean, scale, quat, opacity, sh_degree, _features(rng, n, sh_degree))


def _features(rng, n, sh_degree):
    if sh_degree < 0:
        return rng.uniform(0.0, 1.0, size=(n, 3)).astype(np.float32)
    k = (sh_degree + 1) ** 2
    f = np.empty((n, k, 3), np.float32)
    f[:, 0, :] = rng.uniform(0.0, 1.0, size=(n, 3))
    if k > 1:
        f[:, 1:, :] = rng.normal(0.0, 0.05, size=(n, k - 1, 3))
    return f


def gmm_scene(seed, n, components=64, log_scale=(-4.5, 0.7), sh_degree=3,
              center_box=1.0, comp_std=(0.05, 0.5)) -> Scene:
    """Means drawn from a ``components``-component anisotropic Gaussian mixture
    (centres U[-1,1]^3, per-axis std U[0.05,0.5], random orientation)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-center_box, center_box, size=(components, 3))
    stds = rng.uniform(comp_std[0], comp_std[1], size=(components, 3))
    rots = _random_rotations(rng, components)
    weights = rng.dirichlet(np.full(components, 2.0))
    comp = rng.choice(components, size=n, p=weights)
    z = rng.normal(size=(n, 3)) * stds[comp]
    mean = centres[comp] + np.einsum("nij,nj->ni", rots[comp], z)
    scale, quat, opacity = _common(rng, n, *log_scale)
    return Scene(mean.astype(np.float32), scale, quat, opacity, sh_degree,
                 _features(rng, n, sh_degree))


def target_image(seed, width, height) -> np.ndarray:
    """Seeded U[0,1] target image, float32 [3,H,W]."""
    rng = np.random.default_rng(seed + 7919)
    return rng.uniform(0.0, 1.0, size=(3, height, width)).astype(np.float32)


def upstream_grad(seed, width, height) -> np.ndarray:
    """Seeded dL/d(image) of L1 type: entries in {-1, +1}, float32 [3,H,W]."""
    rng = np.random.default_rng(seed + 104729)
    return np.where(rng.uniform(size=(3, height, width)) < 0.5, -1.0, 1.0).astype(np.float32)


# --- the workload recipes -------------------------------------------------

def tiny_workload(seed=0):
    """1,000 Gaussians in [-1,1]^3 four units in front of a 60-degree pinhole,
    log-scales N(-3, 0.5), RGB ~ U[0,1], one 128x128 view."""
    scene = uniform_scene(seed, 1000, (-3.0, 0.5), sh_degree=-1)
    cam = front_camera(128, 128)
    return scene, cam


def single_view_workload(seed=0, n=500_000):
    """500k Gaussians from a 64-component mixture, log-scales N(-4.5, 0.7),
    SH degree 3, one 1297x840 view."""
    scene = gmm_scene(seed, n, 64, (-4.5, 0.7), 3)
    cam = front_camera(1297, 840)
    return scene, cam


def large_workload(seed=0, n=3_000_000):
    """3M Gaussians from a 256-component mixture, SH degree 3, 1920x1080."""
    scene = gmm_scene(seed, n, 256, (-4.5, 0.7), 3)
    cam = front_camera(1920, 1080)
    return scene, cam


BATCH_RESOLUTIONS = [(256, 256), (800, 800), (1297, 840), (1920, 1080)]


def batched_workload(seed=0, sizes=(50_000, 200_000, 600_000, 1_200_000), views=32):
    """Four scenes of uneven size and ``views`` cameras spread over them, on a
    radius-4 sphere around each scene centre, resolutions mixed."""
    rng = np.random.default_rng(seed + 31337)
    scenes = [gmm_scene(seed + 17 * i, n, 64, (-4.5, 0.7), 3) for i, n in enumerate(sizes)]
    jobs = []
    for v in range(views):
        s = v % len(scenes)
        w, h = BATCH_RESOLUTIONS[v % len(BATCH_RESOLUTIONS)]
        cam = sphere_cameras(rng, 1, (0.0, 0.0, 0.0), 4.0, [(w, h)])[0]
        jobs.append((s, cam))
    return scenes, jobs


def cubemap_workload(seed=0, width=1024, height=1024, R=128, bumps=48):
    """Inputs of the cube-map texture workload (learning an environment map
    from images of a reflective object, the NvDiffRec workload): an
    orthographic view of a mirror sphere filling 90 % of the shorter image
    side, its normals perturbed by seeded bumps (mesh detail), and per pixel
    the reflection of the view ray (0, 0, -1) about the normal, FP32 [H,W,3]
    (zero outside the sphere: no sample).  Also a U[0,1] cube map [6,R,R,4]
    (fourth channel 0) and an L1-type upstream gradient [H,W,3] in {-1,+1}."""
    rng = np.random.default_rng(seed + 4242)
    ys, xs = np.mgrid[0:height, 0:width].astype(np.float64)
    rad = 0.45 * min(width, height)
    px = (xs + 0.5 - width / 2.0) / rad
    py = (ys + 0.5 - height / 2.0) / rad
    r2 = px * px + py * py
    inside = r2 < 1.0
    nz = np.sqrt(np.clip(1.0 - r2, 0.0, 1.0))
    n = np.stack([px, -py, nz], -1)
    # bumps: gradient of a sum of Gaussians over the image plane, added to the normal's tangent part
    c = rng.uniform(-0.9, 0.9, size=(bumps, 2))
    s = rng.uniform(0.05, 0.2, size=bumps)
    a = rng.uniform(-0.15, 0.15, size=bumps)
    gx = np.zeros_like(px)
    gy = np.zeros_like(py)
    for k in range(bumps):
        dx, dy = px - c[k, 0], py - c[k, 1]
        e = a[k] * np.exp(-(dx * dx + dy * dy) / (2 * s[k] * s[k])) / (s[k] * s[k])
        gx -= e * dx
        gy -= e * dy
    n[..., 0] -= gx
    n[..., 1] += gy
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    v = np.array([0.0, 0.0, -1.0])
    vn = n @ v
    r = v[None, None, :] - 2.0 * vn[..., None] * n
    r /= np.linalg.norm(r, axis=-1, keepdims=True)
    dirs = np.where(inside[..., None], r, 0.0).astype(np.float32)
    tex = rng.uniform(0.0, 1.0, size=(6, R, R, 4)).astype(np.float32)
    tex[..., 3] = 0.0
    dL = np.where(rng.uniform(size=(height, width, 3)) < 0.5, -1.0, 1.0).astype(np.float32)
    return dirs, tex, dL
