"""torch.autograd.Function over the libgsr rasterizer.

``rasterize`` renders one view from activated Gaussian parameters (the
forward pass of the training pipeline, Sec. II-B, Fig. 2) and, on backward,
runs the backward blend with the configured accumulation tier and the
backward projection.  ``GaussianModel`` keeps the raw parameters (log-scale,
opacity logit) and applies the activations in PyTorch, as 3DGS does.

``store_T=False`` keeps no per-pixel transmittance state between forward and
backward: the backward kernel recomputes final T and the last contributor
with the forward's own front-to-back walk (bit-identical), trading a
forward-like pre-pass for 8 bytes per pixel.
"""
from __future__ import annotations

import dataclasses

import torch

from . import gsr
from .pipeline import SceneTensors, ViewBuffers


@dataclasses.dataclass
class RasterSettings:
    cam: object
    bg: tuple = (0.0, 0.0, 0.0)
    opts: object = None           # gsr.BackwardOpts; default WARP
    store_T: bool = True
    key_capacity: int | None = None
    deterministic: bool = False   # atomic-free backward: bit-identical gradients run to run
    # view buffers free for reuse, by (Gaussians, device); a forward takes
    # one (or allocates) and its backward gives it back, so a training loop
    # allocates once while views rendered before any backward get their own
    pool: dict = dataclasses.field(default_factory=dict, repr=False, compare=False)

    def take_buffers(self, n, device) -> ViewBuffers:
        free = self.pool.get((int(n), str(device)))
        if free:
            return free.pop()
        return ViewBuffers(n, self.cam, device, self.key_capacity, self.store_T)

    def give_back(self, vb: ViewBuffers):
        self.pool.setdefault((int(vb.n), str(vb.device)), []).append(vb)


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mean, scale, quat, opacity, feat, sh_degree, settings):
        sc = SceneTensors(mean.contiguous(), scale.contiguous(), quat.contiguous(), opacity.contiguous(),
                          feat.contiguous(), int(sh_degree))
        vb = settings.take_buffers(sc.n, mean.device)
        vb.preprocess(sc, zero_grad=True)
        vb.bin()
        vb.forward(settings.bg)
        ctx.vb = vb
        ctx.settings = settings
        ctx.sh_degree = int(sh_degree)
        ctx.save_for_backward(sc.mean, sc.scale, sc.quat, sc.opacity, sc.feat)
        return vb.image.clone()

    @staticmethod
    def backward(ctx, dL_dimage):
        mean, scale, quat, opacity, feat = ctx.saved_tensors
        vb, st = ctx.vb, ctx.settings
        opts = st.opts if st.opts is not None else gsr.default_backward_opts(st.store_T)
        if bool(opts.store_T) != bool(st.store_T):
            opts = gsr.backward_opts(int(opts.reduce_mode), int(opts.threshold), int(opts.lane_layout),
                                     st.store_T, int(opts.pixels_per_thread))
        if st.deterministic:
            vb.backward_deterministic(st.bg, dL_dimage.contiguous(), opts)
        else:
            vb.backward(st.bg, dL_dimage.contiguous(), opts)
        sc = SceneTensors(mean, scale, quat, opacity, feat, ctx.sh_degree)
        g = sc.zeros_like_params()
        vb.backward_project(sc, g)
        ctx.vb = None
        st.give_back(vb)
        return g.mean, g.scale, g.quat, g.opacity, g.feat, None, None


def rasterize(mean, scale, quat, opacity, feat, sh_degree, settings: RasterSettings) -> torch.Tensor:
    """Image [3,H,W] of one view; differentiable w.r.t. all five inputs."""
    return _Rasterize.apply(mean, scale, quat, opacity, feat, sh_degree, settings)


class GaussianModel(torch.nn.Module):
    """Raw trainable parameters of a Gaussian scene (log-scales, opacity
    logits, unnormalised quaternions, SH coefficients or colours)."""

    def __init__(self, scene, device="cuda"):
        super().__init__()
        f = lambda a: torch.nn.Parameter(torch.as_tensor(a, dtype=torch.float32, device=device).clone())
        self.sh_degree = int(scene.sh_degree)
        self.mean = f(scene.mean)
        self.log_scale = f(torch.log(torch.as_tensor(scene.scale, dtype=torch.float32)))
        self.quat = f(scene.quat)
        o = torch.as_tensor(scene.opacity, dtype=torch.float32)
        self.opacity_logit = f(torch.log(o) - torch.log1p(-o))
        self.feat = f(torch.as_tensor(scene.feat, dtype=torch.float32).reshape(len(o), -1))

    def forward(self, settings: RasterSettings) -> torch.Tensor:
        return rasterize(self.mean, torch.exp(self.log_scale), self.quat, torch.sigmoid(self.opacity_logit),
                         self.feat, self.sh_degree, settings)
