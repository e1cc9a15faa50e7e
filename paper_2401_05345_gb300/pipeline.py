"""Per-view device buffers and the render / backward sequence over libgsr.

``SceneTensors`` holds one scene's parameters on the device; ``ViewBuffers``
holds everything one rendered view needs (2D splat records, bins, images) and
grows its key capacity when binning reports GSR_ECAPACITY.  All arithmetic
runs in libgsr kernels; this module only allocates and sequences calls.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import gsr

TILE = (16, 16)


@dataclasses.dataclass
class SceneTensors:
    mean: torch.Tensor
    scale: torch.Tensor
    quat: torch.Tensor
    opacity: torch.Tensor
    feat: torch.Tensor
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    @staticmethod
    def from_scene(scene, device="cuda") -> "SceneTensors":
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
        return SceneTensors(t(scene.mean), t(scene.scale), t(scene.quat), t(scene.opacity),
                            t(scene.feat), int(scene.sh_degree))

    def zeros_like_params(self):
        z = torch.zeros_like
        return SceneTensors(z(self.mean), z(self.scale), z(self.quat), z(self.opacity), z(self.feat),
                            self.sh_degree)

    def tensors(self):
        return [self.mean, self.scale, self.quat, self.opacity, self.feat]

    def nbytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in self.tensors())


class ViewBuffers:
    """Buffers of one (scene, camera) view."""

    def __init__(self, n, cam, device="cuda", key_capacity=None, store_T=True):
        self.n = int(n)
        self.cam = cam
        self.c_cam = gsr.camera(cam)
        self.W, self.H = int(cam.width), int(cam.height)
        self.tw, self.th = TILE
        self.gx = (self.W + self.tw - 1) // self.tw
        self.gy = (self.H + self.th - 1) // self.th
        self.device = device
        f32 = dict(dtype=torch.float32, device=device)
        self.splat2d = torch.zeros((max(self.n, 1), gsr.GSR_REC), **f32)
        self.radius = torch.zeros(max(self.n, 1), dtype=torch.int32, device=device)
        self.grad2d = torch.zeros((max(self.n, 1), gsr.GSR_REC), **f32)
        self.tile_ranges = torch.zeros((self.gx * self.gy, 2), dtype=torch.int32, device=device)
        # order in which the blend kernels take tiles (longest lists first);
        # any permutation is correct, so it starts as the identity
        self.tile_order = torch.arange(self.gx * self.gy, dtype=torch.int32, device=device)
        self.image = torch.zeros((3, self.H, self.W), **f32)
        self.final_T = torch.zeros((self.H, self.W), **f32) if store_T else None
        self.n_contrib = torch.zeros((self.H, self.W), dtype=torch.int32, device=device) if store_T else None
        self.n_keys = 0
        self._alloc_keys(key_capacity if key_capacity is not None else max(1024, 8 * self.n))

    def _alloc_keys(self, cap):
        self.key_capacity = int(cap)
        self.point_list = torch.zeros(max(self.key_capacity, 1), dtype=torch.int32, device=self.device)
        # per-entry cull masks: written by the forward, read by the backward
        # of the same lists (valid only between the two)
        self.block_mask = torch.zeros(max(self.key_capacity, 1), dtype=torch.uint8, device=self.device)
        self.mask_valid = False
        sb = gsr.gsr_bin_scratch_bytes(self.n, self.W, self.H, self.tw, self.th, self.key_capacity)
        self.scratch = torch.empty(sb, dtype=torch.uint8, device=self.device)

    def release_scratch(self):
        """Drops the binning scratch (not needed after binning; regrown on the
        next ``bin``)."""
        self.scratch = None

    def device_bytes(self) -> int:
        ts = [self.splat2d, self.radius, self.grad2d, self.tile_ranges, self.image, self.point_list, self.block_mask]
        ts += [self.scratch] if self.scratch is not None else []
        ts += [t for t in (self.final_T, self.n_contrib) if t is not None]
        return sum(t.numel() * t.element_size() for t in ts)

    # -- stages ------------------------------------------------------------
    def preprocess(self, sc: SceneTensors, zero_grad=True, stream=None):
        self.mask_valid = False
        gsr.gsr_preprocess(self.n, sc.sh_degree, sc.mean, sc.scale, sc.quat, sc.opacity, sc.feat,
                           self.c_cam, self.tw, self.th, self.splat2d, self.radius,
                           self.grad2d if zero_grad else None, stream)

    def bin(self, stream=None, keys_out=None):
        if self.scratch is None:
            sb = gsr.gsr_bin_scratch_bytes(self.n, self.W, self.H, self.tw, self.th, self.key_capacity)
            self.scratch = torch.empty(sb, dtype=torch.uint8, device=self.device)
        while True:
            st, nk = gsr.gsr_bin_sort(self.n, self.W, self.H, self.tw, self.th, self.splat2d, self.radius,
                                      self.key_capacity, self.scratch, self.point_list, self.tile_ranges,
                                      keys_out, stream)
            self.n_keys = nk
            if st == gsr.GSR_OK:
                self.order_tiles(stream)
                return nk
            if keys_out is not None:
                raise RuntimeError("keys_out smaller than the key count %d" % nk)
            self._alloc_keys(int(nk * 1.25) + 1024)

    def bin_async(self, stream=None):
        """Binning without a host sync into the current buffers; the key count
        and status land in ``self.bin_count`` (device int32 [2]).  Check them
        after the step with ``check_bin``."""
        if self.scratch is None:
            sb = gsr.gsr_bin_scratch_bytes(self.n, self.W, self.H, self.tw, self.th, self.key_capacity)
            self.scratch = torch.empty(sb, dtype=torch.uint8, device=self.device)
        if getattr(self, "bin_count", None) is None:
            self.bin_count = torch.zeros(2, dtype=torch.int32, device=self.device)
        # the binning also leaves the longest-first tile order of its lists
        self.mask_valid = False
        gsr.gsr_bin_sort_async(self.n, self.W, self.H, self.tw, self.th, self.splat2d, self.radius,
                               self.key_capacity, self.scratch, self.point_list, self.tile_ranges, self.bin_count,
                               None, stream, tile_order=self.tile_order)

    def order_tiles(self, stream=None):
        """Longest-first tile order of the current lists (gsr_tile_order);
        called after every binning, so it also marks the block masks stale."""
        self.mask_valid = False
        gsr.gsr_tile_order(self.W, self.H, self.tw, self.th, self.tile_ranges, self.tile_order, stream)

    def check_bin(self) -> bool:
        """After an asynchronous binning (and a sync): True if the lists were
        complete; otherwise the key buffers are grown for the next attempt."""
        cnt, status = (int(x) for x in self.bin_count.cpu())
        return self.apply_bin_status(cnt, status)

    def apply_bin_status(self, cnt, status) -> bool:
        """``check_bin`` on a (key count, status) pair the caller already
        copied to the host.  Grown buffers are allocated and zeroed on the
        current stream: make it the stream of their next use."""
        cnt, status = int(cnt), int(status)
        self.n_keys = cnt
        if status == 0:
            return True
        if status == 2:
            raise RuntimeError("inconsistent binning counts")
        self._alloc_keys(int(cnt * 1.25) + 1024)
        return False

    def forward(self, bg, stream=None):
        gsr.gsr_forward(self.W, self.H, self.tw, self.th, self.tile_ranges, self.point_list, self.splat2d,
                        bg, self.image, self.final_T, self.n_contrib, stream, tile_order=self.tile_order,
                        block_mask=self.block_mask)
        self.mask_valid = True

    def forward_l1(self, bg, target, dL_dimage, loss_sum=None, stream=None):
        """Forward with the L1 loss formed in its epilogue (gsr_forward_l1)."""
        gsr.gsr_forward_l1(self.W, self.H, self.tw, self.th, self.tile_ranges, self.point_list, self.splat2d,
                           bg, target, self.image, self.final_T, self.n_contrib, dL_dimage, loss_sum, stream,
                           tile_order=self.tile_order, block_mask=self.block_mask)
        self.mask_valid = True

    def _mask(self):
        """The forward's block masks when they belong to the current lists."""
        return self.block_mask if self.mask_valid else None

    def backward(self, bg, dL_dimage, opts=None, stream=None):
        gsr.gsr_backward(self.W, self.H, self.tw, self.th, self.tile_ranges, self.point_list, self.splat2d,
                         bg, self.final_T, self.n_contrib, dL_dimage, self.grad2d, opts, stream,
                         tile_order=self.tile_order, block_mask=self._mask())

    def red_counts(self, opts, stream=None) -> dict:
        """The global red traffic one ``backward`` with ``opts`` issues
        (gsr_backward_red_counts; PLAIN, WARP or HYBRID, stored T)."""
        c = torch.zeros(39, dtype=torch.int64, device=self.device)
        gsr.gsr_backward_red_counts(self.W, self.H, self.tw, self.th, self.tile_ranges, self.point_list, self.splat2d,
                                    self.final_T, self.n_contrib, opts, c, stream, tile_order=self.tile_order,
                                    block_mask=self._mask())
        v = [int(x) for x in c.cpu()]
        out = dict(zip(gsr.RED_COUNT_NAMES, v))
        out["active_lane_hist"] = v[6:]
        return out

    def backward_deterministic(self, bg, dL_dimage, opts=None, stream=None):
        """Backward without float atomics (bit-identical run to run); keeps
        its per-entry partial buffer between calls, sized by the key capacity
        so that every binning that fits the key buffers fits it too (also
        when the key count is not known on the host: asynchronous binning,
        graph replays)."""
        nk = max(self.n_keys, self.key_capacity, 1)
        if getattr(self, "_det_partial", None) is None or self._det_partial.numel() < 9 * nk:
            self._det_partial = torch.empty(9 * nk, dtype=torch.float32, device=self.device)
            self._det_offsets = torch.empty(self.n + 1, dtype=torch.int32, device=self.device)
            self._det_scratch = torch.empty(gsr.gsr_entry_offsets_scratch_bytes(self.n), dtype=torch.uint8,
                                            device=self.device)
        gsr.gsr_entry_offsets(self.n, self.W, self.H, self.tw, self.th, self.splat2d, self.radius, self._det_scratch,
                              self._det_offsets, stream)
        gsr.gsr_backward_deterministic(self.W, self.H, self.tw, self.th, self.tile_ranges, self.point_list,
                                       self.splat2d, self.radius, self.n, self._det_offsets, bg, self.final_T,
                                       self.n_contrib, dL_dimage, self._det_partial, self.grad2d, opts, stream,
                                       tile_order=self.tile_order, block_mask=self._mask())

    def backward_project(self, sc: SceneTensors, grads: SceneTensors, stream=None, accumulate=True):
        """3D gradients of this view: added to ``grads``, or (accumulate=False)
        written over them."""
        gsr.gsr_backward_project(self.n, sc.sh_degree, sc.mean, sc.scale, sc.quat, sc.opacity, sc.feat,
                                 self.c_cam, self.radius, self.grad2d, grads.mean, grads.scale, grads.quat,
                                 grads.opacity, grads.feat, stream, accumulate)


class Renderer:
    """One view's render + backward through libgsr: the unit of work of the
    training iteration (Sec. II-B, Fig. 2): projection, binning, forward blend
    with the L1 loss gradient formed in its epilogue, backward blend with
    gradient accumulation, backward
    projection."""

    def __init__(self, n, cam, device="cuda", opts=None, store_T=True, key_capacity=None, deterministic=False):
        self.vb = ViewBuffers(n, cam, device, key_capacity, store_T)
        self.opts = opts if opts is not None else gsr.default_backward_opts(store_T)
        self.deterministic = deterministic
        self.dimg = torch.zeros_like(self.vb.image)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)

    def project(self, sc: SceneTensors, stream=None):
        """The step's first stage: the 2D splat records of ``sc`` (with the 2D
        gradient records zeroed in the same pass)."""
        self.vb.preprocess(sc, zero_grad=True, stream=stream)

    def step(self, sc: SceneTensors, target: torch.Tensor, bg, grads: SceneTensors, stream=None,
             on_backward=None, accumulate=True, sync_bin=True):
        """Runs the whole path; ``grads`` accumulates the 3D gradients (or,
        with accumulate=False, receives them: no zeroing needed).  Returns the
        device scalar L1 loss.  ``on_backward(begin: bool)`` is called around
        the backward launch (event recording by benchmarks).  sync_bin=False
        bins without waiting for the key count: nothing in the step waits on
        the host, and ``self.vb.check_bin()`` must be called after the step
        (if it returns False the step has to be redone)."""
        vb = self.vb
        self.loss.zero_()
        self.project(sc, stream)
        if sync_bin:
            vb.bin(stream)
        else:
            vb.bin_async(stream)
        vb.forward_l1(bg, target, self.dimg, self.loss, stream)
        if on_backward:
            on_backward(True)
        if self.deterministic:
            vb.backward_deterministic(bg, self.dimg, self.opts, stream)
        else:
            vb.backward(bg, self.dimg, self.opts, stream)
        if on_backward:
            on_backward(False)
        vb.backward_project(sc, grads, stream, accumulate)
        return self.loss


class StepGraph:
    """One view's training step (``Renderer.step`` with asynchronous binning)
    captured once in a CUDA graph and replayed.  The step's 15 kernel
    launches, the loss reset and the gradient zeroing go to the GPU as one
    graph launch, so no launch gap separates the short binning kernels.

    The graph keeps the device addresses it was captured with: new inputs
    are copied into the same ``target`` tensor (and scene tensors) before a
    replay, and ``loss`` / ``grads`` are overwritten by each replay.  The key
    capacity is fixed at capture: after replays, ``ok()`` (one device read)
    reports whether the binning fitted; if not, the key buffers have been
    grown and the step must be captured again.

    ``backward_events``: optional (begin, end) ``torch.cuda.Event``s created
    with ``enable_timing=True, external=True``; they are recorded around the
    backward launch inside the graph on every replay."""

    def __init__(self, renderer: "Renderer", sc: SceneTensors, target: torch.Tensor, bg, grads: SceneTensors,
                 accumulate=False, backward_events=None):
        self.renderer = renderer
        dev = renderer.vb.device
        side = torch.cuda.Stream(device=dev)
        for attempt in range(2):  # a second pass after check_bin grew the key buffers
            side.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.stream(side):  # lazy allocations and first launches happen outside the capture
                renderer.step(sc, target, bg, grads, accumulate=accumulate, sync_bin=False)
            torch.cuda.current_stream(dev).wait_stream(side)
            torch.cuda.synchronize(dev)
            if renderer.vb.check_bin():
                break
        else:
            raise RuntimeError("binning did not fit the grown key buffers")
        hook = None
        if backward_events is not None:
            b0, b1 = backward_events
            hook = lambda begin: (b0 if begin else b1).record()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            renderer.step(sc, target, bg, grads, on_backward=hook, accumulate=accumulate, sync_bin=False)
        self.loss = renderer.loss

    def replay(self) -> torch.Tensor:
        """Runs the captured step on the current stream; returns the device
        scalar loss (valid once the stream reaches it)."""
        self.graph.replay()
        return self.loss

    def ok(self) -> bool:
        """After replays and a sync: True if every replay's binning fitted the
        key buffers."""
        return self.renderer.vb.check_bin()


class StepPipeline:
    """Training steps of one view fed from host memory with two steps in
    flight.  ``submit`` copies the step's target from pinned host memory on a
    copy stream, replays the captured step once the copy has landed, and
    copies the loss back to pinned memory; ``result`` waits for one step's
    loss.  So the upload of step k+1 overlaps the kernels of step k when the
    caller submits step k+1 before reading step k's loss.

    Each of the two target buffers has its own captured step (StepGraph);
    a buffer is refilled only after the replay that last read it has
    finished.  Handles name the buffer, so read a step's result before
    submitting the step after the next.  Binning overflow works as for StepGraph: ``ok()`` after the
    steps, capture again if it returns False."""

    def __init__(self, renderer: "Renderer", sc: SceneTensors, bg, grads: SceneTensors, accumulate=False):
        vb = renderer.vb
        dev = vb.device
        self.renderer = renderer
        self.targets = [torch.zeros((3, vb.H, vb.W), dtype=torch.float32, device=dev) for _ in range(2)]
        self.graphs = [StepGraph(renderer, sc, t, bg, grads, accumulate) for t in self.targets]
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.copied = [torch.cuda.Event() for _ in range(2)]
        self.done = [torch.cuda.Event() for _ in range(2)]
        self.loss_host = [torch.zeros(1, dtype=torch.float32).pin_memory() for _ in range(2)]
        self.k = 0

    def submit(self, target_host: torch.Tensor) -> int:
        """Queues one step on the current stream; returns its handle."""
        i = self.k % 2
        main = torch.cuda.current_stream(self.targets[i].device)
        if self.k >= 2:
            self.copy_stream.wait_event(self.done[i])  # the replay that read this buffer has finished
        with torch.cuda.stream(self.copy_stream):
            self.targets[i].copy_(target_host, non_blocking=True)
            self.copied[i].record(self.copy_stream)
        main.wait_event(self.copied[i])
        loss = self.graphs[i].replay()
        self.loss_host[i].copy_(loss, non_blocking=True)
        self.done[i].record(main)
        self.k += 1
        return i

    def result(self, handle: int) -> float:
        """The loss of the step ``handle`` (waits for that step only)."""
        self.done[handle].synchronize()
        return float(self.loss_host[handle][0])

    def ok(self) -> bool:
        return self.renderer.vb.check_bin()
