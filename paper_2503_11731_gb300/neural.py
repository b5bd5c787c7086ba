"""Neural-Gaussian scene on the device: anchors, the decode MLP and its Adam
state, over the C ABI (marshalling only; the decode, its backward and the
Adam update run in libgsr.so).

A frame of the learned representation is
    gsr_decode_anchors (BF16 tcgen05 or FP32) -> surfel table -> Renderer,
and a training step adds
    gsr_loss -> gsr_backward -> gsr_decode_backward -> gsr_adam.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import gsr
from .frame import DeviceSurfels, _ptr, _stream_handle


class DeviceAnchors:
    def __init__(self, a, device="cuda"):
        f = lambda x: torch.as_tensor(np.ascontiguousarray(x, np.float32), device=device)
        self.pos, self.feature, self.scale = f(a.pos), f(a.feature), f(a.scale)
        self.offsets, self.intensity = f(a.offsets), f(a.intensity)

    @property
    def n(self):
        return int(self.pos.shape[0])

    @property
    def k(self):
        return int(self.offsets.shape[1])

    def struct(self):
        return gsr.Anchors(self.n, self.k, int(self.feature.shape[1]), _ptr(self.pos), _ptr(self.feature),
                           _ptr(self.scale), _ptr(self.offsets), _ptr(self.intensity))


class NeuralModel:
    """FP32 master weights of the decode MLP (+ the anchor features it trains)."""

    PARAMS = ("w1", "b1", "w2", "b2")

    def __init__(self, w1, b1, w2, b2, device="cuda", head=gsr.HEAD_CAMERA):
        """`head`: gsr.HEAD_CAMERA (the camera scene: colour) or gsr.HEAD_LIDAR
        (the LiDAR scene: intensity and ray drop)."""
        f = lambda x: torch.as_tensor(np.ascontiguousarray(x, np.float32), device=device)
        self.w1, self.b1, self.w2, self.b2 = f(w1), f(b1), f(w2), f(b2)
        self.head = int(head)
        self.device = device
        self.step_count = 0
        self._adam = {}

    def struct(self):
        return gsr.Mlp(int(self.w1.shape[1]), _ptr(self.w1), _ptr(self.b1), _ptr(self.w2), _ptr(self.b2), self.head)

    def new_table(self, anchors: DeviceAnchors) -> DeviceSurfels:
        N = anchors.n * anchors.k
        z = lambda *s: torch.zeros(*s, device=self.device)
        if self.head == gsr.HEAD_LIDAR:
            return DeviceSurfels(z(N, 3), z(N, 2), z(N, 4), z(N), z(N, 1, 3), z(N), ray_drop=z(N),
                                 sees=gsr.SEES_LIDARS)
        return DeviceSurfels(z(N, 3), z(N, 2), z(N, 4), z(N), z(N, 1, 3), z(N))

    def decode(self, anchors: DeviceAnchors, origin, cull_camera=None, precision=gsr.DECODE_BF16_TENSOR,
               out: DeviceSurfels = None, status=None, stream=None) -> DeviceSurfels:
        out = self.new_table(anchors) if out is None else out
        table = gsr.SurfelTable(_ptr(out.pos), _ptr(out.log_scale), _ptr(out.quat), _ptr(out.opacity), _ptr(out.sh),
                                _ptr(out.intensity), _ptr(out.ray_drop))
        cam = None if cull_camera is None else gsr.sensor(cull_camera)
        gsr.decode_anchors(anchors.struct(), self.struct(), origin, cam, precision, table,
                           None if status is None else _ptr(status), _stream_handle(stream))
        return out

    def zero_grads(self, anchors: DeviceAnchors):
        self.grads = {k: torch.zeros_like(getattr(self, k)) for k in self.PARAMS}
        self.grads["feature"] = torch.zeros_like(anchors.feature)

    def backward(self, anchors: DeviceAnchors, origin, surfel_grads: dict, cull_camera=None, stream=None):
        """Accumulate d(loss)/d(w1, b1, w2, b2, features) from d(loss)/d(decoded table)."""
        g = self.grads
        ds = gsr.SurfelGrads(None, _ptr(surfel_grads["log_scale"]), _ptr(surfel_grads["quat"]),
                             _ptr(surfel_grads["opacity"]), _ptr(surfel_grads.get("sh")),
                             _ptr(surfel_grads.get("intensity")), _ptr(surfel_grads.get("ray_drop")))
        out = gsr.MlpGrads(_ptr(g["w1"]), _ptr(g["b1"]), _ptr(g["w2"]), _ptr(g["b2"]), _ptr(g["feature"]))
        cam = None if cull_camera is None else gsr.sensor(cull_camera)
        gsr.decode_backward(anchors.struct(), self.struct(), origin, cam, ds, out, _stream_handle(stream))

    def adam_step(self, anchors: DeviceAnchors, lr=1e-3, lr_feature=None, betas=(0.9, 0.999), eps=1e-8,
                  stream=None):
        self.step_count += 1
        h = _stream_handle(stream)
        targets = [(k, getattr(self, k), lr) for k in self.PARAMS]
        targets.append(("feature", anchors.feature, lr if lr_feature is None else lr_feature))
        for name, p, rate in targets:
            if name not in self._adam:
                self._adam[name] = (torch.zeros_like(p), torch.zeros_like(p))
            m, v = self._adam[name]
            gsr.adam(_ptr(p), _ptr(self.grads[name]), _ptr(m), _ptr(v), p.numel(), rate, betas[0], betas[1], eps,
                     self.step_count, h)


def capture(fn):
    """Capture `fn()` (a sequence of calls into libgsr.so on the current
    stream) into a CUDA graph on a side stream; replay with .replay()."""
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    return g


class NeuralFrame:
    """A frame of the learned scene: the decoded background (surfels
    [0, A k) of the plan, SH degree 0) plus an explicit posed-object table
    (surfels [A k, A k + n_obj), its own SH degree), rendered by one plan:

        gsr_decode_anchors -> gsr_preprocess_part x 2 -> gsr_bin_sort -> gsr_render_rig

    With `lidar` = (model, anchors) of a separate LiDAR scene (its model's
    head gsr.HEAD_LIDAR), the cameras see the first decoded table and the
    LiDARs the second (surfels [A k, A k + A_L k_L)), objects follow both.
    `origin` is the decode's view origin (a camera centre, or the rig centre
    for a rig)."""

    def __init__(self, model: NeuralModel, anchors: DeviceAnchors, renderer, objects: DeviceSurfels = None,
                 poses=None, origin=(0.0, 0.0, 0.0), precision=gsr.DECODE_BF16_TENSOR, lidar=None):
        self.model, self.anchors, self.r = model, anchors, renderer
        self.objects, self.poses = objects, poses
        self.origin = [float(v) for v in origin]
        self.precision = precision
        self.table = model.new_table(anchors)
        self.n_bg = anchors.n * anchors.k
        self.lidar, self.table_l, self.n_l = lidar, None, 0
        if lidar is not None:
            if lidar[0].head != gsr.HEAD_LIDAR:
                raise ValueError("the LiDAR scene's model needs the LiDAR head")
            self.table.sees = gsr.SEES_CAMERAS
            self.table_l = lidar[0].new_table(lidar[1])
            self.n_l = lidar[1].n * lidar[1].k
        n_obj = 0 if objects is None else objects.n
        self._side = None
        if renderer.plan.n_surfels != self.n_bg + self.n_l + n_obj:
            raise ValueError("plan surfel count must equal decoded + object surfels")

    def decode(self, stream=None):
        self.model.decode(self.anchors, self.origin, precision=self.precision, out=self.table, stream=stream)
        if self.lidar is not None:
            self.lidar[0].decode(self.lidar[1], self.origin, precision=self.precision, out=self.table_l,
                                 stream=stream)

    def preprocess(self, stream=None):
        """Preprocess of every part (gsr_preprocess_part per table)."""
        self.r.preprocess(self.table, self.poses, stream, first=0)
        if self.lidar is not None:
            self.r.preprocess(self.table_l, self.poses, stream, first=self.n_bg)
        if self.objects is not None:
            self.r.preprocess(self.objects, self.poses, stream, first=self.n_bg + self.n_l)

    def front(self, stream=None):
        """Preprocess of every part and the binning sort."""
        self.preprocess(stream)
        self.r.bin_sort(stream)

    def decode_objects(self, stream=None):
        """The decode, with the posed-object table's preprocess alongside it
        on a second stream (it reads nothing the decode writes, and the two
        fill disjoint slots); then front_rest().  The decode leaves most of
        each SM's threads free, so the two overlap."""
        s = stream if stream is not None else torch.cuda.current_stream()
        if self.objects is None:
            self.decode(s)
            return
        if self._side is None:
            self._side = torch.cuda.Stream()
        self._side.wait_stream(s)
        self.r.preprocess(self.objects, self.poses, self._side, first=self.n_bg + self.n_l)
        self.decode(s)
        s.wait_stream(self._side)

    def front_rest(self, stream=None):
        """The decoded tables' preprocess and the binning sort (after decode_objects)."""
        self.r.preprocess(self.table, self.poses, stream, first=0)
        if self.lidar is not None:
            self.r.preprocess(self.table_l, self.poses, stream, first=self.n_bg)
        self.r.bin_sort(stream)

    def render(self, stream=None):
        self.decode(stream)
        self.front(stream)
        self.r.composite_rig(stream)
        return self.r.out

    def graphs(self):
        """Replayable graphs of one frame: decode, preprocess + sort, and the
        persistent whole-rig compositing launch; and the same front end as
        decode with the objects' preprocess alongside ("decode_objects")
        followed by the rest ("front_rest")."""
        return {"decode": capture(self.decode), "front": capture(self.front),
                "decode_objects": capture(self.decode_objects), "front_rest": capture(self.front_rest),
                "render_rig": self.r.graph(self.table, self.poses, stages=4)}


class FramePipeline:
    """Frames of a NeuralFrame streamed between pinned host memory and the
    device.  A frame's inputs are uploaded on an upload stream while the
    previous frame composites, and its outputs are read back on a download
    stream while the next frame decodes and sorts; events order every reuse
    of a buffer (an upload waits until the previous frame's front end has
    read the inputs, a compositing launch until the previous frame's outputs
    are read back), so no buffer is doubled.

    inputs: [(device tensor, pinned host tensor)] uploaded before each frame
    (the anchors, MLP weights, object table, poses the frame's graphs read);
    outputs: [(device tensor, pinned host tensor)] read back after it.
    """

    def __init__(self, nf: NeuralFrame, inputs, outputs, stream=None):
        self.G = nf.graphs()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.up, self.down = torch.cuda.Stream(), torch.cuda.Stream()
        self.inputs, self.outputs = list(inputs), list(outputs)
        self.front_done, self.inputs_ready = torch.cuda.Event(), torch.cuda.Event()
        self.render_done, self.outputs_read = torch.cuda.Event(), torch.cuda.Event()
        self.started = False

    def start_after(self, stream):
        """Order the next uploads after the work enqueued on `stream` so far."""
        self.up.wait_stream(stream)

    def frame(self, host_inputs=None, host_outputs=None):
        """Enqueue one frame; host_inputs / host_outputs (optional) replace
        the pinned host side of `inputs` / `outputs` for this frame.  A host
        input may be overwritten once `inputs_ready` has completed, a host
        output read once `outputs_read` has."""
        s = self.stream
        hin = host_inputs if host_inputs is not None else [h for _, h in self.inputs]
        hout = host_outputs if host_outputs is not None else [h for _, h in self.outputs]
        if self.started:
            self.up.wait_event(self.front_done)  # the previous frame has read its inputs
        with torch.cuda.stream(self.up):
            for (d, _), h in zip(self.inputs, hin):
                d.copy_(h, non_blocking=True)
        self.inputs_ready.record(self.up)
        s.wait_event(self.inputs_ready)
        with torch.cuda.stream(s):
            self.G["decode_objects"].replay()
            self.G["front_rest"].replay()
        self.front_done.record(s)
        if self.started:
            s.wait_event(self.outputs_read)  # the previous frame's outputs are read back
        self.G["render_rig"].launch(_stream_handle(s))
        self.render_done.record(s)
        self.down.wait_event(self.render_done)
        with torch.cuda.stream(self.down):
            for (d, _), h in zip(self.outputs, hout):
                h.copy_(d, non_blocking=True)
        self.outputs_read.record(self.down)
        self.started = True

    def finish(self):
        """Make `stream` wait for the last frame's outputs."""
        self.stream.wait_event(self.outputs_read)


class Distiller:
    """Distillation of a learned scene from target camera frames (Sec. III-A:
    the anchor MLP is trained on renders of the scene it stands in for).

    One step, on the library's kernels: decode the anchors (BF16 tensor-core
    or FP32 decode) -> render one camera -> gsr_loss against that camera's
    target frame -> gsr_backward (reverse rasteriser + preprocess backward
    to the decoded table) -> gsr_decode_backward (to the MLP weights and the
    anchor features) -> gsr_adam.  One plan per distinct camera model and
    size; a camera's pose is set with Renderer.move, so plans, workspaces and
    outputs are reused across poses."""

    OUTPUTS = ("rgb", "depth", "normal", "alpha", "trans", "depth_acc", "n_contrib")

    def __init__(self, model: NeuralModel, anchors: DeviceAnchors, tile=(16, 8), max_dup=0, split=(0, 0),
                 loss_weights=(0.0, 0.0)):
        """`loss_weights` = (distortion, normal consistency) of gsr_loss next
        to its L1 colour term."""
        self.model, self.anchors = model, anchors
        self.tile, self.max_dup, self.split = tile, max_dup, split
        self.w_dist, self.w_normal = loss_weights
        self.table = model.new_table(anchors)
        self.grads = {k: torch.zeros_like(getattr(self.table, k))
                      for k in ("pos", "log_scale", "quat", "opacity", "sh")}
        self._plans = {}

    def renderer(self, cam):
        """The plan of `cam`'s model and size, moved to `cam`'s pose."""
        from .frame import Renderer
        key = (cam.kind, cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, cam.near)
        r = self._plans.get(key)
        if r is None:
            r = self._plans[key] = Renderer(self.anchors.n * self.anchors.k, [cam], tiles=[self.tile],
                                            max_dup=self.max_dup, split=self.split, outputs=self.OUTPUTS)
        else:
            r.move([cam])
        return r

    def _render(self, cam, origin, precision):
        self.model.decode(self.anchors, origin, precision=precision, out=self.table)
        r = self.renderer(cam)
        r.render(self.table)
        return r

    def render(self, cam, origin, precision=gsr.DECODE_BF16_TENSOR):
        """Decode and render `cam`; returns the plan's outputs (rgb, depth, alpha, ...)."""
        return self._render(cam, origin, precision).out[0]

    def step(self, cam, target, origin, precision=gsr.DECODE_BF16_TENSOR, lr=3e-3, lr_feature=1e-2):
        """One training step on `cam`'s frame against `target` (3 x H x W);
        returns the loss tensor (on the device: [total, l1, distortion, normal])."""
        from .frame import camera_backward, camera_loss
        r = self._render(cam, origin, precision)
        loss, lo = camera_loss(r, 0, target, w_dist=self.w_dist, w_normal=self.w_normal)
        for g in self.grads.values():
            g.zero_()
        camera_backward(r, 0, lo.struct(), self.table, out=self.grads)
        self.model.zero_grads(self.anchors)
        self.model.backward(self.anchors, origin, self.grads)
        self.model.adam_step(self.anchors, lr=lr, lr_feature=lr_feature)
        return loss
