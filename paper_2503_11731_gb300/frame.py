"""Device buffers and a frame renderer over the C ABI (marshalling only).

PyTorch provides device memory and streams; every step of the render runs in
libgsr.so.  A `Renderer` owns one plan, its workspace and the per-sensor
output tensors, and renders a frame with gsr_preprocess -> gsr_bin_sort ->
gsr_render_camera / gsr_render_lidar on the current CUDA stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import gsr


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class DeviceSurfels:
    """Surfel table on the device (float32, contiguous, 16-byte aligned rows)."""

    def __init__(self, pos, log_scale, quat, opacity, sh, intensity=None, obj_id=None, ray_drop=None, sees=0):
        """`ray_drop`: LiDAR ray-drop logits (None: rho = 0); `sees`: which
        sensors render the table (gsr.SEES_CAMERAS | gsr.SEES_LIDARS, 0 = all)."""
        self.pos, self.log_scale, self.quat, self.opacity, self.sh = pos, log_scale, quat, opacity, sh
        self.intensity, self.obj_id, self.ray_drop, self.sees = intensity, obj_id, ray_drop, int(sees)
        for t in (pos, log_scale, quat, opacity, sh):
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()

    @classmethod
    def from_host(cls, s, device="cuda", sees=0):
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=device)
        rd = getattr(s, "ray_drop", None)
        return cls(f(s.pos), f(s.log_scale), f(s.quat), f(s.opacity), f(s.sh), f(s.intensity),
                   None if getattr(s, "obj_id", None) is None else
                   torch.as_tensor(np.ascontiguousarray(s.obj_id, np.int32), device=device),
                   None if rd is None else f(rd), sees)

    @property
    def n(self):
        return int(self.pos.shape[0])

    @property
    def sh_degree(self):
        return int(round(self.sh.shape[1] ** 0.5)) - 1

    def struct(self) -> gsr.Surfels:
        return gsr.Surfels(self.n, self.sh_degree, _ptr(self.pos), _ptr(self.log_scale), _ptr(self.quat),
                           _ptr(self.opacity), _ptr(self.sh), _ptr(self.intensity), _ptr(self.obj_id),
                           _ptr(self.ray_drop), self.sees)


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Renderer:
    """One plan (surfel count, sensors, tiling) with its workspace and outputs."""

    def __init__(self, n_surfels, sensors, tile=(16, 16), max_dup=0, bg=(0.0, 0.0, 0.0), device="cuda",
                 outputs=("rgb", "depth", "normal", "alpha", "trans", "n_contrib"), tiles=None, batch_depth=0,
                 split=(0, 0), lidar_split=None):
        """`tile` is the default tiling; `tiles` (optional) a per-sensor list of (w, h) or None;
        `batch_depth` the records staged per step of a tile walk (0 = the CTA's thread count);
        `split` = (split_first, split_chunk) of long tile lists (0 = the library's defaults);
        `lidar_split` the LiDARs' own (None = the plan's)."""
        self.descs = list(sensors)
        tiles = tiles if tiles is not None else [None] * len(self.descs)
        if len(tiles) != len(self.descs):
            raise ValueError(f"{len(tiles)} tiles for {len(self.descs)} sensors")
        self.structs = [gsr.sensor(d, bg, t, lidar_split if d.kind == "lidar" else None)
                        for d, t in zip(self.descs, tiles)]
        self.plan = gsr.plan_init(n_surfels, self.structs, tile, max_dup, batch_depth, split)
        self.ws_bytes = gsr.workspace_size(self.plan)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=device)
        base = self.ws.data_ptr()
        self.ws_ptr = ctypes.c_void_p((base + 255) & ~255)
        self.device = device
        self.out = []
        for d in self.descs:
            H, W = (d.beams, d.columns) if d.kind == "lidar" else (d.height, d.width)
            o = {}
            if d.kind == "lidar":
                for k in ("range", "intensity", "alpha", "trans", "drop"):
                    if k in outputs or k in ("range", "intensity"):
                        o[k] = torch.zeros(H, W, device=device)
                for k in ("n_contrib", "n_walk"):
                    if k in outputs:
                        o[k] = torch.zeros(H, W, dtype=torch.int32, device=device)
            else:
                if "rgb" in outputs:
                    o["rgb"] = torch.zeros(3, H, W, device=device)
                if "normal" in outputs:
                    o["normal"] = torch.zeros(3, H, W, device=device)
                for k in ("depth", "alpha", "trans"):
                    if k in outputs:
                        o[k] = torch.zeros(H, W, device=device)
                if "depth_acc" in outputs:
                    o["depth_acc"] = torch.zeros(2, H, W, device=device)
                for k in ("n_contrib", "n_walk"):
                    if k in outputs:
                        o[k] = torch.zeros(H, W, dtype=torch.int32, device=device)
            self.out.append(o)

    def _out_struct(self, i):
        o = self.out[i]
        g = lambda k: _ptr(o.get(k))
        if self.descs[i].kind == "lidar":
            return gsr.LidarOut(g("range"), g("intensity"), g("alpha"), g("trans"), g("n_contrib"), g("n_walk"),
                                g("drop"))
        return gsr.CameraOut(g("rgb"), g("depth"), g("normal"), g("alpha"), g("trans"), g("depth_acc"),
                             g("n_contrib"), g("n_walk"))

    def move(self, sensors):
        """New poses for the plan's sensors (same models, sizes and tiling):
        the plan is re-initialised on the host, the workspace and outputs stay."""
        sensors = list(sensors)
        if len(sensors) != len(self.descs):
            raise ValueError("move() keeps the plan's sensors")
        structs = []
        for i, d in enumerate(sensors):
            st = gsr.sensor(d)
            old = self.plan.sensors[i]
            st.tile_w, st.tile_h = old.tile_w, old.tile_h
            st.split_first, st.split_chunk = old.split_first, old.split_chunk
            st.bg = old.bg
            structs.append(st)
        t = self.plan.tiling
        plan = gsr.plan_init(self.plan.n_surfels, structs, (t.tile_w, t.tile_h), self.plan.max_dup, t.batch_depth,
                             (t.split_first, t.split_chunk))
        if gsr.workspace_size(plan) != self.ws_bytes:
            raise ValueError("move() changed the workspace layout")
        self.plan, self.descs, self.structs = plan, sensors, structs

    def preprocess(self, surfels: DeviceSurfels, objects=None, stream=None, first=None):
        """Whole plan (first None), or surfels [first, first + n) of it (gsr_preprocess_part)."""
        obj = None
        if objects is not None:
            obj = gsr.Objects(int(objects.shape[0]), _ptr(objects))
        if first is None:
            gsr.preprocess(self.plan, surfels.struct(), obj, self.ws_ptr, self.ws_bytes, _stream_handle(stream))
        else:
            gsr.preprocess_part(self.plan, surfels.struct(), obj, first, self.ws_ptr, self.ws_bytes,
                                _stream_handle(stream))

    def bin_sort(self, stream=None):
        gsr.bin_sort(self.plan, self.ws_ptr, self.ws_bytes, _stream_handle(stream))

    def composite(self, sensors=None, stream=None):
        h = _stream_handle(stream)
        for i in (range(len(self.descs)) if sensors is None else sensors):
            if self.descs[i].kind == "lidar":
                gsr.render_lidar(self.plan, self.ws_ptr, self.ws_bytes, i, self._out_struct(i), h)
            else:
                gsr.render_camera(self.plan, self.ws_ptr, self.ws_bytes, i, self._out_struct(i), h)

    def render(self, surfels: DeviceSurfels, objects=None, stream=None):
        self.preprocess(surfels, objects, stream)
        self.bin_sort(stream)
        self.composite(None, stream)
        return self.out

    def composite_rig(self, stream=None):
        """Every sensor in one persistent launch (gsr_render_rig)."""
        gsr.render_rig(self.plan, self.ws_ptr, self.ws_bytes, [self._out_struct(i) for i in range(len(self.descs))],
                       _stream_handle(stream))

    def render_rig(self, surfels: DeviceSurfels, objects=None, stream=None):
        self.preprocess(surfels, objects, stream)
        self.bin_sort(stream)
        self.composite_rig(stream)
        return self.out

    def graph(self, surfels: DeviceSurfels, objects=None, stages=7, stream=None):
        """Capture the selected stages of a frame (gsr_frame_graph_create) on a
        side stream; replay with .launch(stream).  Keeps every pointer."""
        obj = None if objects is None else gsr.Objects(int(objects.shape[0]), _ptr(objects))
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        g = gsr.FrameGraph(self.plan, surfels.struct(), obj, self.ws_ptr, self.ws_bytes,
                           [self._out_struct(i) for i in range(len(self.descs))], stages, _stream_handle(side))
        torch.cuda.current_stream().wait_stream(side)
        g._keep = (surfels, objects, side)
        return g

    def _alloc_workspace(self, nbytes):
        if getattr(self, "ws", None) is None or self.ws.numel() < nbytes + 256:
            self.ws = None
            self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = ctypes.c_void_p((self.ws.data_ptr() + 255) & ~255)

    def autotune(self, parts, objects=None, camera_tiles=((16, 16), (16, 8), (8, 16), (8, 8), (32, 8)),
                 lidar_tiles=((8, 8), (4, 8), (16, 8), (16, 4), (32, 4), (32, 2), (32, 1), (64, 1)),
                 batch_depths=(64, 128, 256),
                 split_firsts=(4096, 8192, 16384, 32768), split_chunks=(256, 384, 512, 1024),
                 lidar_split_firsts=(1024, 2048, 4096, 8192), lidar_split_chunks=(128, 256, 512, 1024), warmup=1,
                 reps=3, stream=None):
        """Pick the tiling of this rig with gsr_autotune over `parts` (DeviceSurfels
        consecutive in the plan) and re-plan with it; returns the trial list.
        The LiDARs first share one tile, then each is tuned on its own."""
        obj = None if objects is None else gsr.Objects(int(objects.shape[0]), _ptr(objects))
        has = {d.kind for d in self.descs}
        lid = "lidar" in has
        space = gsr.autotune_space(camera_tiles if has - {"lidar"} else (), lidar_tiles if lid else (),
                                   batch_depths, warmup, reps, split_firsts, split_chunks,
                                   lidar_split_firsts if lid else (), lidar_split_chunks if lid else ())
        need = gsr.autotune_workspace_size(self.plan, space)
        self._alloc_workspace(need)
        res = gsr.autotune(self.plan, [p.struct() for p in parts], obj, space, self.ws_ptr, need,
                           [self._out_struct(i) for i in range(len(self.descs))], _stream_handle(stream))
        self.plan = res.plan
        self.ws_bytes = gsr.workspace_size(self.plan)
        self._alloc_workspace(self.ws_bytes)
        nl = sum(d.kind == "lidar" for d in self.descs)
        trials = [{"camera_tile": tuple(t.camera_tile), "lidar_tile": tuple(t.lidar_tile),
                   "lidar_tiles": [tuple(x) for x in list(t.lidar_tiles)[:max(nl, 1)]],
                   "batch_depth": t.batch_depth, "split": (t.split_first, t.split_chunk),
                   "lidar_split": (t.lidar_split_first, t.lidar_split_chunk), "ms": t.ms}
                  for t in res.tried[:res.n_tried]]
        return {"best_ms": res.best_ms, "trials": trials, "camera_tile": self.tile_of("camera"),
                "lidar_tile": self.tile_of("lidar"), "batch_depth": self.plan.tiling.batch_depth,
                "split": (self.plan.tiling.split_first, self.plan.tiling.split_chunk),
                "lidar_split": self.lidar_split()}

    def lidar_split(self):
        """(split_first, split_chunk) of the first LiDAR (0 = the plan's), or None."""
        for i, d in enumerate(self.descs):
            if d.kind == "lidar":
                s = self.plan.sensors[i]
                return (s.split_first, s.split_chunk)
        return None

    def tile_of(self, kind):
        """Tile of the first sensor of `kind` ("camera" = pinhole or cylindrical)."""
        for i, d in enumerate(self.descs):
            if d.kind == kind or (kind == "camera" and d.kind != "lidar"):
                s = self.plan.sensors[i]
                return (s.tile_w, s.tile_h)
        return None

    def status(self, stream=None):
        """(device status, visible slots, tile/surfel pairs requested); synchronises."""
        return gsr.read_status(self.plan, self.ws_ptr, _stream_handle(stream))

    def region(self, which, dtype, count=None):
        """A workspace region as a tensor view (for tests)."""
        ptr, nbytes = gsr.workspace_region(self.plan, self.ws_ptr, which)
        off = ptr - self.ws.data_ptr()
        itemsize = torch.tensor([], dtype=dtype).element_size()
        n = nbytes // itemsize if count is None else count
        return self.ws[off:off + n * itemsize].view(dtype)


# ----------------------------------------------------------------- training
class LossOutputs:
    """Per-pixel gradient buffers of gsr_loss for one camera."""

    def __init__(self, H, W, device):
        self.rgb = torch.zeros(3, H, W, device=device)
        self.alpha = torch.zeros(H, W, device=device)
        self.depth_acc = torch.zeros(2, H, W, device=device)
        self.normal = torch.zeros(3, H, W, device=device)
        self.loss = torch.zeros(4, device=device)

    def struct(self):
        return gsr.CameraGrad(_ptr(self.rgb), _ptr(self.alpha), _ptr(self.depth_acc), _ptr(self.normal))


def _grad_struct(g):
    return gsr.SurfelGrads(_ptr(g["pos"]), _ptr(g["log_scale"]), _ptr(g["quat"]), _ptr(g["opacity"]),
                           _ptr(g["sh"]), _ptr(g.get("intensity")), _ptr(g.get("ray_drop")))


class LidarLossOutputs:
    """Per-ray gradient buffers of gsr_lidar_loss for one LiDAR."""

    def __init__(self, B, C, device):
        self.intensity = torch.zeros(B, C, device=device)
        self.alpha = torch.zeros(B, C, device=device)
        self.depth_acc = torch.zeros(2, B, C, device=device)
        self.ray_drop = torch.zeros(B, C, device=device)
        self.loss = torch.zeros(4, device=device)

    def struct(self):
        return gsr.LidarGrad(_ptr(self.intensity), _ptr(self.alpha), _ptr(self.depth_acc), _ptr(self.ray_drop))


def lidar_loss(r: Renderer, sensor, target_range, target_intensity, w_range=1.0, w_intensity=1.0, w_drop=0.1,
               stream=None):
    """gsr_lidar_loss on the last render of LiDAR `sensor` (needs range,
    intensity, alpha and drop outputs).  Returns (loss[4] tensor, LidarLossOutputs)."""
    o = r.out[sensor]
    B, C = o["alpha"].shape
    bufs = r.__dict__.setdefault("_lidar_loss_bufs", {})
    lo = bufs.get(sensor)
    if lo is None:
        lo = bufs[sensor] = LidarLossOutputs(B, C, r.device)
    tr, ti = target_range.contiguous(), target_intensity.contiguous()
    gsr.lidar_loss(r.plan, r.ws_ptr, r.ws_bytes, sensor, r._out_struct(sensor), _ptr(tr), _ptr(ti),
                   gsr.LidarLossWeights(w_range, w_intensity, w_drop), _ptr(lo.loss), lo.struct(),
                   _stream_handle(stream))
    return lo.loss, lo


def lidar_backward(r: Renderer, sensor, grad: "gsr.LidarGrad", surfels: DeviceSurfels, objects=None, out=None,
                   stream=None):
    """gsr_backward_render_lidar + gsr_backward_preprocess for one LiDAR:
    d(loss)/d(surfel parameters incl. intensity and ray-drop logit),
    accumulated into `out` (dict of tensors)."""
    if out is None:
        keys = ["pos", "log_scale", "quat", "opacity", "sh", "intensity"]
        if surfels.ray_drop is not None:
            keys.append("ray_drop")
        out = {k: torch.zeros_like(getattr(surfels, k)) for k in keys}
    h = _stream_handle(stream)
    obj = None if objects is None else gsr.Objects(int(objects.shape[0]), _ptr(objects))
    gsr.backward_render_lidar(r.plan, r.ws_ptr, r.ws_bytes, sensor, r._out_struct(sensor), grad, 0, h)
    gsr.backward_preprocess(r.plan, r.ws_ptr, r.ws_bytes, surfels.struct(), obj, _grad_struct(out), h)
    return out


def camera_loss(r: Renderer, sensor, target, w_dist=0.1, w_normal=0.05, mask_alpha=0.5, stream=None):
    """gsr_loss on the last render of camera `sensor` (needs rgb, alpha,
    depth_acc, normal outputs).  Returns (loss[4] tensor, LossOutputs)."""
    o = r.out[sensor]
    H, W = o["alpha"].shape
    lo = getattr(r, "_loss_bufs", {}).get(sensor)
    if lo is None:
        lo = LossOutputs(H, W, r.device)
        r._loss_bufs = getattr(r, "_loss_bufs", {})
        r._loss_bufs[sensor] = lo
    target = target.contiguous()
    gsr.loss(r.plan, r.ws_ptr, r.ws_bytes, sensor, r._out_struct(sensor), _ptr(target),
             gsr.LossWeights(w_dist, w_normal, mask_alpha), _ptr(lo.loss), lo.struct(), _stream_handle(stream))
    return lo.loss, lo


def camera_backward(r: Renderer, sensor, grad: "gsr.CameraGrad", surfels: DeviceSurfels, objects=None,
                    out=None, stream=None):
    """gsr_backward for one camera: d(loss)/d(surfel parameters), accumulated into `out` (dict of tensors)."""
    if out is None:
        out = {k: torch.zeros_like(getattr(surfels, k)) for k in ("pos", "log_scale", "quat", "opacity", "sh")}
    h = _stream_handle(stream)
    obj = None if objects is None else gsr.Objects(int(objects.shape[0]), _ptr(objects))
    gsr.backward_render(r.plan, r.ws_ptr, r.ws_bytes, sensor, r._out_struct(sensor), grad, 0, h)
    gsr.backward_preprocess(r.plan, r.ws_ptr, r.ws_bytes, surfels.struct(), obj, _grad_struct(out), h)
    return out


class RenderCameraFunction(torch.autograd.Function):
    """Differentiable render of one camera through the C ABI.

    forward: (pos, log_scale, quat, opacity, sh) -> (rgb, alpha, depth_acc, normal)
    backward: gsr_backward_render + gsr_backward_preprocess.
    The renderer's buffers hold the forward state: one forward/backward pair
    per renderer is in flight at a time.
    """

    @staticmethod
    def forward(ctx, renderer, sensor, pos, log_scale, quat, opacity, sh):
        surf = DeviceSurfels(pos.detach().contiguous(), log_scale.detach().contiguous(),
                             quat.detach().contiguous(), opacity.detach().contiguous(), sh.detach().contiguous())
        renderer.render(surf)
        o = renderer.out[sensor]
        ctx.renderer, ctx.sensor, ctx.surf = renderer, sensor, surf
        return o["rgb"].clone(), o["alpha"].clone(), o["depth_acc"].clone(), o["normal"].clone()

    @staticmethod
    def backward(ctx, g_rgb, g_alpha, g_dacc, g_normal):
        z = lambda t, ref: torch.zeros_like(ref) if t is None else t.contiguous()
        o = ctx.renderer.out[ctx.sensor]
        g_rgb, g_alpha = z(g_rgb, o["rgb"]), z(g_alpha, o["alpha"])
        g_dacc, g_normal = z(g_dacc, o["depth_acc"]), z(g_normal, o["normal"])
        cg = gsr.CameraGrad(_ptr(g_rgb), _ptr(g_alpha), _ptr(g_dacc), _ptr(g_normal))
        g = camera_backward(ctx.renderer, ctx.sensor, cg, ctx.surf)
        return None, None, g["pos"], g["log_scale"], g["quat"], g["opacity"], g["sh"]


class CameraLossFunction(torch.autograd.Function):
    """gsr_loss as an autograd node: (rgb, alpha, depth_acc, normal) -> scalar loss."""

    @staticmethod
    def forward(ctx, renderer, sensor, target, rgb, alpha, depth_acc, normal, w_dist=0.1, w_normal=0.05):
        o = renderer.out[sensor]
        for k, t in (("rgb", rgb), ("alpha", alpha), ("depth_acc", depth_acc), ("normal", normal)):
            o[k].copy_(t)
        loss, lo = camera_loss(renderer, sensor, target, w_dist, w_normal)
        ctx.grads = (lo.rgb.clone(), lo.alpha.clone(), lo.depth_acc.clone(), lo.normal.clone())
        return loss[0].clone()

    @staticmethod
    def backward(ctx, g):
        gr, ga, gd, gn = (t * g for t in ctx.grads)
        return None, None, None, gr, ga, gd, gn, None, None
