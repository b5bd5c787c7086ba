"""Thin ctypes binding of the C ABI in include/gsr.h (argument marshalling only).

Every function keeps the C name without the `gsr_` prefix and forwards to
libgsr.so; all rendering work runs in the library's CUDA kernels.  Loading
fails loudly (ImportError) when the library is missing: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgsr.so")

MAX_SENSORS = 16
PINHOLE, LIDAR, CYLINDRICAL = 0, 1, 2

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_WORKSPACE, ERR_CAPACITY, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_TOO_LARGE = range(8)
NOALLOC_MAX_PIXELS = 2097152

c_i32, c_i64, c_u64, c_f32, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float, ctypes.c_void_p


class Surfels(ctypes.Structure):
    _fields_ = [("n", c_i32), ("sh_degree", c_i32), ("pos", c_vp), ("log_scale", c_vp), ("quat", c_vp),
                ("opacity", c_vp), ("sh", c_vp), ("intensity", c_vp), ("obj_id", c_vp), ("ray_drop", c_vp),
                ("sees", c_i32)]


class Objects(ctypes.Structure):
    _fields_ = [("n_objects", c_i32), ("pose", c_vp)]


class Sensor(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("width", c_i32), ("height", c_i32),
                ("fx", c_f32), ("fy", c_f32), ("cx", c_f32), ("cy", c_f32),
                ("el_min_deg", c_f32), ("el_max_deg", c_f32), ("az0_deg", c_f32), ("near_plane", c_f32),
                ("world_to_sensor", c_f32 * 16), ("bg", c_f32 * 3), ("tile_w", c_i32), ("tile_h", c_i32),
                ("split_first", c_i32), ("split_chunk", c_i32)]


class Tiling(ctypes.Structure):
    _fields_ = [("tile_w", c_i32), ("tile_h", c_i32), ("batch_depth", c_i32), ("split_first", c_i32),
                ("split_chunk", c_i32)]


class Plan(ctypes.Structure):
    _fields_ = [("n_surfels", c_i32), ("n_sensors", c_i32), ("sensors", Sensor * MAX_SENSORS),
                ("tiling", Tiling), ("max_dup", c_i64), ("tiles_x", c_i32 * MAX_SENSORS),
                ("tiles_y", c_i32 * MAX_SENSORS), ("tile_base", c_i32 * (MAX_SENSORS + 1)),
                ("sort_ctas", c_i32), ("off", c_u64 * 32), ("workspace_bytes", c_u64)]


class CameraOut(ctypes.Structure):
    _fields_ = [("rgb", c_vp), ("depth", c_vp), ("normal", c_vp), ("alpha", c_vp), ("trans", c_vp),
                ("depth_acc", c_vp), ("n_contrib", c_vp), ("n_walk", c_vp)]


class LidarOut(ctypes.Structure):
    _fields_ = [("range", c_vp), ("intensity", c_vp), ("alpha", c_vp), ("trans", c_vp), ("n_contrib", c_vp),
                ("n_walk", c_vp), ("ray_drop", c_vp)]


class CameraGrad(ctypes.Structure):
    _fields_ = [("rgb", c_vp), ("alpha", c_vp), ("depth_acc", c_vp), ("normal", c_vp)]


class LidarGrad(ctypes.Structure):
    _fields_ = [("intensity", c_vp), ("alpha", c_vp), ("depth_acc", c_vp), ("ray_drop", c_vp)]


class LidarLossWeights(ctypes.Structure):
    _fields_ = [("w_range", c_f32), ("w_intensity", c_f32), ("w_drop", c_f32)]


class SurfelGrads(ctypes.Structure):
    _fields_ = [("pos", c_vp), ("log_scale", c_vp), ("quat", c_vp), ("opacity", c_vp), ("sh", c_vp),
                ("intensity", c_vp), ("ray_drop", c_vp)]


class LossWeights(ctypes.Structure):
    _fields_ = [("w_dist", c_f32), ("w_normal", c_f32), ("mask_alpha", c_f32)]


class Anchors(ctypes.Structure):
    _fields_ = [("n", c_i32), ("k", c_i32), ("feat_dim", c_i32), ("pos", c_vp), ("feature", c_vp), ("scale", c_vp),
                ("offsets", c_vp), ("intensity", c_vp)]


class Mlp(ctypes.Structure):
    _fields_ = [("hidden", c_i32), ("w1", c_vp), ("b1", c_vp), ("w2", c_vp), ("b2", c_vp), ("head", c_i32)]


class MlpGrads(ctypes.Structure):
    _fields_ = [("w1", c_vp), ("b1", c_vp), ("w2", c_vp), ("b2", c_vp), ("feature", c_vp)]


class SurfelTable(ctypes.Structure):
    _fields_ = [("pos", c_vp), ("log_scale", c_vp), ("quat", c_vp), ("opacity", c_vp), ("sh", c_vp),
                ("intensity", c_vp), ("ray_drop", c_vp)]


AUTOTUNE_MAX = 8


class AutotuneSpace(ctypes.Structure):
    _fields_ = [("n_camera_tiles", c_i32), ("camera_tiles", (c_i32 * 2) * AUTOTUNE_MAX),
                ("n_lidar_tiles", c_i32), ("lidar_tiles", (c_i32 * 2) * AUTOTUNE_MAX),
                ("n_batch_depths", c_i32), ("batch_depths", c_i32 * AUTOTUNE_MAX),
                ("n_split_firsts", c_i32), ("split_firsts", c_i32 * AUTOTUNE_MAX),
                ("n_split_chunks", c_i32), ("split_chunks", c_i32 * AUTOTUNE_MAX),
                ("n_lidar_split_firsts", c_i32), ("lidar_split_firsts", c_i32 * AUTOTUNE_MAX),
                ("n_lidar_split_chunks", c_i32), ("lidar_split_chunks", c_i32 * AUTOTUNE_MAX),
                ("warmup", c_i32), ("reps", c_i32)]


AUTOTUNE_LIDARS = 4


class AutotuneTrial(ctypes.Structure):
    _fields_ = [("camera_tile", c_i32 * 2), ("lidar_tile", c_i32 * 2), ("batch_depth", c_i32),
                ("split_first", c_i32), ("split_chunk", c_i32), ("lidar_split_first", c_i32),
                ("lidar_split_chunk", c_i32), ("lidar_tiles", (c_i32 * 2) * AUTOTUNE_LIDARS), ("ms", c_f32)]


class AutotuneResult(ctypes.Structure):
    _fields_ = [("plan", Plan), ("best_ms", c_f32), ("n_tried", c_i32),
                ("tried", AutotuneTrial * ((7 + AUTOTUNE_LIDARS) * AUTOTUNE_MAX + 1))]


class ZoneGrid(ctypes.Structure):
    _fields_ = [("x0", c_f32), ("y0", c_f32), ("zone_size", c_f32), ("padding", c_f32), ("nx", c_i32),
                ("ny", c_i32)]


class Streamer(ctypes.Structure):
    _fields_ = [("capacity", c_i32), ("sh_degree", c_i32), ("buf", SurfelTable * 2), ("zone", c_i32 * 2),
                ("count", c_i32 * 2), ("front", c_i32), ("released_valid", c_i32 * 2), ("copy_stream", c_vp),
                ("ready", c_vp * 2), ("released", c_vp * 2)]


DECODE_BF16_TENSOR, DECODE_F32 = 0, 1
HEAD_CAMERA, HEAD_LIDAR = 0, 1
SEES_CAMERAS, SEES_LIDARS = 1, 2

_STRUCTS = [Plan, Sensor, Surfels, Objects, CameraOut, LidarOut, Tiling, CameraGrad, SurfelGrads, LossWeights,
            Anchors, Mlp, MlpGrads, SurfelTable, AutotuneSpace, AutotuneResult, ZoneGrid, Streamer, LidarGrad,
            LidarLossWeights]

# exported symbols and their ctypes signatures (restype, argtypes)
SIGNATURES = {
    "gsr_plan_init": (c_i32, [ctypes.POINTER(Plan), c_i32, ctypes.POINTER(Sensor), c_i32,
                              ctypes.POINTER(Tiling), c_i64]),
    "gsr_workspace_size": (c_i32, [ctypes.POINTER(Plan), ctypes.POINTER(ctypes.c_size_t)]),
    "gsr_preprocess": (c_i32, [ctypes.POINTER(Plan), ctypes.POINTER(Surfels), ctypes.POINTER(Objects),
                               c_vp, ctypes.c_size_t, c_vp]),
    "gsr_preprocess_part": (c_i32, [ctypes.POINTER(Plan), ctypes.POINTER(Surfels), ctypes.POINTER(Objects),
                                    c_i32, c_vp, ctypes.c_size_t, c_vp]),
    "gsr_bin_sort": (c_i32, [ctypes.POINTER(Plan), c_vp, ctypes.c_size_t, c_vp]),
    "gsr_render_camera": (c_i32, [ctypes.POINTER(Plan), c_vp, ctypes.c_size_t, c_i32,
                                  ctypes.POINTER(CameraOut), c_vp]),
    "gsr_render_lidar": (c_i32, [ctypes.POINTER(Plan), c_vp, ctypes.c_size_t, c_i32,
                                 ctypes.POINTER(LidarOut), c_vp]),
    "gsr_read_status": (c_i32, [ctypes.POINTER(Plan), c_vp, ctypes.POINTER(c_i32), ctypes.POINTER(c_i64),
                                ctypes.POINTER(c_i64), c_vp]),
    "gsr_fma_peak_kernel": (c_i32, [c_vp, c_i32, c_i32, ctypes.POINTER(c_i64), c_vp]),
    "gsr_selftest_wait_timeout": (c_i32, [ctypes.POINTER(Plan), c_vp, ctypes.c_size_t, ctypes.c_uint32, c_vp]),
    "gsr_status_string": (ctypes.c_char_p, [c_i32]),
    "gsr_last_cuda_error": (ctypes.c_char_p, []),
    "gsr_workspace_region": (c_i32, [ctypes.POINTER(Plan), c_vp, c_i32, ctypes.POINTER(c_vp),
                                     ctypes.POINTER(ctypes.c_size_t)]),
    "gsr_struct_size": (ctypes.c_size_t, [c_i32]),
    "gsr_autotune_workspace_size": (c_i32, [ctypes.POINTER(Plan), ctypes.POINTER(AutotuneSpace),
                                            ctypes.POINTER(ctypes.c_size_t)]),
    "gsr_autotune": (c_i32, [ctypes.POINTER(Plan), ctypes.POINTER(Surfels), c_i32, ctypes.POINTER(Objects),
                             ctypes.POINTER(AutotuneSpace), c_vp, ctypes.c_size_t, ctypes.POINTER(CameraOut),
                             ctypes.POINTER(LidarOut), ctypes.POINTER(AutotuneResult), c_vp]),
    "gsr_loss": (c_i32, [ctypes.POINTER(Plan), c_vp, ctypes.c_size_t, c_i32, ctypes.POINTER(CameraOut), c_vp,
                         ctypes.POINTER(LossWeights), c_vp, ctypes.POINTER(CameraGrad), c_vp]),
    "gsr_backward_render": (c_i32, [ctypes.POINTER(Plan), c_vp, ctypes.c_size_t, c_i32, ctypes.POINTER(CameraOut),
                                    ctypes.POINTER(CameraGrad), c_i32, c_vp]),
    "gsr_lidar_loss": (c_i32, [ctypes.POINTER(Plan), c_vp, ctypes.c_size_t, c_i32, ctypes.POINTER(LidarOut), c_vp,
                               c_vp, ctypes.POINTER(LidarLossWeights), c_vp, ctypes.POINTER(LidarGrad), c_vp]),
    "gsr_backward_render_lidar": (c_i32, [ctypes.POINTER(Plan), c_vp, ctypes.c_size_t, c_i32,
                                          ctypes.POINTER(LidarOut), ctypes.POINTER(LidarGrad), c_i32, c_vp]),
    "gsr_backward_preprocess": (c_i32, [ctypes.POINTER(Plan), c_vp, ctypes.c_size_t, ctypes.POINTER(Surfels),
                                        ctypes.POINTER(Objects), ctypes.POINTER(SurfelGrads), c_vp]),
    "gsr_render_rig": (c_i32, [ctypes.POINTER(Plan), c_vp, ctypes.c_size_t, ctypes.POINTER(CameraOut),
                               ctypes.POINTER(LidarOut), c_vp]),
    "gsr_frame_graph_create": (c_i32, [ctypes.POINTER(Plan), ctypes.POINTER(Surfels), ctypes.POINTER(Objects), c_vp,
                                       ctypes.c_size_t, ctypes.POINTER(CameraOut), ctypes.POINTER(LidarOut), c_i32,
                                       c_vp, ctypes.POINTER(c_vp)]),
    "gsr_frame_graph_launch": (c_i32, [c_vp, c_vp]),
    "gsr_frame_graph_destroy": (c_i32, [c_vp]),
    "gsr_decode_anchors": (c_i32, [ctypes.POINTER(Anchors), ctypes.POINTER(Mlp), ctypes.POINTER(c_f32),
                                   ctypes.POINTER(Sensor), c_i32, ctypes.POINTER(SurfelTable), c_vp, c_vp]),
    "gsr_decode_backward": (c_i32, [ctypes.POINTER(Anchors), ctypes.POINTER(Mlp), ctypes.POINTER(c_f32),
                                    ctypes.POINTER(Sensor), ctypes.POINTER(SurfelGrads), ctypes.POINTER(MlpGrads),
                                    c_vp]),
    "gsr_adam": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, c_f32, c_f32, c_f32, c_f32, c_i32, c_vp]),
    "gsr_zone_of": (c_i32, [ctypes.POINTER(ZoneGrid), c_f32, c_f32]),
    "gsr_zone_count": (c_i32, [ctypes.POINTER(ZoneGrid), c_vp, c_i64, c_vp]),
    "gsr_zone_members": (c_i32, [ctypes.POINTER(ZoneGrid), c_vp, c_i64, c_vp, c_vp]),
    "gsr_zone_pack": (c_i32, [ctypes.POINTER(Surfels), c_vp, c_i64, ctypes.POINTER(SurfelTable)]),
    "gsr_streamer_init": (c_i32, [ctypes.POINTER(Streamer), c_i32, c_i32, ctypes.POINTER(SurfelTable), c_vp]),
    "gsr_streamer_prefetch": (c_i32, [ctypes.POINTER(Streamer), c_i32, ctypes.POINTER(Surfels)]),
    "gsr_streamer_acquire": (c_i32, [ctypes.POINTER(Streamer), c_i32, c_vp, ctypes.POINTER(Surfels)]),
    "gsr_streamer_destroy": (c_i32, [ctypes.POINTER(Streamer)]),
    "gsr_loss_noalloc": (c_i32, [ctypes.POINTER(Sensor), ctypes.POINTER(CameraOut), c_vp,
                                 ctypes.POINTER(LossWeights), c_vp, ctypes.POINTER(CameraGrad), c_vp]),
    "gsr_backward": (c_i32, [ctypes.POINTER(Plan), c_vp, ctypes.c_size_t, c_i32, ctypes.POINTER(CameraOut),
                             ctypes.POINTER(CameraGrad), ctypes.POINTER(Surfels), ctypes.POINTER(Objects),
                             ctypes.POINTER(SurfelGrads), c_vp]),
}

_lib = None


class GsrError(RuntimeError):
    def __init__(self, code, where):
        msg = f"{where}: {status_string(code)}"
        if code == ERR_CUDA:
            msg += f" ({lib().gsr_last_cuda_error().decode()})"
        super().__init__(msg)
        self.code = code


def lib(path: str = LIB_PATH):
    """Load libgsr.so (raises ImportError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libgsr.so not built at {path}; run paper_2503_11731_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        for i, st in enumerate(_STRUCTS):
            got = L.gsr_struct_size(i)
            if got != ctypes.sizeof(st):
                raise ImportError(f"ABI mismatch for {st.__name__}: C {got} B, binding {ctypes.sizeof(st)} B")
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().gsr_status_string(int(code)).decode()


def _check(code, where):
    if code != OK:
        raise GsrError(code, where)


# ----------------------------------------------------------------- structs
def sensor(desc, bg=(0.0, 0.0, 0.0), tile=None, split=None) -> Sensor:
    """Sensor struct from a synth.Pinhole / synth.Cylindrical / synth.Lidar-like description;
    `tile` = (w, h) and `split` = (split_first, split_chunk) override the
    plan's tiling and list split for this sensor."""
    s = Sensor()
    if tile is not None:
        s.tile_w, s.tile_h = int(tile[0]), int(tile[1])
    if split is not None:
        s.split_first, s.split_chunk = int(split[0]), int(split[1])
    kind = getattr(desc, "kind", "pinhole")
    if kind == "lidar":
        s.kind = LIDAR
        s.width, s.height = int(desc.columns), int(desc.beams)
        s.el_min_deg, s.el_max_deg, s.az0_deg = float(desc.el_min_deg), float(desc.el_max_deg), float(desc.az0_deg)
    else:
        s.kind = CYLINDRICAL if kind == "cylindrical" else PINHOLE
        s.width, s.height = int(desc.width), int(desc.height)
        s.fx, s.fy, s.cx, s.cy = float(desc.fx), float(desc.fy), float(desc.cx), float(desc.cy)
    s.near_plane = float(desc.near)
    M = np.asarray(desc.world_to_sensor, np.float64).reshape(16)
    for k in range(16):
        s.world_to_sensor[k] = float(M[k])
    for k in range(3):
        s.bg[k] = float(bg[k])
    return s


def plan_init(n_surfels: int, sensors, tile=(16, 16), max_dup: int = 0, batch_depth: int = 0, split=(0, 0)) -> Plan:
    """split = (split_first, split_chunk) of long tile lists; 0 = the library's default."""
    arr = (Sensor * len(sensors))(*sensors)
    p = Plan()
    t = Tiling(int(tile[0]), int(tile[1]), int(batch_depth), int(split[0]), int(split[1]))
    _check(lib().gsr_plan_init(ctypes.byref(p), int(n_surfels), arr, len(sensors), ctypes.byref(t), int(max_dup)),
           "gsr_plan_init")
    return p


def workspace_size(plan: Plan) -> int:
    n = ctypes.c_size_t()
    _check(lib().gsr_workspace_size(ctypes.byref(plan), ctypes.byref(n)), "gsr_workspace_size")
    return int(n.value)


def preprocess(plan, surfels: Surfels, objects, ws, ws_bytes, stream):
    _check(lib().gsr_preprocess(ctypes.byref(plan), ctypes.byref(surfels),
                                ctypes.byref(objects) if objects is not None else None,
                                ws, ws_bytes, stream), "gsr_preprocess")


def preprocess_part(plan, surfels: Surfels, objects, first, ws, ws_bytes, stream):
    _check(lib().gsr_preprocess_part(ctypes.byref(plan), ctypes.byref(surfels),
                                     ctypes.byref(objects) if objects is not None else None,
                                     int(first), ws, ws_bytes, stream), "gsr_preprocess_part")


def bin_sort(plan, ws, ws_bytes, stream):
    _check(lib().gsr_bin_sort(ctypes.byref(plan), ws, ws_bytes, stream), "gsr_bin_sort")


def render_camera(plan, ws, ws_bytes, sensor_idx, out: CameraOut, stream):
    _check(lib().gsr_render_camera(ctypes.byref(plan), ws, ws_bytes, int(sensor_idx), ctypes.byref(out), stream),
           "gsr_render_camera")


def render_lidar(plan, ws, ws_bytes, sensor_idx, out: LidarOut, stream):
    _check(lib().gsr_render_lidar(ctypes.byref(plan), ws, ws_bytes, int(sensor_idx), ctypes.byref(out), stream),
           "gsr_render_lidar")


def read_status(plan, ws, stream):
    st, nv, npairs = c_i32(), c_i64(), c_i64()
    _check(lib().gsr_read_status(ctypes.byref(plan), ws, ctypes.byref(st), ctypes.byref(nv), ctypes.byref(npairs),
                                 stream), "gsr_read_status")
    return int(st.value), int(nv.value), int(npairs.value)


def fma_peak_kernel(out_ptr, blocks, iters, stream):
    """Launch the FP32 FMA-chain measurement kernel; returns the FMAs launched."""
    n = c_i64()
    _check(lib().gsr_fma_peak_kernel(out_ptr, int(blocks), int(iters), ctypes.byref(n), stream),
           "gsr_fma_peak_kernel")
    return int(n.value)


def selftest_wait_timeout(plan, ws, ws_bytes, tries, stream):
    """Make one bounded device wait give up (see gsr_selftest_wait_timeout)."""
    _check(lib().gsr_selftest_wait_timeout(ctypes.byref(plan), ws, ws_bytes, int(tries), stream),
           "gsr_selftest_wait_timeout")


def workspace_region(plan, ws, which):
    ptr, n = c_vp(), ctypes.c_size_t()
    _check(lib().gsr_workspace_region(ctypes.byref(plan), ws, int(which), ctypes.byref(ptr), ctypes.byref(n)),
           "gsr_workspace_region")
    return int(ptr.value or 0), int(n.value)


def loss(plan, ws, ws_bytes, sensor_idx, fwd: CameraOut, target, weights: LossWeights, loss_out, grad: CameraGrad,
         stream):
    _check(lib().gsr_loss(ctypes.byref(plan), ws, ws_bytes, int(sensor_idx), ctypes.byref(fwd), target,
                          ctypes.byref(weights), loss_out, ctypes.byref(grad), stream), "gsr_loss")


def backward_render(plan, ws, ws_bytes, sensor_idx, fwd: CameraOut, grad: CameraGrad, accumulate, stream):
    _check(lib().gsr_backward_render(ctypes.byref(plan), ws, ws_bytes, int(sensor_idx), ctypes.byref(fwd),
                                     ctypes.byref(grad), int(accumulate), stream), "gsr_backward_render")


def lidar_loss(plan, ws, ws_bytes, sensor_idx, fwd: LidarOut, target_range, target_intensity,
               weights: LidarLossWeights, loss_out, grad: LidarGrad, stream):
    _check(lib().gsr_lidar_loss(ctypes.byref(plan), ws, ws_bytes, int(sensor_idx), ctypes.byref(fwd), target_range,
                                target_intensity, ctypes.byref(weights), loss_out, ctypes.byref(grad), stream),
           "gsr_lidar_loss")


def backward_render_lidar(plan, ws, ws_bytes, sensor_idx, fwd: LidarOut, grad: LidarGrad, accumulate, stream):
    _check(lib().gsr_backward_render_lidar(ctypes.byref(plan), ws, ws_bytes, int(sensor_idx), ctypes.byref(fwd),
                                           ctypes.byref(grad), int(accumulate), stream), "gsr_backward_render_lidar")


def backward_preprocess(plan, ws, ws_bytes, surfels: Surfels, objects, out: SurfelGrads, stream):
    _check(lib().gsr_backward_preprocess(ctypes.byref(plan), ws, ws_bytes, ctypes.byref(surfels),
                                         ctypes.byref(objects) if objects is not None else None,
                                         ctypes.byref(out), stream), "gsr_backward_preprocess")


STAGE_PREPROCESS, STAGE_BIN_SORT, STAGE_RENDER_RIG = 1, 2, 4


def _rig_out_arrays(plan, outs):
    n = plan.n_sensors
    cams = (CameraOut * n)()
    lids = (LidarOut * n)()
    for i, o in enumerate(outs):
        if isinstance(o, CameraOut):
            cams[i] = o
        else:
            lids[i] = o
    return cams, lids


def render_rig(plan, ws, ws_bytes, outs, stream):
    """outs: per-sensor CameraOut / LidarOut structs (index = sensor)."""
    cams, lids = _rig_out_arrays(plan, outs)
    _check(lib().gsr_render_rig(ctypes.byref(plan), ws, ws_bytes, cams, lids, stream), "gsr_render_rig")


def autotune_space(camera_tiles=(), lidar_tiles=(), batch_depths=(), warmup=1, reps=3, split_firsts=(),
                   split_chunks=(), lidar_split_firsts=(), lidar_split_chunks=()) -> AutotuneSpace:
    sp = AutotuneSpace()
    for name, vals in (("camera_tiles", camera_tiles), ("lidar_tiles", lidar_tiles)):
        if len(vals) > AUTOTUNE_MAX:
            raise ValueError(f"at most {AUTOTUNE_MAX} {name}")
        setattr(sp, "n_" + name, len(vals))
        arr = getattr(sp, name)
        for i, (w, h) in enumerate(vals):
            arr[i][0], arr[i][1] = int(w), int(h)
    for name, vals in (("batch_depths", batch_depths), ("split_firsts", split_firsts),
                       ("split_chunks", split_chunks), ("lidar_split_firsts", lidar_split_firsts),
                       ("lidar_split_chunks", lidar_split_chunks)):
        if len(vals) > AUTOTUNE_MAX:
            raise ValueError(f"at most {AUTOTUNE_MAX} {name}")
        setattr(sp, "n_" + name, len(vals))
        arr = getattr(sp, name)
        for i, d in enumerate(vals):
            arr[i] = int(d)
    sp.warmup, sp.reps = int(warmup), int(reps)
    return sp


def autotune_workspace_size(plan, space: AutotuneSpace) -> int:
    n = ctypes.c_size_t()
    _check(lib().gsr_autotune_workspace_size(ctypes.byref(plan), ctypes.byref(space), ctypes.byref(n)),
           "gsr_autotune_workspace_size")
    return int(n.value)


def autotune(plan, parts, objects, space: AutotuneSpace, ws, ws_bytes, outs, stream) -> AutotuneResult:
    """parts: Surfels structs consecutive in the plan; outs as render_rig."""
    arr = (Surfels * len(parts))(*parts)
    cams, lids = _rig_out_arrays(plan, outs)
    res = AutotuneResult()
    _check(lib().gsr_autotune(ctypes.byref(plan), arr, len(parts),
                              ctypes.byref(objects) if objects is not None else None, ctypes.byref(space), ws,
                              ws_bytes, cams, lids, ctypes.byref(res), stream), "gsr_autotune")
    return res


class FrameGraph:
    """A captured frame (or the stages selected by `stages`) replayed with launch()."""

    def __init__(self, plan, surfels: Surfels, objects, ws, ws_bytes, outs, stages, stream):
        cams, lids = _rig_out_arrays(plan, outs)
        h = c_vp()
        _check(lib().gsr_frame_graph_create(ctypes.byref(plan), ctypes.byref(surfels),
                                            ctypes.byref(objects) if objects is not None else None, ws, ws_bytes,
                                            cams, lids, int(stages), stream, ctypes.byref(h)),
               "gsr_frame_graph_create")
        self.handle = h

    def launch(self, stream):
        _check(lib().gsr_frame_graph_launch(self.handle, stream), "gsr_frame_graph_launch")

    def close(self):
        if self.handle:
            lib().gsr_frame_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def decode_anchors(anchors: Anchors, mlp: Mlp, origin, cull_camera, precision, out: SurfelTable, status, stream):
    o = (c_f32 * 3)(*[float(v) for v in origin])
    _check(lib().gsr_decode_anchors(ctypes.byref(anchors), ctypes.byref(mlp), o,
                                    ctypes.byref(cull_camera) if cull_camera is not None else None, int(precision),
                                    ctypes.byref(out), status, stream), "gsr_decode_anchors")


def decode_backward(anchors: Anchors, mlp: Mlp, origin, cull_camera, d_surfels: SurfelGrads, out: MlpGrads, stream):
    o = (c_f32 * 3)(*[float(v) for v in origin])
    _check(lib().gsr_decode_backward(ctypes.byref(anchors), ctypes.byref(mlp), o,
                                     ctypes.byref(cull_camera) if cull_camera is not None else None,
                                     ctypes.byref(d_surfels), ctypes.byref(out), stream), "gsr_decode_backward")


def adam(param, grad, m, v, n, lr, beta1, beta2, eps, step, stream):
    _check(lib().gsr_adam(param, grad, m, v, int(n), float(lr), float(beta1), float(beta2), float(eps), int(step),
                          stream), "gsr_adam")


# ------------------------------------------------------------ zones
def zone_grid(x0, y0, zone_size=40.0, padding=0.25, nx=1, ny=1) -> ZoneGrid:
    return ZoneGrid(float(x0), float(y0), float(zone_size), float(padding), int(nx), int(ny))


def zone_of(grid: ZoneGrid, x, y) -> int:
    return int(lib().gsr_zone_of(ctypes.byref(grid), float(x), float(y)))


def zone_members(grid: ZoneGrid, pos):
    """(offsets [nz+1] int64, members int64) of a host float32 [n, 3] array."""
    import numpy as np
    pos = np.ascontiguousarray(pos, np.float32)
    nz = grid.nx * grid.ny
    counts = np.zeros(nz, np.int64)
    p = pos.ctypes.data_as(c_vp)
    _check(lib().gsr_zone_count(ctypes.byref(grid), p, int(pos.shape[0]), counts.ctypes.data_as(c_vp)),
           "gsr_zone_count")
    offsets = np.zeros(nz + 1, np.int64)
    offsets[1:] = np.cumsum(counts)
    members = np.zeros(int(offsets[-1]), np.int64)
    _check(lib().gsr_zone_members(ctypes.byref(grid), p, int(pos.shape[0]), offsets.ctypes.data_as(c_vp),
                                  members.ctypes.data_as(c_vp)), "gsr_zone_members")
    return offsets, members


def streamer_init(capacity, sh_degree, buffers, copy_stream) -> Streamer:
    s = Streamer()
    arr = (SurfelTable * 2)(*buffers)
    _check(lib().gsr_streamer_init(ctypes.byref(s), int(capacity), int(sh_degree), arr, copy_stream),
           "gsr_streamer_init")
    return s


def streamer_prefetch(s: Streamer, zone, host_zone: Surfels):
    _check(lib().gsr_streamer_prefetch(ctypes.byref(s), int(zone), ctypes.byref(host_zone)), "gsr_streamer_prefetch")


def streamer_acquire(s: Streamer, zone, render_stream) -> Surfels:
    out = Surfels()
    _check(lib().gsr_streamer_acquire(ctypes.byref(s), int(zone), render_stream, ctypes.byref(out)),
           "gsr_streamer_acquire")
    return out


def streamer_destroy(s: Streamer):
    _check(lib().gsr_streamer_destroy(ctypes.byref(s)), "gsr_streamer_destroy")
