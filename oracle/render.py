"""ctypes wrapper of the FP64 oracle (gsr_oracle.c): brute force, or the
same arithmetic over per-tile candidate lists (`tile` > 0).

TEST INFRASTRUCTURE, NOT PRODUCT CODE (see the package docstring).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, IEEE FP64, OpenMP).  Returns the .so path."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.POINTER(ctypes.c_int)
        L = ctypes.POINTER(ctypes.c_longlong)
        c_int, c_double = ctypes.c_int, ctypes.c_double
        lib.oracle_render_pinhole.restype = c_int
        lib.oracle_render_pinhole.argtypes = [
            c_int, D, D, D, D, c_int, D, I, D,
            c_int, c_int, c_double, c_double, c_double, c_double, c_double, D, D,
            c_int, L, c_int, D, D, D, D, D, D, D, D, I]
        lib.oracle_render_cylindrical.restype = c_int
        lib.oracle_render_cylindrical.argtypes = lib.oracle_render_pinhole.argtypes
        lib.oracle_render_lidar.restype = c_int
        lib.oracle_render_lidar.argtypes = [
            c_int, D, D, D, D, D, D, I, D,
            c_int, c_int, c_double, c_double, c_double, c_double, D,
            c_int, L, c_int, D, D, D, D, D, D, D, I]
        lib.oracle_sh_basis.restype = c_double
        lib.oracle_sh_basis.argtypes = [c_int, c_int, D]
        lib.oracle_num_threads.restype = c_int
        lib.oracle_intersect.restype = c_int
        lib.oracle_intersect.argtypes = [c_int, D, D, D, D, D, c_double, c_double, D]
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _obj(s, obj_pose):
    if getattr(s, "obj_id", None) is None or obj_pose is None:
        return None, None, None, None
    ids = np.ascontiguousarray(s.obj_id, dtype=np.int32)
    P = np.ascontiguousarray(obj_pose, dtype=np.float64).reshape(-1, 12)
    return ids, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), P, P.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def sh_basis(l: int, m: int, d) -> float:
    a, p = _d(np.asarray(d, np.float64))
    return float(_load().oracle_sh_basis(l, m, p))


def render_pinhole(s, cam, bg=(0.0, 0.0, 0.0), pixels=None, obj_pose=None, tile=0):
    """FP64 render of a camera frame: pinhole (Eq. 3) or, for
    cam.kind == "cylindrical", the cylindrical camera (Eq. 4).  tile == 0
    checks every surfel for every pixel; tile > 0 walks per-tile candidate
    lists (tile x tile pixels) from the oracle's own conservative bound,
    with the same arithmetic and bit-identical results.

    `s` holds the surfel arrays (pos, log_scale, quat, opacity, sh, obj_id);
    `cam` the intrinsics and world_to_sensor.  `pixels` (optional) lists the
    linear pixel indices y*W+x to render.  Returns a dict of numpy arrays:
    rgb [P,3], depth [P], normal [P,3], alpha [P], T [P], acc [P,3]
    (sum w, sum w z, sum w z^2), flip [P] (largest output change that an
    FP32-flippable threshold decision could cause; 0 if none), slack [P],
    slack_n [P] and slack_z [P] (bounds of the change a reordering of
    near-tied surfels can make to colour, normal and sum w z), slack_c [P]
    (bound of the change of any output, relative for depth, that FP32
    rounding can cause through the conditioning of Eq. 2, or by sorting a
    near-tied hit before the surfel that stops the ray), n_contrib [P].
    With pixels=None, arrays are reshaped to images (rgb [H,W,3], ...).
    """
    lib = _load()
    keep = []

    def D(a):
        arr, ptr = _d(a)
        keep.append(arr)
        return ptr
    ids, ids_p, P, P_p = _obj(s, obj_pose)
    keep += [ids, P]
    npix = cam.width * cam.height if pixels is None else len(pixels)
    pix_arr = None
    pix_p = None
    if pixels is not None:
        pix_arr = np.ascontiguousarray(pixels, dtype=np.int64)
        pix_p = pix_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))
    out = {k: np.zeros(sh, np.float64) for k, sh in
           [("rgb", (npix, 3)), ("depth", (npix,)), ("normal", (npix, 3)), ("alpha", (npix,)),
            ("T", (npix,)), ("acc", (npix, 3)), ("flip", (npix,)), ("slack2", (npix, 4))]}
    out["n_contrib"] = np.zeros(npix, np.int32)
    dp = {k: v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for k, v in out.items() if v.dtype == np.float64}
    deg = int(round(np.sqrt(s.sh.shape[1]))) - 1
    fn = lib.oracle_render_cylindrical if getattr(cam, "kind", "pinhole") == "cylindrical" else lib.oracle_render_pinhole
    rc = fn(
        int(s.pos.shape[0]), D(s.pos), D(s.log_scale), D(s.quat), D(s.opacity), deg, D(s.sh),
        ids_p, P_p,
        int(cam.width), int(cam.height), float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy),
        float(cam.near), D(cam.world_to_sensor), D(np.asarray(bg, np.float64)),
        int(npix), pix_p, int(tile),
        dp["rgb"], dp["depth"], dp["normal"], dp["alpha"], dp["T"], dp["acc"], dp["flip"], dp["slack2"],
        out["n_contrib"].ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc != 0:
        raise RuntimeError("oracle camera render failed")
    s2 = out.pop("slack2")
    out["slack"], out["slack_n"], out["slack_z"], out["slack_c"] = (s2[:, i].copy() for i in range(4))
    if pixels is None:
        H, W = cam.height, cam.width
        out = {k: v.reshape((H, W) + v.shape[1:]) for k, v in out.items()}
    return out


def render_lidar(s, lid, rays=None, obj_pose=None, tile=0):
    """FP64 LiDAR range image (tile as for render_pinhole; columns wrap).  Returns range, intensity, drop
    (ray-drop probability: sum w rho + T with rho = sigmoid of the surfels'
    ray_drop logit, 0 when `s` has none), alpha, T, flip, slack (intensity
    and ray drop), slack_z (sum w t), n_contrib (each
    [R], or [beams, columns] with rays=None)."""
    lib = _load()
    keep = []

    def D(a):
        arr, ptr = _d(a)
        keep.append(arr)
        return ptr
    ids, ids_p, P, P_p = _obj(s, obj_pose)
    keep += [ids, P]
    nr = lid.beams * lid.columns if rays is None else len(rays)
    ray_p = None
    if rays is not None:
        ray_arr = np.ascontiguousarray(rays, dtype=np.int64)
        keep.append(ray_arr)
        ray_p = ray_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))
    out = {k: np.zeros(nr, np.float64) for k in ("range", "intensity", "drop", "alpha", "T", "flip")}
    out["slack2"] = np.zeros((nr, 4), np.float64)
    rd = getattr(s, "ray_drop", None)
    rd_p = None if rd is None else D(rd)
    out["n_contrib"] = np.zeros(nr, np.int32)
    dp = {k: v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for k, v in out.items() if v.dtype == np.float64}
    rc = lib.oracle_render_lidar(
        int(s.pos.shape[0]), D(s.pos), D(s.log_scale), D(s.quat), D(s.opacity), D(s.intensity), rd_p,
        ids_p, P_p,
        int(lid.beams), int(lid.columns), float(lid.el_min_deg), float(lid.el_max_deg), float(lid.az0_deg),
        float(lid.near), D(lid.world_to_sensor),
        int(nr), ray_p, int(tile),
        dp["range"], dp["intensity"], dp["drop"], dp["alpha"], dp["T"], dp["flip"], dp["slack2"],
        out["n_contrib"].ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc != 0:
        raise RuntimeError("oracle_render_lidar failed")
    s2 = out.pop("slack2")
    out["slack"], out["slack_n"], out["slack_z"], out["slack_c"] = (s2[:, i].copy() for i in range(4))
    if rays is None:
        out = {k: v.reshape(lid.beams, lid.columns) for k, v in out.items()}
    return out


def intersect(kind, pos, log_scale, quat, world_to_sensor, cam=(0, 0, 0, 0), a=0.0, b=0.0):
    """Eq. 2 for one surfel: (u, v, depth) at pixel (a, b) = (px, py) for the
    pinhole (kind 0), or (u, v, distance) at (az, el) radians for LiDAR (kind 1).
    Returns None when the two plane rows are parallel."""
    lib = _load()
    keep = [np.asarray(x, np.float64).ravel().copy() for x in (pos, log_scale, quat, world_to_sensor, cam)]
    ptrs = [k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for k in keep]
    out = np.zeros(3, np.float64)
    ok = lib.oracle_intersect(int(kind), ptrs[0], ptrs[1], ptrs[2], ptrs[3], ptrs[4], float(a), float(b),
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out if ok else None
