"""Seeded synthetic inputs: surfel scenes, anchor scenes and sensor rigs.

This module only draws random numbers and builds sensor poses; it holds none
of the rendering arithmetic, so both the CUDA path and the CPU oracle can take
their inputs from it.  The paper's datasets (Para-Lane, the proprietary
driving clips, 3DRealCar) are not available, so these scenes stand in for
driving-scale inputs with the shapes, sizes and value distributions of the
workloads the renderer is measured on (Sec. III-A; Tab. 1 renders driving
clips with one camera and one spinning LiDAR).

Conventions
-----------
* world frame: z up; the road is the plane z = 0, driving direction +x.
* camera frame: x right, y down, z forward; LiDAR frame: x forward, y left,
  z up.  `world_to_sensor` is a row-major 4x4 rigid transform.
* surfel parameters (float32, one row per surfel):
  pos [N,3], log_scale [N,2], quat [N,4] (w,x,y,z, not necessarily unit),
  opacity [N] (logit), sh [N,K,3] with K = (degree+1)^2, intensity [N].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 2503_11731

# Real SH band-0 constant 1/(2 sqrt(pi)); used only to store a colour as a
# degree-0 coefficient, (rgb - 0.5) / Y00, so that the renderer reproduces it.
_Y00 = 0.28209479177387814


@dataclasses.dataclass
class Surfels:
    pos: np.ndarray
    log_scale: np.ndarray
    quat: np.ndarray
    opacity: np.ndarray
    sh: np.ndarray
    intensity: np.ndarray
    obj_id: np.ndarray | None = None  # int32 [N], -1 = background
    ray_drop: np.ndarray | None = None  # float32 [N] LiDAR ray-drop logit (None: rho = 0)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def sh_degree(self) -> int:
        return int(round(math.sqrt(self.sh.shape[1]))) - 1

    def subset(self, idx) -> "Surfels":
        return Surfels(self.pos[idx], self.log_scale[idx], self.quat[idx], self.opacity[idx],
                       self.sh[idx], self.intensity[idx],
                       None if self.obj_id is None else self.obj_id[idx],
                       None if self.ray_drop is None else self.ray_drop[idx])

    def concat(self, other: "Surfels") -> "Surfels":
        def ids(s):
            return s.obj_id if s.obj_id is not None else np.full(s.n, -1, np.int32)
        assert self.sh.shape[1] == other.sh.shape[1]
        def drops(s):
            return s.ray_drop if s.ray_drop is not None else np.full(s.n, -1e4, np.float32)
        rd = None if self.ray_drop is None and other.ray_drop is None else \
            np.concatenate([drops(self), drops(other)]).astype(np.float32)
        return Surfels(np.concatenate([self.pos, other.pos]),
                       np.concatenate([self.log_scale, other.log_scale]),
                       np.concatenate([self.quat, other.quat]),
                       np.concatenate([self.opacity, other.opacity]),
                       np.concatenate([self.sh, other.sh]),
                       np.concatenate([self.intensity, other.intensity]),
                       np.concatenate([ids(self), ids(other)]).astype(np.int32), rd)


@dataclasses.dataclass
class Pinhole:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    world_to_sensor: np.ndarray  # [4,4] float64
    near: float = 0.2
    kind: str = "pinhole"


@dataclasses.dataclass
class Cylindrical:
    """Cylindrical (fisheye) camera: column x looks along azimuth
    (x + 0.5 - cx) / fx about the camera's y axis, row y along height
    (y + 0.5 - cy) / fy on the unit cylinder (camera frame as the pinhole)."""
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    world_to_sensor: np.ndarray  # [4,4] float64
    near: float = 0.2
    kind: str = "cylindrical"


@dataclasses.dataclass
class Lidar:
    beams: int
    columns: int
    el_min_deg: float
    el_max_deg: float
    world_to_sensor: np.ndarray
    az0_deg: float = -180.0
    near: float = 0.2
    kind: str = "lidar"

    @property
    def width(self) -> int:
        return self.columns

    @property
    def height(self) -> int:
        return self.beams


def rgb_to_sh0(rgb: np.ndarray, dtype=np.float32) -> np.ndarray:
    """Degree-0 SH coefficients [N,1,3] that render as the colour `rgb`."""
    return ((np.asarray(rgb, np.float64) - 0.5) / _Y00).astype(dtype)[:, None, :]


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _quat_from_frame(tu, tv, n):
    """Quaternion (w,x,y,z) of the rotation with columns tu, tv, n (rows: surfels)."""
    R = np.stack([tu, tv, n], axis=2)  # [N,3,3], columns
    m00, m11, m22 = R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]
    w = np.sqrt(np.maximum(0.0, 1 + m00 + m11 + m22)) / 2
    x = np.sqrt(np.maximum(0.0, 1 + m00 - m11 - m22)) / 2
    y = np.sqrt(np.maximum(0.0, 1 - m00 + m11 - m22)) / 2
    z = np.sqrt(np.maximum(0.0, 1 - m00 - m11 + m22)) / 2
    x = np.copysign(x, R[:, 2, 1] - R[:, 1, 2])
    y = np.copysign(y, R[:, 0, 2] - R[:, 2, 0])
    z = np.copysign(z, R[:, 1, 0] - R[:, 0, 1])
    q = np.stack([w, x, y, z], axis=1)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _plane_quats(rng, normal, n):
    """Random in-plane rotation of surfels whose normal is `normal` (3,)."""
    normal = np.asarray(normal, np.float64)
    helper = np.array([1.0, 0, 0]) if abs(normal[0]) < 0.9 else np.array([0, 1.0, 0])
    e1 = np.cross(normal, helper)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(normal, e1)
    th = rng.uniform(0, 2 * np.pi, n)
    tu = np.cos(th)[:, None] * e1 + np.sin(th)[:, None] * e2
    nn = np.broadcast_to(normal, (n, 3))
    tv = np.cross(nn, tu)
    return _quat_from_frame(tu, tv, nn)


# ---------------------------------------------------------------------------
# Sensors
# ---------------------------------------------------------------------------
def camera_pose(position, yaw_deg=0.0, pitch_deg=0.0, f32=True) -> np.ndarray:
    """world->camera for a camera at `position` looking along yaw (from +x
    towards +y); rounded to float32 values unless f32=False."""
    yaw, pitch = math.radians(yaw_deg), math.radians(pitch_deg)
    f = np.array([math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch), math.sin(pitch)])
    up = np.array([0.0, 0.0, 1.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])  # rows: camera axes in world
    M = np.eye(4)
    M[:3, :3] = R
    M[:3, 3] = -R @ np.asarray(position, np.float64)
    return _f32(M) if f32 else M


def _f32(a):
    """Round to float32-representable values: the C ABI carries poses in
    float32, so every consumer sees exactly the same numbers."""
    return np.asarray(a, np.float32).astype(np.float64)


def lidar_pose(position, yaw_deg=0.0, f32=True) -> np.ndarray:
    yaw = math.radians(yaw_deg)
    R = np.array([[math.cos(yaw), math.sin(yaw), 0.0],
                  [-math.sin(yaw), math.cos(yaw), 0.0],
                  [0.0, 0.0, 1.0]])
    M = np.eye(4)
    M[:3, :3] = R
    M[:3, 3] = -R @ np.asarray(position, np.float64)
    return _f32(M) if f32 else M


def pinhole(width, height, f, position=(0, 0, 0), yaw_deg=0.0, pitch_deg=0.0, pose=None, near=0.2):
    return Pinhole(width, height, float(f), float(f), width / 2.0, height / 2.0,
                   camera_pose(position, yaw_deg, pitch_deg) if pose is None else np.asarray(pose, np.float64),
                   near)


def cylindrical(width, height, hfov_deg, vfov_deg, position=(0, 0, 0), yaw_deg=0.0, pitch_deg=0.0, pose=None,
                near=0.2):
    """Cylindrical camera with horizontal field hfov (degrees, may exceed 180)
    and vertical field vfov at the image centre; `pose` (world->camera)
    overrides position / yaw / pitch."""
    fx = width / math.radians(hfov_deg)
    fy = 0.5 * height / math.tan(math.radians(0.5 * vfov_deg))
    M = np.asarray(pose, np.float64) if pose is not None else camera_pose(position, yaw_deg, pitch_deg)
    return Cylindrical(width, height, fx, fy, width / 2.0, height / 2.0, M, near)


def spinning_lidar(beams, columns, el_min, el_max, position=(0, 0, 0), yaw_deg=0.0, near=0.2):
    return Lidar(beams, columns, float(el_min), float(el_max), lidar_pose(position, yaw_deg), -180.0, near)


# ---------------------------------------------------------------------------
# Scenes
# ---------------------------------------------------------------------------
def plain_scene(n=8000, seed=SEED_BASE + 0):
    """Object-space test scene: centres in [-10,10]x[-3,3]x[5,40] in front of a
    camera at the origin looking +z, log-scales U[-3,0], uniform unit quats,
    opacity logit N(0,1), colour U[0,1] stored as SH degree 0."""
    rng = np.random.default_rng(seed)
    pos = np.stack([rng.uniform(-10, 10, n), rng.uniform(-3, 3, n), rng.uniform(5, 40, n)], 1).astype(np.float32)
    log_scale = rng.uniform(-3, 0, (n, 2)).astype(np.float32)
    quat = _unit_quats(rng, n)
    opacity = rng.standard_normal(n).astype(np.float32)
    rgb = rng.uniform(0, 1, (n, 3))
    intensity = rng.uniform(0, 1, n).astype(np.float32)
    return Surfels(pos, log_scale, quat, opacity, rgb_to_sh0(rgb), intensity)


def plain_camera(width=256, height=160, f=200.0):
    return Pinhole(width, height, f, f, width / 2.0, height / 2.0, np.eye(4), 0.2)


def driving_scene(n=1_500_000, seed=SEED_BASE + 1, sh_degree=3, x_range=(-60.0, 120.0), n_boxes=40):
    """Road + roadside boxes.  60% of surfels on the road plane (x in x_range,
    |y| <= 8, z ~ N(0, 0.05), normal up, random in-plane angle); 40% on the
    faces of `n_boxes` boxes with |y| in [8,15], z in [0,6].  Log-scales
    U[-3,0]; SH coefficients N(0, 0.2); opacity logit N(0,1); intensity U[0,1]."""
    rng = np.random.default_rng(seed)
    n_road = int(round(0.6 * n))
    n_box = n - n_road
    pos = np.empty((n, 3), np.float32)
    quat = np.empty((n, 4), np.float32)
    pos[:n_road, 0] = rng.uniform(x_range[0], x_range[1], n_road)
    pos[:n_road, 1] = rng.uniform(-8, 8, n_road)
    pos[:n_road, 2] = rng.normal(0, 0.05, n_road)
    quat[:n_road] = _plane_quats(rng, (0, 0, 1), n_road)

    # boxes: centre x, side, extent; surfels on the faces proportional to area
    bx = rng.uniform(x_range[0], x_range[1], n_boxes)
    side = np.where(rng.uniform(size=n_boxes) < 0.5, -1.0, 1.0)
    dy = rng.uniform(2, 7, n_boxes)      # box depth across the road, inside |y| in [8,15]
    y_lo = np.where(side > 0, 8.0, -8.0 - dy)
    lx = rng.uniform(4, 12, n_boxes)
    hz = rng.uniform(2, 6, n_boxes)
    faces = []  # (box, normal, origin, e1, e2, extent1, extent2)
    for b in range(n_boxes):
        x0, x1 = bx[b] - lx[b] / 2, bx[b] + lx[b] / 2
        ya, yb = y_lo[b], y_lo[b] + dy[b]
        h = hz[b]
        faces += [
            ((-1, 0, 0), (x0, ya, 0), (0, 1, 0), (0, 0, 1), dy[b], h),
            ((1, 0, 0), (x1, ya, 0), (0, 1, 0), (0, 0, 1), dy[b], h),
            ((0, -1, 0), (x0, ya, 0), (1, 0, 0), (0, 0, 1), lx[b], h),
            ((0, 1, 0), (x0, yb, 0), (1, 0, 0), (0, 0, 1), lx[b], h),
            ((0, 0, 1), (x0, ya, h), (1, 0, 0), (0, 1, 0), lx[b], dy[b]),
        ]
    areas = np.array([f[4] * f[5] for f in faces])
    face_of = rng.choice(len(faces), size=n_box, p=areas / areas.sum())
    counts = np.bincount(face_of, minlength=len(faces))
    k = n_road
    for fi, cnt in enumerate(counts):
        if cnt == 0:
            continue
        nrm, org, e1, e2, a1, a2 = faces[fi]
        s1 = rng.uniform(0, a1, cnt)[:, None]
        s2 = rng.uniform(0, a2, cnt)[:, None]
        pos[k:k + cnt] = np.asarray(org) + s1 * np.asarray(e1) + s2 * np.asarray(e2)
        quat[k:k + cnt] = _plane_quats(rng, nrm, cnt)
        k += cnt
    K = (sh_degree + 1) ** 2
    log_scale = rng.uniform(-3, 0, (n, 2)).astype(np.float32)
    opacity = rng.standard_normal(n).astype(np.float32)
    sh = rng.normal(0, 0.2, (n, K, 3)).astype(np.float32)
    intensity = rng.uniform(0, 1, n).astype(np.float32)
    return Surfels(pos, log_scale, quat, opacity, sh, intensity)


def driving_camera(width=1920, height=1080, f=1000.0, position=(0.0, 0.0, 1.5), yaw_deg=0.0):
    return pinhole(width, height, f, position, yaw_deg)


def driving_lidar(beams=128, columns=1800, el_min=-25.0, el_max=15.0, position=(0.0, 0.0, 1.8)):
    return spinning_lidar(beams, columns, el_min, el_max, position)


def perturbed(s: Surfels, seed, pos_sigma=0.05, scale_sigma=0.1, sh_sigma=0.05, opacity_sigma=0.2) -> Surfels:
    """A seeded perturbed copy (the target scene of a reconstruction step)."""
    rng = np.random.default_rng(seed)
    return Surfels(
        (s.pos + rng.normal(0, pos_sigma, s.pos.shape)).astype(np.float32),
        (s.log_scale + rng.normal(0, scale_sigma, s.log_scale.shape)).astype(np.float32),
        (s.quat + rng.normal(0, 0.05, s.quat.shape)).astype(np.float32),
        (s.opacity + rng.normal(0, opacity_sigma, s.opacity.shape)).astype(np.float32),
        (s.sh + rng.normal(0, sh_sigma, s.sh.shape)).astype(np.float32),
        s.intensity.copy(), None if s.obj_id is None else s.obj_id.copy())


# ---------------------------------------------------------------------------
# Inserted objects and the surround rig
# ---------------------------------------------------------------------------
def object_asset(n=50_000, seed=SEED_BASE + 5, size=(4.5, 1.8, 1.5), sh_degree=3):
    """A car-sized box of surfels in its own frame (origin on the ground,
    centred), faces sampled by area, SH N(0,0.2), opacity logit N(1,1)."""
    rng = np.random.default_rng(seed)
    L, Wd, Ht = size
    faces = [
        ((-1, 0, 0), (-L / 2, -Wd / 2, 0), (0, 1, 0), (0, 0, 1), Wd, Ht),
        ((1, 0, 0), (L / 2, -Wd / 2, 0), (0, 1, 0), (0, 0, 1), Wd, Ht),
        ((0, -1, 0), (-L / 2, -Wd / 2, 0), (1, 0, 0), (0, 0, 1), L, Ht),
        ((0, 1, 0), (-L / 2, Wd / 2, 0), (1, 0, 0), (0, 0, 1), L, Ht),
        ((0, 0, 1), (-L / 2, -Wd / 2, Ht), (1, 0, 0), (0, 1, 0), L, Wd),
    ]
    areas = np.array([f[4] * f[5] for f in faces])
    face_of = rng.choice(len(faces), size=n, p=areas / areas.sum())
    pos = np.empty((n, 3), np.float32)
    quat = np.empty((n, 4), np.float32)
    k = 0
    for fi, cnt in enumerate(np.bincount(face_of, minlength=len(faces))):
        nrm, org, e1, e2, a1, a2 = faces[fi]
        s1 = rng.uniform(0, a1, cnt)[:, None]
        s2 = rng.uniform(0, a2, cnt)[:, None]
        pos[k:k + cnt] = np.asarray(org) + s1 * np.asarray(e1) + s2 * np.asarray(e2)
        quat[k:k + cnt] = _plane_quats(rng, nrm, cnt)
        k += cnt
    K = (sh_degree + 1) ** 2
    return Surfels(pos,
                   rng.uniform(-4, -1.5, (n, 2)).astype(np.float32),
                   quat,
                   rng.normal(1.0, 1.0, n).astype(np.float32),
                   rng.normal(0, 0.2, (n, K, 3)).astype(np.float32),
                   rng.uniform(0, 1, n).astype(np.float32))


def object_poses(n_obj, seed, x_range=(-40.0, 80.0)):
    """Rigid poses [n_obj,3,4] (R|t) uniform on the road with a random yaw."""
    rng = np.random.default_rng(seed)
    P = np.zeros((n_obj, 3, 4), np.float64)
    for k in range(n_obj):
        yaw = rng.uniform(-np.pi, np.pi)
        c, s = math.cos(yaw), math.sin(yaw)
        P[k, :3, :3] = [[c, -s, 0], [s, c, 0], [0, 0, 1]]
        P[k, :, 3] = [rng.uniform(*x_range), rng.uniform(-6.5, 6.5), 0.0]
    return _f32(P)


def surround_rig(x=0.0, y=0.0, yaw_deg=0.0):
    """2 cameras 1920x1080 (front/back, f=1000), 4 cameras 1280x720 at yaw
    +-60 and +-120 deg (f=640), a 128x1800 LiDAR (el -25..15 deg) and a
    32x1024 LiDAR (el -30..10 deg), on a vehicle at (x, y) on the road facing
    yaw_deg (the origin facing +x by default)."""
    c, s = math.cos(math.radians(yaw_deg)), math.sin(math.radians(yaw_deg))
    at = lambda px, py, pz: (x + c * px - s * py, y + s * px + c * py, pz)
    cams = [pinhole(1920, 1080, 1000.0, at(1.5, 0, 1.5), yaw_deg + 0.0),
            pinhole(1920, 1080, 1000.0, at(-1.5, 0, 1.5), yaw_deg + 180.0)]
    for yaw in (60.0, -60.0, 120.0, -120.0):
        cams.append(pinhole(1280, 720, 640.0, at(0.0, 0.0, 1.6), yaw_deg + yaw))
    lidars = [spinning_lidar(128, 1800, -25.0, 15.0, at(0.0, 0.0, 1.8), yaw_deg),
              spinning_lidar(32, 1024, -30.0, 10.0, at(0.5, 0.0, 1.9), yaw_deg)]
    return cams + lidars


# ---------------------------------------------------------------------------
# Anchor scene (neural Gaussians: anchor feature -> MLP -> k offset surfels)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Anchors:
    pos: np.ndarray        # [A,3] float32
    feature: np.ndarray    # [A,32] float32
    scale: np.ndarray      # [A] float32 (l_a, offset length scale)
    offsets: np.ndarray    # [A,k,3] float32
    intensity: np.ndarray  # [A,k] float32

    @property
    def n(self):
        return int(self.pos.shape[0])

    @property
    def k(self):
        return int(self.offsets.shape[1])


def anchors_from_surfels(s: Surfels, k=10, seed=SEED_BASE + 2, feat_dim=32):
    """Group Morton-adjacent surfels in runs of k: anchor = group mean, offsets
    = member - anchor (l_a = 1), feature ~ N(0,1).  Returns the anchors and the
    permutation that puts the explicit surfels in anchor order."""
    rng = np.random.default_rng(seed)
    n = (s.n // k) * k
    p = s.pos[:n].astype(np.float64)
    lo, hi = p.min(0), p.max(0)
    q = ((p - lo) / np.maximum(hi - lo, 1e-9) * 1023).astype(np.uint64)

    def spread(v):
        v = v & np.uint64(0x3FF)
        v = (v | (v << np.uint64(16))) & np.uint64(0x30000FF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x300F00F)
        v = (v | (v << np.uint64(4))) & np.uint64(0x30C30C3)
        v = (v | (v << np.uint64(2))) & np.uint64(0x9249249)
        return v
    code = spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1)) | (spread(q[:, 2]) << np.uint64(2))
    order = np.argsort(code, kind="stable")
    grp = s.pos[order].reshape(-1, k, 3).astype(np.float64)
    apos = grp.mean(1)
    offs = grp - apos[:, None, :]
    A = grp.shape[0]
    return Anchors(apos.astype(np.float32),
                   rng.standard_normal((A, feat_dim)).astype(np.float32),
                   np.ones(A, np.float32),
                   offs.astype(np.float32),
                   s.intensity[order].reshape(A, k).astype(np.float32)), order


def road_poses(n_poses, seed, x_range=(-40.0, 80.0), yaw_deg=10.0, height=1.5):
    """Seeded camera positions/yaws along the road."""
    rng = np.random.default_rng(seed)
    xs = rng.uniform(*x_range, n_poses)
    yaws = rng.uniform(-yaw_deg, yaw_deg, n_poses)
    return [(float(x), float(yw)) for x, yw in zip(xs, yaws)]


def init_mlp(seed, feat_dim=32, hidden=64, k=10):
    """Seeded anchor-MLP weights W1 [feat_dim+4, hidden], b1, W2 [hidden, 10 k],
    b2 (float32).  Uniform He-style weights; biases start every offset at
    opacity logit 0, grey colour, log-scale -2 and the identity rotation."""
    rng = np.random.default_rng(seed)
    n_in = feat_dim + 4
    W1 = rng.uniform(-1, 1, (n_in, hidden)) * math.sqrt(6.0 / n_in) * 0.5
    b1 = np.zeros(hidden)
    W2 = rng.uniform(-1, 1, (hidden, 10 * k)) * math.sqrt(6.0 / hidden) * 0.1
    b2 = np.tile(np.array([0.0, 0.0, 0.0, 0.0, -2.0, -2.0, 1.0, 0.0, 0.0, 0.0]), k)
    return W1.astype(np.float32), b1.astype(np.float32), W2.astype(np.float32), b2.astype(np.float32)


def init_lidar_mlp(seed, feat_dim=32, hidden=64, k=10):
    """Seeded weights of the LiDAR scene's anchor MLP (the LiDAR head reads
    an offset's 10 outputs as opacity, intensity, ray-drop logit, unused,
    log-scales, quaternion): as init_mlp, with every offset starting at
    intensity 0.5 and ray-drop probability sigmoid(-1)."""
    W1, b1, W2, b2 = init_mlp(seed, feat_dim, hidden, k)
    b2 = b2.copy()
    b2[2::10] = -1.0
    return W1, b1, W2, b2
