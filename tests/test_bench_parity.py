"""The benchmark's every-ray parity accounting (CPU): flagged rays are
excluded and counted, each output's error is taken beyond its slack, depth
and range are relative and checked only where alpha >= 0.01, and a ray
beyond tolerance + slack is counted."""
import sys
import types
from pathlib import Path

import numpy as np

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))
import bench  # noqa: E402

H, W = 2, 4


def _sensor(kind):
    return types.SimpleNamespace(kind=kind, width=W, height=H)


def _oracle_lidar():
    z = np.zeros((H, W))
    return {"range": np.full((H, W), 20.0), "intensity": np.full((H, W), 0.5), "alpha": np.full((H, W), 0.9),
            "flip": z.copy(), "slack": z.copy(), "slack_n": z.copy(), "slack_z": z.copy(), "slack_c": z.copy()}


def _gpu_lidar(o):
    return {k: o[k].astype(np.float32).copy() for k in ("range", "intensity", "alpha")}


def test_identical_outputs_are_within():
    o = _oracle_lidar()
    rep = bench.frame_parity([_sensor("lidar")], [_gpu_lidar(o)], [o])[0]
    assert rep["rays_over_tolerance"] == 0 and rep["flagged_frac"] == 0.0
    assert max(rep["max_err_beyond_slack"].values()) <= 1e-6


def test_a_ray_beyond_tolerance_is_counted_unless_flagged_or_covered_by_slack():
    o = _oracle_lidar()
    g = _gpu_lidar(o)
    g["intensity"][1, 2] += 2e-4
    rep = bench.frame_parity([_sensor("lidar")], [g], [o])[0]
    assert rep["rays_over_tolerance"] == 1
    assert abs(rep["max_err_beyond_slack"]["intensity"] - 2e-4) < 1e-6
    # its reordering slack covers it
    o2 = _oracle_lidar()
    o2["slack"][1, 2] = 1.5e-4
    rep = bench.frame_parity([_sensor("lidar")], [g], [o2])[0]
    assert rep["rays_over_tolerance"] == 0
    assert rep["tied_frac"] == 1.0 / (H * W)
    # a flippable threshold on that ray excludes it, and it is counted as flagged
    o3 = _oracle_lidar()
    o3["flip"][1, 2] = 1e-3
    rep = bench.frame_parity([_sensor("lidar")], [g], [o3])[0]
    assert rep["rays_over_tolerance"] == 0
    assert rep["flagged_frac"] == 1.0 / (H * W)


def test_range_is_relative_and_checked_only_where_alpha_counts():
    o = _oracle_lidar()
    g = _gpu_lidar(o)
    g["range"][0, 0] = 20.0 * (1 + 5e-5)   # within 1e-4 relative
    g["range"][0, 1] = 20.0 * (1 + 3e-4)   # beyond
    rep = bench.frame_parity([_sensor("lidar")], [g], [o])[0]
    assert rep["rays_over_tolerance"] == 1
    o["alpha"][0, 1] = 0.005               # a beam that barely returns: its range is not checked
    g = _gpu_lidar(o)
    g["range"][0, 1] = 20.0 * (1 + 3e-4)
    rep = bench.frame_parity([_sensor("lidar")], [g], [o])[0]
    assert rep["rays_over_tolerance"] == 0


def test_camera_planes_against_pixel_major_oracle():
    rng = np.random.default_rng(1)
    z = np.zeros((H, W))
    o = {"rgb": rng.uniform(0, 1, (H, W, 3)), "normal": rng.uniform(-1, 1, (H, W, 3)),
         "depth": rng.uniform(5, 50, (H, W)), "alpha": np.full((H, W), 0.95),
         "flip": z.copy(), "slack": z.copy(), "slack_n": z.copy(), "slack_z": z.copy(), "slack_c": z.copy()}
    g = {"rgb": np.moveaxis(o["rgb"], -1, 0).astype(np.float32).copy(),
         "normal": np.moveaxis(o["normal"], -1, 0).astype(np.float32).copy(),
         "depth": o["depth"].astype(np.float32), "alpha": o["alpha"].astype(np.float32)}
    rep = bench.frame_parity([_sensor("pinhole")], [g], [o])[0]
    assert rep["rays_over_tolerance"] == 0
    g["normal"][2, 1, 3] += 3e-4            # one channel of one pixel's normal
    rep = bench.frame_parity([_sensor("pinhole")], [g], [o])[0]
    assert rep["rays_over_tolerance"] == 1
    o["slack_n"][1, 3] = 3e-4               # the normal's own reordering slack covers it
    rep = bench.frame_parity([_sensor("pinhole")], [g], [o])[0]
    assert rep["rays_over_tolerance"] == 0


def test_slack_of_every_output_covers_alpha_and_relative_depth():
    """slack_c bounds the change of every output (the conditioning of Eq. 2,
    and hits past the stop that FP32 may composite first): alpha and the
    colour / intensity get it absolutely, the range relatively over alpha."""
    o = _oracle_lidar()
    g = _gpu_lidar(o)
    g["alpha"][0, 2] += 3e-4
    g["intensity"][0, 2] += 3e-4
    g["range"][0, 2] = 20.0 * (1 + 4e-4)
    rep = bench.frame_parity([_sensor("lidar")], [g], [o])[0]
    assert rep["rays_over_tolerance"] == 1
    o2 = _oracle_lidar()
    o2["slack_c"][0, 2] = 3e-4      # range: 4e-4 relative <= 1e-4 + 3e-4 / 0.9
    rep = bench.frame_parity([_sensor("lidar")], [g], [o2])[0]
    assert rep["rays_over_tolerance"] == 0 and rep["flagged_frac"] == 0.0
    assert rep["cond_slack_over_tol_frac"] == 1.0 / (H * W)
