"""The benchmarked surround-rig frame against the oracle.

The frame is the benchmark's configuration: 6 pinhole cameras (2 x 1920x1080,
4 x 1280x720) and 2 spinning LiDARs (128x1800, 32x1024); 300k anchors x 10
offsets decoded by the anchor MLP (trained on the GPU on the explicit
background's frames, as the benchmark does) into 3M surfels plus 20 rigidly
posed 50k-surfel SH-3 objects; the tiling, staging depth and list splits
chosen by gsr_autotune, rendered by the persistent whole-rig launch.

Nothing the GPU computed enters the oracle.  The oracle decodes the trained
anchors in FP64 itself (Sec. III-A, anchors decoded by an MLP), and the check
has two parts:
* the decode: the GPU's FP32 decode of every anchor against the oracle's,
  parameter by parameter;
* the render at identical inputs: the oracle's decoded table rounded to
  FP32 is rendered by the GPU with the benchmark's tuned plan (the same
  kernels, tiles and list splits as the decoded frame) and by the oracle
  (tiled mode, bit-identical to brute force), 4,096 sampled rays per sensor.
A render fed the GPU's own FP32 decode differs from the oracle's FP64 decode
by the decode's rounding carried through Eq. 2, which no bound for
identical inputs covers: the benchmark's every-ray block reports those rays.
"""
import numpy as np
import pytest
import torch

from oracle import render as OR
from parity import check_camera, check_lidar

pytestmark = pytest.mark.gpu

SAMPLES = 4096
# flagged-fraction caps per sensor: the measured fractions (every ray of
# trained networks' frames: 0.8, 2.3, 0.5-0.6 % on the cameras, 1.2-1.4 and
# 2.6-3.0 % on the LiDARs) with a margin; the back camera sees the boxes'
# coplanar faces head on, where runs of near-tied centre depths end rays;
# the 32-beam LiDAR's coarse cells leave many surfels to the low-pass
# fallback, whose thresholds FP32 can move by the centre's reach in cells
CAPS = [0.015, 0.035, 0.01, 0.01, 0.01, 0.01, 0.025, 0.04]


def test_configured_rig_frame_matches_oracle(gpu_lib):
    import bench
    from paper_2503_11731_gb300 import gsr
    from paper_2503_11731_gb300.frame import DeviceSurfels
    from paper_2503_11731_gb300.neural import NeuralFrame
    from paper_2503_11731_gb300 import synth
    bg, objs, poses, sensors = bench.rig_parts()
    anchors, mlp = bench.rig_neural(bg)
    origin = bench.rig_origin(sensors)
    model, da, _ = bench.rig_distillation(bg, anchors, mlp)
    del bg
    # the trained parameters as the oracle receives them
    anchors = synth.Anchors(anchors.pos, da.feature.cpu().numpy(), anchors.scale, anchors.offsets, anchors.intensity)
    mlp = tuple(getattr(model, k).cpu().numpy() for k in ("w1", "b1", "w2", "b2"))
    n_bg = anchors.n * anchors.k
    n = n_bg + objs.n
    # the benchmark's outputs: no final T (a frame that requests none skips
    # keeping the per-chunk states of split lists)
    r = bench.rig_renderer(n, sensors, outputs=("rgb", "depth", "normal", "alpha", "n_contrib", "n_walk"))
    pose_t = torch.as_tensor(poses.reshape(-1, 12).astype(np.float32), device="cuda")
    d_obj = DeviceSurfels.from_host(objs)
    nf = NeuralFrame(model, da, r, d_obj, pose_t, origin, gsr.DECODE_F32)
    nf.render()
    torch.cuda.synchronize()
    tuned = r.autotune([nf.table, d_obj], pose_t, warmup=1, reps=2)
    nf.render()
    torch.cuda.synchronize()
    st, nvis, npairs = r.status()
    assert st == 0, st
    print("tiling", tuned["camera_tile"], tuned["lidar_tile"], tuned["split"], tuned["lidar_split"],
          "pairs", npairs)
    scene, _, dec = bench.oracle_rig_scene(objs, anchors, mlp, origin, decoded=True)

    # 1. the decode: the GPU's FP32 table against the oracle's FP64 decode
    for k in bench.DECODED:
        got = getattr(nf.table, k).cpu().numpy()
        ref = dec[k].detach().numpy().reshape(got.shape)
        err = np.abs(got - ref).max()
        print("decode", k, "max error", err)
        assert err <= 1e-5 * max(1.0, np.abs(ref).max()), k
    del dec

    # 2. the render at identical inputs, with the tuned plan
    scene = bench.round32(scene)
    back = synth.Surfels(scene.pos[:n_bg], scene.log_scale[:n_bg], scene.quat[:n_bg], scene.opacity[:n_bg],
                         np.ascontiguousarray(scene.sh[:n_bg, :1]), scene.intensity[:n_bg])
    assert not np.any(scene.sh[:n_bg, 1:])
    d_back = DeviceSurfels.from_host(back)
    del back
    r.preprocess(d_back, pose_t, first=0)
    r.preprocess(d_obj, pose_t, first=n_bg)
    r.bin_sort()
    r.composite_rig()
    out = r.out
    torch.cuda.synchronize()
    st, nvis, npairs = r.status()
    assert st == 0, st
    # the tuned plan splits long lists (the path the benchmark times)
    info = r.region(8, torch.int32).view(-1, 4)
    assert int((info[:, 0] > 0).sum()) > 0
    g = [{k: v.cpu().numpy() for k, v in o.items()} for o in out]
    rng = np.random.default_rng(2503)
    for i, (s, gg) in enumerate(zip(sensors, g)):
        idx = rng.choice(s.width * s.height, SAMPLES, replace=False)
        name = f"rig frame sensor {i} ({s.kind} {s.width}x{s.height})"
        if s.kind == "lidar":
            o = OR.render_lidar(scene, s, rays=idx, obj_pose=poses, tile=8)
            check_lidar(gg, o, rays=idx, max_flag=CAPS[i], name=name)
        else:
            o = OR.render_pinhole(scene, s, pixels=idx, obj_pose=poses, tile=16)
            check_camera(gg, o, pix=idx, max_flag=CAPS[i], name=name)
