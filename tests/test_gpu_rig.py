"""GPU tests of the batched rig path: the persistent whole-rig compositing
launch (gsr_render_rig), the captured frame graph, mixed per-sensor tile
shapes, and rigidly posed inserted objects -- against the per-sensor calls
(bit-exact) and against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import render as OR
from paper_2503_11731_gb300 import synth
from parity import check_camera, check_lidar

# flagged-fraction caps: the measured fractions (of 400-600 sampled rays,
# so one ray is 0.17-0.25 %) with a margin
CAP = {"camera": 0.02, "lidar": 0.015}

pytestmark = pytest.mark.gpu


def _small_rig():
    bg = synth.driving_scene(n=60_000, seed=71, x_range=(-25.0, 40.0), n_boxes=8)
    poses = synth.object_poses(3, seed=72, x_range=(-10.0, 20.0))
    objs = None
    for k in range(3):
        a = synth.object_asset(4000, seed=73 + k)
        a.obj_id = np.full(a.n, k, np.int32)
        objs = a if objs is None else objs.concat(a)
    scene = bg.concat(objs)
    sensors = [synth.pinhole(320, 180, 170.0, (1.5, 0, 1.5), 0.0),
               synth.pinhole(256, 144, 120.0, (0.0, 0.0, 1.6), 60.0),
               synth.spinning_lidar(32, 360, -25.0, 15.0, (0.0, 0.0, 1.8)),
               synth.spinning_lidar(16, 256, -30.0, 10.0, (0.5, 0.0, 1.9)),
               synth.cylindrical(480, 120, 200.0, 60.0, (0.0, 0.0, 1.7), yaw_deg=180.0)]
    return scene, poses, sensors


def _renderer(scene, sensors, tiles):
    from paper_2503_11731_gb300.frame import Renderer
    return Renderer(scene.n, sensors, tiles=tiles,
                    outputs=("rgb", "depth", "normal", "alpha", "trans", "n_contrib", "n_walk"))


TILES = [(16, 16), (32, 8), (8, 8), (16, 4), (16, 8)]


def test_rig_launch_equals_per_sensor_calls(gpu_lib):
    from paper_2503_11731_gb300.frame import DeviceSurfels
    scene, poses, sensors = _small_rig()
    d = DeviceSurfels.from_host(scene)
    P = torch.as_tensor(poses.reshape(-1, 12).astype(np.float32), device="cuda")
    r = _renderer(scene, sensors, TILES)
    a = [{k: v.clone() for k, v in o.items()} for o in r.render(d, P)]
    b = r.render_rig(d, P)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    for i, (oa, ob) in enumerate(zip(a, b)):
        for k in oa:
            assert torch.equal(oa[k], ob[k]), (i, k)


def test_rig_matches_oracle_with_posed_objects(gpu_lib):
    from paper_2503_11731_gb300.frame import DeviceSurfels
    scene, poses, sensors = _small_rig()
    d = DeviceSurfels.from_host(scene)
    P = torch.as_tensor(poses.reshape(-1, 12).astype(np.float32), device="cuda")
    r = _renderer(scene, sensors, TILES)
    out = [{k: v.cpu().numpy() for k, v in o.items()} for o in r.render_rig(d, P)]
    rng = np.random.default_rng(5)
    for s, g in zip(sensors, out):
        idx = rng.choice(s.width * s.height, 600, replace=False)
        if s.kind == "lidar":
            check_lidar(g, OR.render_lidar(scene, s, rays=idx, obj_pose=poses), rays=idx, max_flag=CAP[s.kind if s.kind == "lidar" else "camera"])
        else:
            check_camera(g, OR.render_pinhole(scene, s, pixels=idx, obj_pose=poses), pix=idx, max_flag=CAP[s.kind if s.kind == "lidar" else "camera"])
    # the objects are visible somewhere (the test exercises the pose path)
    assert (scene.obj_id >= 0).sum() > 0


def test_frame_graph_replays_and_follows_in_place_updates(gpu_lib):
    from paper_2503_11731_gb300.frame import DeviceSurfels
    scene, poses, sensors = _small_rig()
    d = DeviceSurfels.from_host(scene)
    P = torch.as_tensor(poses.reshape(-1, 12).astype(np.float32), device="cuda")
    r = _renderer(scene, sensors, TILES)
    ref = [{k: v.clone() for k, v in o.items()} for o in r.render_rig(d, P)]
    g = r.graph(d, P, stages=7)
    for o in r.out:
        for v in o.values():
            v.zero_()
    stream = torch.cuda.current_stream()
    import ctypes
    h = ctypes.c_void_p(stream.cuda_stream)
    g.launch(h)
    g.launch(h)
    torch.cuda.synchronize()
    for i, (oa, ob) in enumerate(zip(ref, r.out)):
        for k in oa:
            assert torch.equal(oa[k], ob[k]), (i, k)
    # move the objects in place: the replayed graph renders the new poses
    P[:, 3] += 2.0
    ref2 = [{k: v.clone() for k, v in o.items()} for o in r.render_rig(d, P)]
    for o in r.out:
        for v in o.values():
            v.zero_()
    g.launch(h)
    torch.cuda.synchronize()
    assert not torch.equal(ref2[0]["rgb"], ref[0]["rgb"])
    for i, (oa, ob) in enumerate(zip(ref2, r.out)):
        for k in oa:
            assert torch.equal(oa[k], ob[k]), (i, k)
    g.close()


def test_preprocess_parts_mix_sh_degrees(gpu_lib):
    """A plan fed by two tables (SH-0 background, SH-3 posed objects) through
    gsr_preprocess_part renders exactly like one table with the background's
    SH padded by zero coefficients, and matches the oracle."""
    from paper_2503_11731_gb300.frame import DeviceSurfels
    bg = synth.driving_scene(n=30_000, seed=91, x_range=(-20.0, 30.0), n_boxes=4, sh_degree=0)
    poses = synth.object_poses(2, seed=92, x_range=(-5.0, 15.0))
    objs = synth.object_asset(3000, seed=93)
    objs.obj_id = np.arange(objs.n, dtype=np.int32) % 2
    pad = np.zeros((bg.n, 16, 3), np.float32)
    pad[:, :1] = bg.sh
    bg3 = synth.Surfels(bg.pos, bg.log_scale, bg.quat, bg.opacity, pad, bg.intensity)
    whole = bg3.concat(objs)
    sensors = [synth.pinhole(320, 180, 170.0, (1.5, 0, 1.5), 0.0),
               synth.spinning_lidar(32, 360, -25.0, 15.0, (0.0, 0.0, 1.8))]
    P = torch.as_tensor(poses.reshape(-1, 12).astype(np.float32), device="cuda")
    r = _renderer(whole, sensors, [(16, 16), (8, 8)])
    ref = [{k: v.clone() for k, v in o.items()} for o in r.render_rig(DeviceSurfels.from_host(whole), P)]
    for o in r.out:
        for v in o.values():
            v.zero_()
    d_obj, d_bg = DeviceSurfels.from_host(objs), DeviceSurfels.from_host(bg)
    r.preprocess(d_obj, P, first=bg.n)   # parts in any order; first == 0 clears the status word
    r.preprocess(d_bg, P, first=0)
    r.bin_sort()
    r.composite_rig()
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    for i, (oa, ob) in enumerate(zip(ref, r.out)):
        for k in oa:
            assert torch.equal(oa[k], ob[k]), (i, k)
    s = sensors[0]
    idx = np.random.default_rng(9).choice(s.width * s.height, 500, replace=False)
    o = OR.render_pinhole(whole, s, pixels=idx, obj_pose=poses)
    yy, xx = np.divmod(idx, s.width)
    check_camera({k: v.cpu().numpy() for k, v in r.out[0].items()}, o, pix=idx, max_flag=CAP[s.kind if s.kind == "lidar" else "camera"])
    assert (r.out[0]["n_contrib"].cpu().numpy()[yy, xx] > 0).mean() > 0.5


def test_batch_depth_and_tile_shape_change_speed_only(gpu_lib):
    """The staged batch depth never changes a result (bit-exact); another
    tile shape changes only list lengths, so results agree to rounding of
    the split-tile merge (none where no list is split)."""
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer
    scene, poses, sensors = _small_rig()
    d = DeviceSurfels.from_host(scene)
    P = torch.as_tensor(poses.reshape(-1, 12).astype(np.float32), device="cuda")
    outs = ("rgb", "depth", "normal", "alpha", "trans", "n_contrib", "n_walk")
    ref = None
    for bd in (0, 32, 128, 512):
        r = Renderer(scene.n, sensors, tiles=TILES, outputs=outs, batch_depth=bd)
        o = [{k: v.clone() for k, v in x.items()} for x in r.render_rig(d, P)]
        torch.cuda.synchronize()
        assert r.status()[0] == 0
        if ref is None:
            ref = o
            continue
        for i, (oa, ob) in enumerate(zip(ref, o)):
            for k in oa:
                assert torch.equal(oa[k], ob[k]), (bd, i, k)
    r = Renderer(scene.n, sensors, tiles=[(8, 8), (8, 4), (16, 16), (8, 8), (32, 8)], outputs=outs)
    o = r.render_rig(d, P)
    torch.cuda.synchronize()
    for i, (oa, ob) in enumerate(zip(ref, o)):
        for key in (("rgb", "depth") if "rgb" in oa else ("intensity", "range")):
            scale = 1.0 if key in ("rgb", "intensity") else max(1.0, float(oa[key].abs().max()))
            assert (oa[key] - ob[key]).abs().max() <= 1e-4 * scale, (i, key)


def test_autotune_picks_the_fastest_measured_tiling(gpu_lib):
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer
    scene, poses, sensors = _small_rig()
    bg_n = 60_000
    whole = DeviceSurfels.from_host(scene)
    parts = [DeviceSurfels.from_host(scene.subset(np.arange(bg_n))),
             DeviceSurfels.from_host(scene.subset(np.arange(bg_n, scene.n)))]
    P = torch.as_tensor(poses.reshape(-1, 12).astype(np.float32), device="cuda")
    outs = ("rgb", "depth", "normal", "alpha", "trans", "n_contrib", "n_walk")
    ref = Renderer(scene.n, sensors, tiles=TILES, outputs=outs)
    ref_out = [{k: v.clone() for k, v in o.items()} for o in ref.render_rig(whole, P)]
    r = Renderer(scene.n, sensors, tiles=TILES, outputs=outs)
    res = r.autotune(parts, P, camera_tiles=((16, 16), (8, 8)), lidar_tiles=((8, 8), (4, 8)),
                     batch_depths=(64, 128), warmup=1, reps=2)
    ok = [t for t in res["trials"] if t["ms"] > 0]
    assert len(res["trials"]) >= 4 and len(ok) == len(res["trials"])
    best = min(ok, key=lambda t: t["ms"])
    assert res["best_ms"] == pytest.approx(best["ms"])
    assert res["camera_tile"] == best["camera_tile"] and res["lidar_tile"] == best["lidar_tile"]
    assert res["batch_depth"] == best["batch_depth"]
    # each LiDAR's tile was tuned on its own too, and the plan keeps the best
    lidar_tiles = [(r.plan.sensors[i].tile_w, r.plan.sensors[i].tile_h)
                   for i, s in enumerate(sensors) if s.kind == "lidar"]
    assert lidar_tiles == [tuple(t) for t in best["lidar_tiles"][:2]]
    assert any(tuple(t["lidar_tiles"][0]) != tuple(t["lidar_tiles"][1]) for t in res["trials"])
    # the tuned plan renders the same frame (to the split-merge rounding)
    o = r.render_rig(whole, P)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    for i, (oa, ob) in enumerate(zip(ref_out, o)):
        for key in (("rgb", "depth") if "rgb" in oa else ("intensity", "range")):
            scale = 1.0 if key in ("rgb", "intensity") else max(1.0, float(oa[key].abs().max()))
            assert (oa[key] - ob[key]).abs().max() <= 1e-4 * scale, (i, key)


def test_split_lists_match_oracle_and_unsplit_render(gpu_lib):
    """Force every list longer than 256 positions to split into 64-position
    chunks: the merged frame matches the oracle and the unsplit frame (to
    the reassociated transmittance products)."""
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer
    scene, poses, sensors = _small_rig()
    d = DeviceSurfels.from_host(scene)
    P = torch.as_tensor(poses.reshape(-1, 12).astype(np.float32), device="cuda")
    outs = ("rgb", "depth", "normal", "alpha", "trans", "n_contrib", "n_walk")
    whole = Renderer(scene.n, sensors, tiles=TILES, outputs=outs, split=(1 << 24, 1 << 24))
    ref = [{k: v.clone() for k, v in o.items()} for o in whole.render_rig(d, P)]
    r = Renderer(scene.n, sensors, tiles=TILES, outputs=outs, split=(256, 64))
    out = r.render_rig(d, P)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    # the split path really ran: some lists are longer than 256
    ranges = r.region(6, torch.int32).view(-1, 2)
    assert int((ranges[:, 1] - ranges[:, 0]).max()) > 4 * 256
    for i, (oa, ob) in enumerate(zip(ref, out)):
        for key in (("rgb", "depth") if "rgb" in oa else ("intensity", "range")):
            scale = 1.0 if key in ("rgb", "intensity") else max(1.0, float(oa[key].abs().max()))
            assert (oa[key] - ob[key]).abs().max() <= 1e-5 * scale, (i, key)
        # the same stop positions and last contributors, except at rare rounding flips
        assert (oa["n_walk"] != ob["n_walk"]).float().mean() <= 1e-3
    g = [{k: v.cpu().numpy() for k, v in o.items()} for o in out]
    rng = np.random.default_rng(11)
    for s, gg in zip(sensors, g):
        idx = rng.choice(s.width * s.height, 400, replace=False)
        if s.kind == "lidar":
            check_lidar(gg, OR.render_lidar(scene, s, rays=idx, obj_pose=poses), rays=idx, max_flag=CAP[s.kind if s.kind == "lidar" else "camera"])
        else:
            check_camera(gg, OR.render_pinhole(scene, s, pixels=idx, obj_pose=poses), pix=idx, max_flag=CAP[s.kind if s.kind == "lidar" else "camera"])


def test_lidar_split_is_per_sensor(gpu_lib):
    """The LiDARs' own list split (gsr_sensor.split_*): LiDAR lists split
    into 64-position chunks while the cameras stay unsplit -- camera frames
    bit-exact against the unsplit plan, LiDAR frames to the merge rounding;
    the autotuner's LiDAR split candidates are measured and kept."""
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer
    scene, poses, sensors = _small_rig()
    d = DeviceSurfels.from_host(scene)
    P = torch.as_tensor(poses.reshape(-1, 12).astype(np.float32), device="cuda")
    outs = ("rgb", "depth", "normal", "alpha", "trans", "n_contrib", "n_walk")
    whole = Renderer(scene.n, sensors, tiles=TILES, outputs=outs, split=(1 << 24, 1 << 24))
    ref = [{k: v.clone() for k, v in o.items()} for o in whole.render_rig(d, P)]
    r = Renderer(scene.n, sensors, tiles=TILES, outputs=outs, split=(1 << 24, 1 << 24), lidar_split=(256, 64))
    assert r.lidar_split() == (256, 64)
    out = r.render_rig(d, P)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    info = r.region(8, torch.int32).view(-1, 4)
    for i, s in enumerate(sensors):
        tb = r.plan.tile_base[i], r.plan.tile_base[i + 1]
        n_split = int((info[tb[0]:tb[1], 0] > 0).sum())
        if s.kind == "lidar":
            assert n_split > 0, i
            for key in ("intensity", "range"):
                scale = 1.0 if key == "intensity" else max(1.0, float(ref[i][key].abs().max()))
                assert (ref[i][key] - out[i][key]).abs().max() <= 1e-5 * scale, (i, key)
        else:
            assert n_split == 0, i
            for key in ref[i]:
                assert torch.equal(ref[i][key], out[i][key]), (i, key)
    res = r.autotune([d], P, camera_tiles=(), lidar_tiles=(), batch_depths=(), split_firsts=(), split_chunks=(),
                     lidar_split_firsts=(512, 2048), lidar_split_chunks=(128,), warmup=1, reps=2)
    best = min((t for t in res["trials"] if t["ms"] > 0), key=lambda t: t["ms"])
    assert {t["lidar_split"][0] for t in res["trials"]} >= {512, 2048}
    assert res["lidar_split"] == best["lidar_split"]
