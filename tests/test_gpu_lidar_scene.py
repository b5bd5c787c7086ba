"""GPU parity of the LiDAR scene G^L (Sec. III-A: a camera scene and a
separate LiDAR scene, the LiDAR one carrying the ray-drop probability rho
and the intensity r), through the C ABI:

* the ray-drop output (sum w rho + T) of a LiDAR frame against the FP64
  oracle, 1e-4 absolute;
* a camera table and a LiDAR table in one plan (gsr_surfels.sees): each
  sensor sees only its own scene -- bit-exact against a plan holding that
  table alone, and against the oracle;
* the LiDAR head of the anchor decode (intensity, ray-drop logit) in FP32
  against the FP64 oracle and on the tensor cores against a BF16 emulation,
  and its backward against FP64 autograd.
"""
import numpy as np
import pytest
import torch

from oracle import mlp as OM
from oracle import render as OR
from paper_2503_11731_gb300 import gsr, synth

from parity import record
from test_gpu_forward import FLIP, _check_camera, _check_lidar

pytestmark = pytest.mark.gpu


def _lidar_scene(n, seed):
    s = synth.driving_scene(n=n, seed=seed, x_range=(-30.0, 30.0), n_boxes=8)
    rng = np.random.default_rng(seed + 1000)
    s.ray_drop = rng.normal(-1.0, 1.5, n).astype(np.float32)
    s.sh = np.zeros((n, 1, 3), np.float32)
    return s


def _check_drop(g, o, rays=None):
    drop = g["drop"]
    if rays is not None:
        yy, xx = np.divmod(np.asarray(rays), drop.shape[1])
        drop = drop[yy, xx]
    ok = o["flip"] <= FLIP
    err = np.abs(drop - o["drop"])[ok].max(initial=0)
    record(dict(kind="lidar", drop=err, flagged=int((~ok).sum()), n=int(ok.size), flagged_frac=float((~ok).mean()),
                cap=1.0))
    assert err <= 1e-4
    assert 0.05 < o["drop"].mean() < 0.95


def test_lidar_ray_drop_full_frame_parity(gpu_lib):
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer
    s = _lidar_scene(30_000, seed=21)
    lid = synth.spinning_lidar(32, 720, -25.0, 15.0, (0.0, 0.0, 1.8))
    r = Renderer(s.n, [lid], outputs=("range", "intensity", "drop", "alpha", "trans"))
    out = r.render(DeviceSurfels.from_host(s))
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    g = {k: v.cpu().numpy() for k, v in out[0].items()}
    o = OR.render_lidar(s, lid)
    _check_lidar(g, o, max_flag=0.006)  # measured 0.40 %
    _check_drop(g, o)
    # T and the drop output agree where nothing is hit
    miss = g["alpha"] == 0.0
    assert miss.any() and np.all(g["drop"][miss] == 1.0)


def test_camera_and_lidar_scenes_share_one_plan(gpu_lib):
    """G^C seen by the cameras only, G^L by the LiDARs only, in one plan, one
    sort and one compositing launch."""
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer
    C = synth.driving_scene(n=40_000, seed=22, x_range=(-20.0, 40.0), n_boxes=6)
    L = _lidar_scene(30_000, seed=23)
    cam = synth.pinhole(320, 200, 180.0, (0.0, 0.5, 1.5), yaw_deg=5.0)
    cyl = synth.cylindrical(480, 120, 200.0, 60.0, (0.0, 0.0, 1.6), yaw_deg=180.0)
    lid = synth.spinning_lidar(32, 720, -25.0, 15.0, (0.0, 0.0, 1.8))
    outs = ("rgb", "depth", "normal", "alpha", "trans", "range", "intensity", "drop")
    sensors = [cam, lid, cyl]
    r = Renderer(C.n + L.n, sensors, tiles=[(16, 8), (8, 8), (16, 8)], outputs=outs)
    dC = DeviceSurfels.from_host(C, sees=gsr.SEES_CAMERAS)
    dL = DeviceSurfels.from_host(L, sees=gsr.SEES_LIDARS)
    r.preprocess(dC, first=0)
    r.preprocess(dL, first=C.n)
    r.bin_sort()
    r.composite_rig()
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    got = [{k: v.clone() for k, v in o.items()} for o in r.out]
    # each sensor's frame equals a plan that holds its own scene alone
    for sens, scene, idx in (([cam, cyl], C, (0, 2)), ([lid], L, (1,))):
        alone = Renderer(scene.n, sens, tiles=[(16, 8) if s.kind != "lidar" else (8, 8) for s in sens],
                         outputs=outs)
        ref = alone.render_rig(DeviceSurfels.from_host(scene))
        torch.cuda.synchronize()
        for j, i in enumerate(idx):
            for k in ref[j]:
                assert torch.equal(ref[j][k], got[i][k]), (i, k)
    # and the oracle of each scene alone
    rng = np.random.default_rng(24)
    pix = rng.choice(cam.width * cam.height, 1500, replace=False)
    _check_camera({k: v.cpu().numpy() for k, v in got[0].items()}, OR.render_pinhole(C, cam, pixels=pix), pix=pix,
                  max_flag=0.004)  # measured 0.20 %
    rays = rng.choice(lid.beams * lid.columns, 1500, replace=False)
    ol = OR.render_lidar(L, lid, rays=rays)
    gl = {k: v.cpu().numpy() for k, v in got[1].items()}
    _check_lidar(gl, ol, rays=rays, max_flag=0.004)  # measured 0.20 %
    _check_drop(gl, ol, rays=rays)


def _anchors(n_surfels=20_000, seed=91):
    s = synth.driving_scene(n=n_surfels, seed=seed, x_range=(0.0, 30.0), n_boxes=4)
    anchors, _ = synth.anchors_from_surfels(s, k=10, seed=seed + 1)
    return anchors


def _lidar_model(seed=17):
    from paper_2503_11731_gb300.neural import NeuralModel
    W1, b1, W2, b2 = synth.init_lidar_mlp(seed)
    return (W1, b1, W2, b2), NeuralModel(W1, b1, W2, b2, head=gsr.HEAD_LIDAR)


def _lidar_table(t):
    return {k: getattr(t, k).cpu().numpy() for k in ("pos", "log_scale", "quat", "opacity", "intensity", "ray_drop")}


def test_lidar_head_decode_f32_matches_oracle(gpu_lib):
    from paper_2503_11731_gb300.neural import DeviceAnchors
    a = _anchors()
    origin = np.array([2.0, 0.0, 1.8])
    W, m = _lidar_model()
    tab = m.decode(DeviceAnchors(a), origin, precision=gsr.DECODE_F32)
    assert tab.sees == gsr.SEES_LIDARS
    t = _lidar_table(tab)
    ref = OM.decode(a, *W, origin, head="lidar")
    for k in ("pos", "log_scale", "quat", "opacity", "intensity", "ray_drop"):
        r = ref[k].detach().numpy().reshape(t[k].shape)
        assert np.abs(t[k] - r).max() <= 1e-5 * max(1.0, np.abs(r).max()), k
    assert np.all(tab.sh.cpu().numpy() == 0.0)


def test_lidar_head_decode_bf16_matches_emulation(gpu_lib):
    from paper_2503_11731_gb300.neural import DeviceAnchors
    a = _anchors()
    origin = np.array([2.0, 0.0, 1.8])
    (W1, b1, W2, b2), m = _lidar_model()
    t = _lidar_table(m.decode(DeviceAnchors(a), origin, precision=gsr.DECODE_BF16_TENSOR))
    ref = OM.decode(a, W1, b1, W2, b2, origin, head="lidar")
    bf = lambda x: torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float64)
    H = torch.relu(bf(ref["X"].numpy()) @ bf(W1) + torch.as_tensor(b1, dtype=torch.float64))
    Y = (bf(H.numpy()) @ bf(W2) + torch.as_tensor(b2, dtype=torch.float64)).numpy().reshape(-1, 10)
    assert np.abs(t["ray_drop"] - Y[:, 2]).max() <= 2e-2
    assert np.abs(t["intensity"] - 1 / (1 + np.exp(-Y[:, 1]))).max() <= 1e-2
    assert np.abs(t["opacity"] - Y[:, 0]).max() <= 2e-2


def test_lidar_head_decode_backward_matches_autograd(gpu_lib):
    from paper_2503_11731_gb300.neural import DeviceAnchors
    a = _anchors(n_surfels=5000, seed=93)
    origin = np.array([1.0, -1.0, 1.8])
    W0, m = _lidar_model()
    rng = np.random.default_rng(5)
    N = a.n * a.k
    g = {"opacity": rng.normal(size=N), "intensity": rng.normal(size=N), "ray_drop": rng.normal(size=N),
         "log_scale": rng.normal(size=(N, 2)), "quat": rng.normal(size=(N, 4))}
    W = [torch.tensor(x, dtype=torch.float64, requires_grad=True) for x in W0]
    f = torch.tensor(a.feature, dtype=torch.float64, requires_grad=True)
    out = OM.decode(a, *W, origin, features=f, head="lidar")
    L = sum((out[k] * torch.as_tensor(v)).sum() for k, v in g.items())
    L.backward()
    da = DeviceAnchors(a)
    m.zero_grads(da)
    m.backward(da, origin, {k: torch.as_tensor(v, dtype=torch.float32, device="cuda") for k, v in g.items()})
    torch.cuda.synchronize()
    for name, ref in zip(("w1", "b1", "w2", "b2", "feature"), (*W, f)):
        got = m.grads[name].cpu().numpy()
        r = ref.grad.numpy()
        err = np.abs(got - r).max() / np.abs(r).max()
        print(name, "rel err", err)
        assert err <= 1e-4, name
