"""GPU parity of the learned decode (anchor MLP) and its training kernels.

* FP32 SIMT decode vs the FP64 oracle (1e-5);
* BF16 tcgen05 decode vs an FP64 emulation of its BF16 rounding (inputs,
  weights and hidden activations rounded to BF16, FP32/FP64 accumulation);
* gsr_decode_backward vs FP64 autograd of the oracle decode;
* gsr_adam vs the closed-form Adam update;
* distillation: the network trained on the GPU by the project's own kernels
  (decode -> render -> loss -> backward -> decode backward -> Adam) against
  renders of the explicit scene, checked for its gain over the untrained
  network on held-out poses and for the BF16-vs-FP32 decode gap (<= 0.5 dB).
"""
import math

import numpy as np
import pytest
import torch

from oracle import mlp as OM
from paper_2503_11731_gb300 import gsr, synth

pytestmark = pytest.mark.gpu


def _setup(n_surfels=20_000, seed=81):
    s = synth.driving_scene(n=n_surfels, seed=seed, x_range=(0.0, 30.0), n_boxes=4)
    anchors, order = synth.anchors_from_surfels(s, k=10, seed=seed + 1)
    return s, anchors, order


def _model(seed=7):
    from paper_2503_11731_gb300.neural import NeuralModel
    return NeuralModel(*synth.init_mlp(seed))


def _table_np(t):
    return {k: getattr(t, k).cpu().numpy() for k in ("pos", "log_scale", "quat", "opacity", "sh", "intensity")}


def test_decode_f32_matches_oracle(gpu_lib):
    from paper_2503_11731_gb300.neural import DeviceAnchors
    _, a, _ = _setup()
    cam = synth.pinhole(160, 96, 90.0, (2.0, 0.0, 1.5), 0.0)
    origin = -cam.world_to_sensor[:3, :3].T @ cam.world_to_sensor[:3, 3]
    m = _model()
    t = _table_np(m.decode(DeviceAnchors(a), origin, cull_camera=cam, precision=gsr.DECODE_F32))
    ref = OM.decode(a, *synth.init_mlp(7), origin, cam=cam)
    culled = OM.cull_mask(a.pos.astype(np.float64), a.scale.astype(np.float64), a.offsets.astype(np.float64), cam)
    assert 0 < culled.sum() < a.n
    for k in ("pos", "log_scale", "quat", "opacity", "sh", "intensity"):
        r = ref[k].detach().numpy().reshape(t[k].shape)
        assert np.abs(t[k] - r).max() <= 1e-5 * max(1.0, np.abs(r).max()), k


def _bf16(x):
    return torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float64)


def test_decode_bf16_tensor_cores_match_bf16_emulation(gpu_lib):
    """The tcgen05 path: layer inputs and weights are BF16, accumulation FP32."""
    from paper_2503_11731_gb300.neural import DeviceAnchors
    _, a, _ = _setup()
    origin = np.array([1.0, 0.5, 1.5])
    W1, b1, W2, b2 = synth.init_mlp(7)
    m = _model()
    t = _table_np(m.decode(DeviceAnchors(a), origin, precision=gsr.DECODE_BF16_TENSOR))
    # emulation: X, W1 -> BF16; pre = X W1 + b1; H = relu(pre) -> BF16; Y = H W2 + b2 (W2 BF16)
    ref = OM.decode(a, W1, b1, W2, b2, origin)
    X = _bf16(ref["X"].numpy())
    H = torch.relu(X @ _bf16(W1) + torch.as_tensor(b1, dtype=torch.float64))
    Y = (_bf16(H.numpy()) @ _bf16(W2) + torch.as_tensor(b2, dtype=torch.float64)).numpy().reshape(-1, 10)
    got_logit = t["opacity"]
    err = np.abs(got_logit - Y[:, 0])
    print("bf16 decode: max |opacity logit - emulation|", err.max(), "max |logit|", np.abs(Y[:, 0]).max())
    assert err.max() <= 2e-2
    assert np.abs(t["quat"] - Y[:, 6:10]).max() <= 2e-2
    assert np.abs(t["log_scale"] - (Y[:, 4:6] + np.log(a.scale).repeat(10)[:, None])).max() <= 2e-2
    # and it is a real BF16 computation: close to, but not equal to, the FP32 path
    t32 = _table_np(m.decode(DeviceAnchors(a), origin, precision=gsr.DECODE_F32))
    d = np.abs(t["opacity"] - t32["opacity"])
    assert 0 < d.max() <= 5e-2


def test_decode_backward_matches_autograd(gpu_lib):
    from paper_2503_11731_gb300.neural import DeviceAnchors
    _, a, _ = _setup(n_surfels=5000, seed=83)
    cam = synth.pinhole(160, 96, 90.0, (2.0, 0.0, 1.5), 0.0)
    origin = -cam.world_to_sensor[:3, :3].T @ cam.world_to_sensor[:3, 3]
    rng = np.random.default_rng(2)
    N = a.n * a.k
    g = {"opacity": rng.normal(size=N), "sh": rng.normal(size=(N, 1, 3)), "log_scale": rng.normal(size=(N, 2)),
         "quat": rng.normal(size=(N, 4))}
    W = [torch.tensor(x, dtype=torch.float64, requires_grad=True) for x in synth.init_mlp(7)]
    f = torch.tensor(a.feature, dtype=torch.float64, requires_grad=True)
    out = OM.decode(a, *W, origin, cam=cam, features=f)
    L = sum((out[k] * torch.as_tensor(v)).sum() for k, v in g.items())
    L.backward()
    m = _model()
    da = DeviceAnchors(a)
    m.zero_grads(da)
    m.backward(da, origin, {k: torch.as_tensor(v, dtype=torch.float32, device="cuda") for k, v in g.items()},
               cull_camera=cam)
    torch.cuda.synchronize()
    for name, ref in zip(("w1", "b1", "w2", "b2", "feature"), (*W, f)):
        got = m.grads[name].cpu().numpy()
        r = ref.grad.numpy()
        err = np.abs(got - r).max() / np.abs(r).max()
        print(name, "rel err", err)
        assert err <= 1e-4, name


def test_adam_matches_closed_form(gpu_lib):
    rng = np.random.default_rng(3)
    p0 = rng.normal(size=1000).astype(np.float32)
    grads = [rng.normal(size=1000).astype(np.float32) for _ in range(3)]
    p = torch.as_tensor(p0, device="cuda").clone()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    import ctypes
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    pr, mr, vr = p0.astype(np.float64), np.zeros(1000), np.zeros(1000)
    for step, gg in enumerate(grads, 1):
        g = torch.as_tensor(gg, device="cuda")
        gsr.adam(P(p), P(g), P(m), P(v), 1000, 1e-2, 0.9, 0.999, 1e-8, step, None)
        mr = 0.9 * mr + 0.1 * gg
        vr = 0.999 * vr + 0.001 * gg.astype(np.float64) ** 2
        pr = pr - 1e-2 * (mr / (1 - 0.9 ** step)) / (np.sqrt(vr / (1 - 0.999 ** step)) + 1e-8)
    torch.cuda.synchronize()
    assert np.abs(p.cpu().numpy() - pr).max() <= 1e-5


def _psnr(a, b):
    mse = float(((a - b) ** 2).mean())
    return 10 * math.log10(1.0 / max(mse, 1e-12))


def test_distillation_trains_the_network_on_the_gpu(gpu_lib):
    """Train decode MLP + anchor features on renders of the explicit scene."""
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer, camera_backward, camera_loss
    from paper_2503_11731_gb300.neural import DeviceAnchors
    s, a, order = _setup()
    rng = np.random.default_rng(5)
    W, H, f = 96, 64, 60.0
    poses = [((rng.uniform(-4, 4), rng.uniform(-1, 1), 1.5), rng.uniform(-8, 8)) for _ in range(10)]
    train, held = poses[:7], poses[7:]
    cams = [synth.pinhole(W, H, f, p, yaw) for p, yaw in poses]
    ds = DeviceSurfels.from_host(s)
    targets = []
    for cam in cams:
        r = Renderer(s.n, [cam])
        targets.append(r.render(ds)[0]["rgb"].clone())
    da = DeviceAnchors(a)
    m = _model()
    outputs = ("rgb", "depth", "normal", "alpha", "trans", "depth_acc", "n_contrib")
    rends = [Renderer(a.n * a.k, [cam], outputs=outputs) for cam in cams]
    origin = lambda cam: -cam.world_to_sensor[:3, :3].T @ cam.world_to_sensor[:3, 3]

    def evaluate(idx, precision):
        vals = []
        for i in idx:
            t = m.decode(da, origin(cams[i]), precision=precision)
            img = rends[i].render(t)[0]["rgb"]
            vals.append(_psnr(img.clamp(0, 1).cpu().numpy(), targets[i].clamp(0, 1).cpu().numpy()))
        return float(np.mean(vals))

    held_idx = list(range(7, 10))
    before = evaluate(held_idx, gsr.DECODE_BF16_TENSOR)
    losses = []
    for step in range(240):
        i = step % 7
        cam = cams[i]
        t = m.decode(da, origin(cam), precision=gsr.DECODE_BF16_TENSOR)
        rends[i].render(t)
        loss, lo = camera_loss(rends[i], 0, targets[i], w_dist=0.0, w_normal=0.0)
        g = camera_backward(rends[i], 0, lo.struct(), t)
        m.zero_grads(da)
        m.backward(da, origin(cam), g)
        m.adam_step(da, lr=3e-3, lr_feature=1e-2)
        losses.append(float(loss[0]))
    after_bf16 = evaluate(held_idx, gsr.DECODE_BF16_TENSOR)
    after_f32 = evaluate(held_idx, gsr.DECODE_F32)
    print(f"held-out PSNR: untrained {before:.2f} dB, trained BF16 {after_bf16:.2f} dB, FP32 {after_f32:.2f} dB; "
          f"loss {np.mean(losses[:7]):.4f} -> {np.mean(losses[-7:]):.4f}")
    assert np.mean(losses[-7:]) < 0.8 * np.mean(losses[:7])
    assert after_bf16 >= before + 2.0          # the trained network's gain over the untrained one
    assert abs(after_bf16 - after_f32) <= 0.5  # BF16 decode within 0.5 dB of the FP32 decode
