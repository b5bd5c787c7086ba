"""GPU parity of the reconstruction loss and the hand-written backward pass.

* gsr_loss on oracle-rendered images vs the FP64 loss and its autograd
  per-pixel gradients;
* the full chain render -> loss -> gsr_backward (reverse rasteriser +
  preprocess backward) vs the FP64 oracle gradient on a 64x64 image with 200
  surfels: per parameter group max|g - g_ref| <= 1e-3 max|g_ref|, and
  elementwise relative 1e-3 where |g_ref| >= 1e-2 max|g_ref| (a small count
  of threshold-flip outliers allowed and reported);
* finite differences of the GPU loss along random directions;
* the 2M-surfel 1920x1080 step: finite, deterministic-in-loss, zero for
  surfels no pixel sees, a directional finite-difference check of the GPU
  loss, and the GPU gradient along a direction over 48 surfels against the
  central difference of the FP64 oracle's whole-frame loss.
"""
import numpy as np
import pytest
import torch

from oracle import grad as OG
from paper_2503_11731_gb300 import synth

pytestmark = pytest.mark.gpu


def _scene(n=200, seed=41, deg=1):
    s = synth.plain_scene(n=n, seed=seed)
    rng = np.random.default_rng(seed + 1)
    K = (deg + 1) ** 2
    sh = np.concatenate([s.sh, rng.normal(0, 0.2, (n, K - 1, 3)).astype(np.float32)], 1)
    # larger surfels than the forward test scene, so the small image is covered
    return synth.Surfels(s.pos, (s.log_scale + 1.0).astype(np.float32), s.quat, s.opacity, sh, s.intensity)


def _cam():
    return synth.plain_camera(64, 64, 48.0)


def _renderer(s, cam):
    from paper_2503_11731_gb300.frame import Renderer
    return Renderer(s.n, [cam], outputs=("rgb", "depth", "normal", "alpha", "trans", "depth_acc", "n_contrib"))


def _target(seed=3, H=64, W=64):
    return np.random.default_rng(seed).uniform(0, 1, (H, W, 3))


def test_loss_kernel_matches_fp64_loss(gpu_lib):
    """gsr_loss on the oracle's own images: loss terms and per-pixel gradients."""
    from paper_2503_11731_gb300.frame import camera_loss
    s, cam = _scene(), _cam()
    p = OG.surfel_tensors(s)
    out = OG.render_pinhole(p, cam)
    leaves = {k: out[k].detach().clone().requires_grad_(True) for k in ("rgb", "A", "B", "D", "normal")}
    tgt = _target()
    L, parts = OG.loss(leaves, torch.as_tensor(tgt), cam)
    L.backward()
    r = _renderer(s, cam)
    o = r.out[0]
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    o["rgb"].copy_(dev(np.moveaxis(leaves["rgb"].detach().numpy(), -1, 0)))
    o["alpha"].copy_(dev(leaves["A"].detach().numpy()))
    o["depth_acc"].copy_(dev(np.stack([leaves["B"].detach().numpy(), leaves["D"].detach().numpy()])))
    o["normal"].copy_(dev(np.moveaxis(leaves["normal"].detach().numpy(), -1, 0)))
    loss, g = camera_loss(r, 0, dev(np.moveaxis(tgt, -1, 0)))
    torch.cuda.synchronize()
    lv = loss.cpu().numpy()
    assert lv[0] == pytest.approx(float(L), rel=1e-4)
    assert lv[1] == pytest.approx(float(parts["l1"]), rel=1e-4)
    assert lv[2] == pytest.approx(0.1 * float(parts["dist"]), rel=1e-4, abs=1e-7)
    assert lv[3] == pytest.approx(0.05 * float(parts["normal"]), rel=1e-4, abs=1e-7)
    ref = {"rgb": np.moveaxis(leaves["rgb"].grad.numpy(), -1, 0), "alpha": leaves["A"].grad.numpy(),
           "depth_acc": np.stack([leaves["B"].grad.numpy(), leaves["D"].grad.numpy()]),
           "normal": np.moveaxis(leaves["normal"].grad.numpy(), -1, 0)}
    for k in ref:
        got = getattr(g, k).cpu().numpy()
        scale = np.abs(ref[k]).max()
        err = np.abs(got - ref[k]).max()
        print(k, "max|ref|", scale, "max err", err)
        assert err <= 1e-4 * scale + 1e-9, k


def _gpu_grad(s, cam, tgt):
    from paper_2503_11731_gb300.frame import DeviceSurfels, camera_backward, camera_loss
    r = _renderer(s, cam)
    d = DeviceSurfels.from_host(s)
    r.render(d)
    loss, lo = camera_loss(r, 0, torch.as_tensor(np.moveaxis(tgt, -1, 0).copy(), dtype=torch.float32, device="cuda"))
    g = camera_backward(r, 0, lo.struct(), d)
    torch.cuda.synchronize()
    return float(loss[0]), {k: v.cpu().numpy() for k, v in g.items()}


def _compare_groups(g, ref, tol=1e-3, max_outliers=0.01):
    for k in ("pos", "log_scale", "quat", "opacity", "sh"):
        a, b = g[k].reshape(-1), ref[k].reshape(-1)
        scale = np.abs(b).max()
        err = np.abs(a - b)
        big = np.abs(b) >= 1e-2 * scale
        rel = err[big] / np.abs(b[big])
        n_out = int((rel > tol).sum())
        print(f"{k}: max|ref| {scale:.3e} max err {err.max():.3e} ({err.max() / scale:.2e} of max), "
              f"elementwise rel>1e-3: {n_out}/{big.sum()}")
        assert err.max() <= tol * scale, k
        assert n_out <= max(1, int(max_outliers * big.sum())), k


def test_gradient_matches_fp64_oracle(gpu_lib):
    """64x64 image, 200 surfels (SH degree 1): full chain vs FP64 autograd."""
    s, cam = _scene(), _cam()
    tgt = _target()
    L_ref, g_ref, parts = OG.loss_and_grad(s, cam, tgt)
    assert parts["normal"] > 0 and parts["dist"] > 0
    L, g = _gpu_grad(s, cam, tgt)
    assert L == pytest.approx(L_ref, rel=1e-4)
    _compare_groups(g, g_ref)


def test_gradient_matches_oracle_sh3_posed_camera(gpu_lib):
    s = synth.driving_scene(n=200, seed=43, x_range=(3.0, 12.0), n_boxes=2)
    s = synth.Surfels(s.pos, (s.log_scale + 0.5).astype(np.float32), s.quat, s.opacity, s.sh, s.intensity)
    cam = synth.pinhole(64, 64, 40.0, (0.0, 0.0, 1.5), yaw_deg=5.0, pitch_deg=-12.0)
    tgt = _target(5)
    L_ref, g_ref, _ = OG.loss_and_grad(s, cam, tgt)
    L, g = _gpu_grad(s, cam, tgt)
    assert L == pytest.approx(L_ref, rel=1e-4)
    _compare_groups(g, g_ref)


def test_gradient_finite_differences_on_gpu(gpu_lib):
    """Central differences of the GPU loss (FP32) along random directions."""
    from paper_2503_11731_gb300.frame import DeviceSurfels, camera_loss
    s, cam = _scene(seed=51), _cam()
    tgt = _target(7)
    L0, g = _gpu_grad(s, cam, tgt)
    r = _renderer(s, cam)
    t = torch.as_tensor(np.moveaxis(tgt, -1, 0).copy(), dtype=torch.float32, device="cuda")

    def loss_of(ss):
        r.render(DeviceSurfels.from_host(ss))
        return float(camera_loss(r, 0, t)[0][0])
    rng = np.random.default_rng(9)
    # perturb a few surfels at a time: a shift of every surfel crosses many
    # support / alpha-skip boundaries, which FP32 differences cannot resolve.
    # Rotations are left out: turning a surfel moves its whole hard support
    # boundary, so the loss jumps along that direction and the difference
    # quotient grows as the step shrinks instead of converging; the rotation
    # gradient is checked against the FP64 oracle gradient above.
    steps = {"pos": 1e-3, "log_scale": 1e-3, "opacity": 1e-2, "sh": 1e-2}
    tols = {}
    for name, h in steps.items():
        base = getattr(s, name)
        v = rng.normal(size=base.shape).astype(np.float32)
        keep = np.zeros(base.shape[0], bool)
        keep[rng.choice(base.shape[0], 16, replace=False)] = True
        v[~keep] = 0.0
        mk = lambda sign: synth.Surfels(**{**{k: getattr(s, k) for k in ("pos", "log_scale", "quat", "opacity",
                                                                            "sh", "intensity")},
                                           name: (base + sign * h * v).astype(np.float32)})
        fd = (loss_of(mk(1)) - loss_of(mk(-1))) / (2 * h)
        ad = float((g[name] * v).sum())
        print(name, "fd", fd, "ad", ad)
        assert ad == pytest.approx(fd, rel=tols.get(name, 5e-2), abs=2e-5), name


def test_backward_full_size_step(gpu_lib):
    """2M surfels at 1920x1080 (the backward-step workload)."""
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer, camera_backward, camera_loss
    s = synth.driving_scene(n=2_000_000, seed=synth.SEED_BASE + 3)
    tgt_scene = synth.perturbed(s, seed=synth.SEED_BASE + 30)
    cam = synth.driving_camera()
    r = Renderer(s.n, [cam], outputs=("rgb", "depth", "normal", "alpha", "trans", "depth_acc", "n_contrib"))
    r.render(DeviceSurfels.from_host(tgt_scene))
    target = r.out[0]["rgb"].clone()
    d = DeviceSurfels.from_host(s)
    r.render(d)
    loss, lo = camera_loss(r, 0, target)
    g = camera_backward(r, 0, lo.struct(), d)
    L1 = float(loss[0])
    # the loss is deterministic; gradients are finite
    r.render(d)
    loss2, _ = camera_loss(r, 0, target)
    assert float(loss2[0]) == L1
    for k, v in g.items():
        assert torch.isfinite(v).all(), k
    # surfels no camera record reached get exactly zero gradient
    counts = r.region(2, torch.int32)[: s.n]
    invisible = counts == 0
    assert invisible.any()
    assert (g["opacity"][invisible] == 0).all() and (g["pos"][invisible] == 0).all()
    # directional finite difference along the gradient of the opacity logits
    gop = g["opacity"]
    v = gop / gop.norm()
    h = 0.05

    def loss_with(op):
        dd = DeviceSurfels(d.pos, d.log_scale, d.quat, op.contiguous(), d.sh)
        r.render(dd)
        return float(camera_loss(r, 0, target)[0][0])
    fd = (loss_with(d.opacity + h * v) - loss_with(d.opacity - h * v)) / (2 * h)
    ad = float((gop * v).sum())
    print("full-size directional derivative fd", fd, "ad", ad)
    assert ad == pytest.approx(fd, rel=5e-2)


def test_autograd_function_matches_direct_calls(gpu_lib):
    from paper_2503_11731_gb300.frame import CameraLossFunction, RenderCameraFunction
    s, cam = _scene(seed=61), _cam()
    tgt = _target(11)
    L_direct, g_direct = _gpu_grad(s, cam, tgt)
    r = _renderer(s, cam)
    f = lambda a: torch.as_tensor(a, dtype=torch.float32, device="cuda").requires_grad_(True)
    params = [f(s.pos), f(s.log_scale), f(s.quat), f(s.opacity), f(s.sh)]
    rgb, A, dacc, nrm = RenderCameraFunction.apply(r, 0, *params)
    t = torch.as_tensor(np.moveaxis(tgt, -1, 0).copy(), dtype=torch.float32, device="cuda")
    L = CameraLossFunction.apply(r, 0, t, rgb, A, dacc, nrm)
    L.backward()
    assert float(L) == pytest.approx(L_direct, rel=1e-6)
    for k, p in zip(("pos", "log_scale", "quat", "opacity", "sh"), params):
        np.testing.assert_allclose(p.grad.cpu().numpy(), g_direct[k], rtol=1e-4, atol=1e-7 * np.abs(g_direct[k]).max())


def test_split_backward_matches_unsplit(gpu_lib):
    """Long lists split (forward chunks merged, backward chunks walked in
    parallel from the states the merge stored) give the gradients of the
    unsplit walk, to the reassociation of the transmittance products."""
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer, camera_backward, camera_loss
    s = synth.driving_scene(n=60_000, seed=synth.SEED_BASE + 61, x_range=(-10.0, 40.0), n_boxes=6)
    tgt = synth.perturbed(s, seed=synth.SEED_BASE + 62)
    cam = synth.pinhole(320, 192, 200.0, (0.0, 0.0, 1.5), 0.0)
    outs = ("rgb", "depth", "normal", "alpha", "trans", "depth_acc", "n_contrib")
    grads = []
    for split in ((1 << 24, 1 << 24), (256, 64)):
        r = Renderer(s.n, [cam], tiles=[(16, 8)], outputs=outs, split=split)
        r.render(DeviceSurfels.from_host(tgt))
        target = r.out[0]["rgb"].clone()
        d = DeviceSurfels.from_host(s)
        r.render(d)
        loss, lo = camera_loss(r, 0, target)
        g = camera_backward(r, 0, lo.struct(), d)
        torch.cuda.synchronize()
        assert r.status()[0] == 0
        if split[0] == 256:
            ranges = r.region(6, torch.int32).view(-1, 2)
            assert int((ranges[:, 1] - ranges[:, 0]).max()) > 8 * 256  # the chunk path ran
        grads.append({k: v.cpu().numpy() for k, v in g.items()})
    for k in grads[0]:
        a, b = grads[0][k], grads[1][k]
        scale = np.abs(a).max()
        assert scale > 0, k
        err = np.abs(a - b).max() / scale
        print("split vs unsplit gradient", k, err)
        assert err <= 1e-3, k


def test_full_size_gradient_matches_oracle_directional_derivative(gpu_lib):
    """2M surfels at 1920x1080 (the backward-step workload; loss L1 + 0.1
    distortion + 0.05 normal consistency against the oracle's render of a
    perturbed copy): the GPU gradient along a random direction v over the
    parameters of 48 large on-screen surfels equals the central difference
    of the FP64 oracle's loss (its tiled whole-frame render) along v.

    The rendered image jumps where two surfels' centre depths cross (the
    compositing order swaps), and the scene's coplanar box faces hold
    surfels with exactly equal centre depths: v moves only surfels whose
    centre depth lies at least 1e-4 from every other surfel's, so no order
    (FP64 or FP32 key) changes within +-h.  It also jumps where a pixel's
    alpha crosses the 1/255 skip threshold (about 1e-9 of the loss each);
    such a crossing adds J / 2h to the difference, and its odds grow with
    h.  For this v the difference is 4.124e-3 at h = 1e-6, 4.278e-3 at
    1e-8 and 4.272e-3 at 1e-9: h = 1e-8 keeps the crossings' share below
    6e-6, a tenth of the tolerance, while the FP64 loss's rounding (about
    1e-14) adds about 5e-7.  The
    surfels are chosen on the host: the 48 with the largest projected scale
    whose centres lie in view.  Tolerance: 2e-3 of sum_i |g_i v_i|, the FP32
    gradient's accumulated rounding with margin."""
    from oracle import render as OR
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer, camera_backward, camera_loss
    s = synth.driving_scene(n=2_000_000, seed=synth.SEED_BASE + 3)
    tgt_scene = synth.perturbed(s, seed=synth.SEED_BASE + 30)
    cam = synth.driving_camera()
    target = OR.render_pinhole(tgt_scene, cam, tile=16)["rgb"]                      # [H, W, 3] FP64
    r = Renderer(s.n, [cam], outputs=("rgb", "depth", "normal", "alpha", "trans", "depth_acc", "n_contrib"))
    d = DeviceSurfels.from_host(s)
    r.render(d)
    t_gpu = torch.as_tensor(np.moveaxis(target, -1, 0).astype(np.float32).copy(), device="cuda")
    loss, lo = camera_loss(r, 0, t_gpu)
    g = camera_backward(r, 0, lo.struct(), d)
    torch.cuda.synchronize()
    g = {k: v.double().cpu().numpy() for k, v in g.items()}
    P = np.c_[s.pos.astype(np.float64), np.ones(s.n)] @ np.asarray(cam.world_to_sensor, np.float64).T
    zc = P[:, 2]
    zs = np.where(zc > 0, zc, 1.0)
    u, w = cam.fx * P[:, 0] / zs + cam.cx, cam.fy * P[:, 1] / zs + cam.cy
    inside = (zc > 1.0) & (u > 0) & (u < cam.width) & (w > 0) & (w < cam.height)
    size = np.exp(s.log_scale.astype(np.float64).max(1)) * cam.fx / zs
    order = np.argsort(zc, kind="stable")
    close = np.diff(zc[order]) < 1e-4
    tied = np.zeros(s.n, bool)
    tied[order[1:][close]] = True
    tied[order[:-1][close]] = True
    cand = np.flatnonzero(inside & ~tied)
    idx = cand[np.argsort(-size[cand], kind="stable")[:48]]
    assert len(idx) == 48
    rng = np.random.default_rng(7)
    names = ("pos", "log_scale", "quat", "opacity", "sh")
    v = {k: np.zeros(getattr(s, k).shape, np.float64) for k in names}
    for k in names:
        v[k][idx] = rng.normal(size=v[k][idx].shape)
    terms = np.concatenate([(g[k] * v[k]).ravel() for k in names])
    ad = float(terms.sum())

    def oracle_loss(eps):
        moved = synth.Surfels(*(getattr(s, k).astype(np.float64) + eps * v[k] for k in names),
                              s.intensity.astype(np.float64))
        o = OR.render_pinhole(moved, cam, tile=16)
        out = {"rgb": torch.as_tensor(o["rgb"]), "A": torch.as_tensor(o["acc"][..., 0]),
               "B": torch.as_tensor(o["acc"][..., 1]), "D": torch.as_tensor(o["acc"][..., 2]),
               "normal": torch.as_tensor(o["normal"])}
        return float(OG.loss(out, torch.as_tensor(target), cam)[0])
    h = 1e-8
    fd = (oracle_loss(h) - oracle_loss(-h)) / (2 * h)
    scale = float(np.abs(terms).sum())
    print("full-size directional derivative: GPU", ad, "FP64 oracle central difference", fd, "scale", scale)
    assert scale > 0
    assert abs(ad - fd) <= 2e-3 * scale
