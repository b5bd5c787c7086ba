"""Pins of the FP64 gradient oracle (oracle/grad.py).

The gradient oracle is autograd over a tensor restatement of the render; it
is pinned by central finite differences of the *C* oracle (an independent
implementation of the same definitions), by an analytic depth-normal case,
and by the pairwise form of the distortion term.
"""
import math

import numpy as np
import pytest
import torch

from oracle import grad as OG
from oracle import render as R
from paper_2503_11731_gb300 import synth


def _small_scene(n=60, seed=21, deg=1):
    s = synth.plain_scene(n=n, seed=seed)
    rng = np.random.default_rng(seed + 1)
    K = (deg + 1) ** 2
    sh = np.concatenate([s.sh.astype(np.float64), rng.normal(0, 0.2, (n, K - 1, 3))], 1)
    return synth.Surfels(s.pos.astype(np.float64), s.log_scale.astype(np.float64) + 0.8,
                         s.quat.astype(np.float64), s.opacity.astype(np.float64), sh,
                         s.intensity.astype(np.float64))


def _with(s, name, arr):
    d = dict(pos=s.pos, log_scale=s.log_scale, quat=s.quat, opacity=s.opacity, sh=s.sh, intensity=s.intensity)
    d[name] = arr
    return synth.Surfels(**d)


def _c_outputs(s, cam):
    o = R.render_pinhole(s, cam, bg=(0.1, 0.2, 0.3))
    return {"rgb": o["rgb"], "A": o["acc"][..., 0], "B": o["acc"][..., 1], "D": o["acc"][..., 2],
            "normal": o["normal"]}


@pytest.mark.parametrize("seed", [21, 22])
def test_render_vjp_matches_fd_of_c_oracle(seed):
    """<d(sum r.out)/dp, v> by autograd == central FD of the C oracle along v."""
    s = _small_scene(seed=seed)
    cam = synth.plain_camera(32, 24, 24.0)
    rng = np.random.default_rng(seed + 100)
    outs = _c_outputs(s, cam)
    weights = {k: rng.normal(size=v.shape) for k, v in outs.items()}
    weights["B"] *= 0.05
    weights["D"] *= 0.002
    p = OG.surfel_tensors(s, requires_grad=True)
    t = OG.render_pinhole(p, cam, bg=(0.1, 0.2, 0.3))
    tot = sum((torch.as_tensor(weights[k]) * t[k]).sum() for k in weights)
    tot.backward()
    h = 1e-6
    for name in ("pos", "log_scale", "quat", "opacity", "sh"):
        v = rng.normal(size=getattr(s, name).shape)
        base = getattr(s, name)
        fp = _c_outputs(_with(s, name, base + h * v), cam)
        fm = _c_outputs(_with(s, name, base - h * v), cam)
        fd = sum(((weights[k] * (fp[k] - fm[k])).sum() for k in weights)) / (2 * h)
        ad = float((p[name].grad.numpy() * v).sum())
        assert ad == pytest.approx(fd, rel=2e-5, abs=1e-6), name


def test_loss_gradient_matches_fd():
    """Full loss (L1 + distortion + normal consistency) through the C render."""
    s = _small_scene(n=80, seed=31, deg=0)
    cam = synth.plain_camera(28, 20, 20.0)
    rng = np.random.default_rng(5)
    target = rng.uniform(0, 1, (20, 28, 3))
    L, g, parts = OG.loss_and_grad(s, cam, target, bg=(0.1, 0.2, 0.3))
    assert parts["normal"] > 0 and parts["dist"] > 0

    def c_loss(ss):
        o = _c_outputs(ss, cam)
        out = {"rgb": torch.as_tensor(o["rgb"]), "A": torch.as_tensor(o["A"]), "B": torch.as_tensor(o["B"]),
               "D": torch.as_tensor(o["D"]), "normal": torch.as_tensor(o["normal"])}
        return float(OG.loss(out, torch.as_tensor(target), cam)[0])
    assert c_loss(s) == pytest.approx(L, rel=1e-12)
    h = 1e-6
    for name in ("pos", "log_scale", "quat", "opacity", "sh"):
        v = rng.normal(size=getattr(s, name).shape)
        base = getattr(s, name)
        fd = (c_loss(_with(s, name, base + h * v)) - c_loss(_with(s, name, base - h * v))) / (2 * h)
        ad = float((g[name] * v).sum())
        assert ad == pytest.approx(fd, rel=1e-4, abs=1e-7), name


def test_depth_normal_of_a_tilted_plane():
    """N_d from central differences of the back-projected depth of a plane
    n.X = c is the plane normal facing the camera, at every interior pixel,
    so the normal term is 0 when the rendered normal is that normal (A = 1)."""
    cam = synth.Pinhole(24, 16, 30.0, 32.0, 12.0, 8.0, np.eye(4), 0.2)
    n = np.array([0.3, -0.4, -1.0])
    n /= np.linalg.norm(n)
    c = -5.0  # plane n.X = c, in front of the camera (n points back at it)
    ys, xs = np.mgrid[0:16, 0:24]
    ray = np.stack([(xs + 0.5 - 12.0) / 30.0, (ys + 0.5 - 8.0) / 32.0, np.ones_like(xs, float)], -1)
    Z = c / (ray @ n)
    A = torch.ones(16, 24, dtype=torch.float64)
    out = {"rgb": torch.zeros(16, 24, 3, dtype=torch.float64), "A": A,
           "B": torch.as_tensor(Z), "D": torch.as_tensor(Z * Z),
           "normal": torch.as_tensor(np.broadcast_to(n, (16, 24, 3)).copy())}
    L, parts = OG.loss(out, torch.zeros(16, 24, 3, dtype=torch.float64), cam)
    assert float(parts["normal"]) == pytest.approx(0.0, abs=1e-12)
    assert float(parts["dist"]) == pytest.approx(0.0, abs=1e-9)
    # with the opposite rendered normal every interior pixel costs 2
    out["normal"] = -out["normal"]
    _, parts = OG.loss(out, torch.zeros(16, 24, 3, dtype=torch.float64), cam)
    assert float(parts["normal"]) == pytest.approx(2.0 * 14 * 22 / (16 * 24), rel=1e-12)


def _lidar_scene(seed):
    s = synth.driving_scene(n=300, seed=seed, x_range=(-8.0, 8.0), n_boxes=1)
    rng = np.random.default_rng(seed + 7)
    f = lambda a: np.asarray(a, np.float64)
    return synth.Surfels(f(s.pos), f(s.log_scale) + 0.3, f(s.quat), f(s.opacity), f(s.sh), f(s.intensity),
                         ray_drop=rng.normal(0, 1, s.n))


def _c_lidar(s, lid):
    o = R.render_lidar(s, lid)
    return {"A": o["alpha"], "B": o["range"] * o["alpha"], "I": o["intensity"], "drop": o["drop"], "T": o["T"]}


@pytest.mark.parametrize("seed", [3, 4])
def test_lidar_render_vjp_matches_fd_of_c_oracle(seed):
    """Eq. 5 LiDAR render: <d(sum r.out)/dp, v> by autograd == central FD of
    the C oracle along v, for alpha, sum w t, intensity, ray drop and T."""
    s = _lidar_scene(seed)
    lid = synth.spinning_lidar(10, 72, -25.0, 10.0, (0.0, 0.0, 1.8))
    rng = np.random.default_rng(seed + 200)
    outs = _c_lidar(s, lid)
    assert (outs["A"] > 0.5).mean() > 0.1  # the scene covers part of the scan
    weights = {k: rng.normal(size=v.shape) for k, v in outs.items()}
    weights["B"] *= 0.05
    names = ("pos", "log_scale", "quat", "opacity", "intensity", "ray_drop")
    p = {k: torch.tensor(getattr(s, k), requires_grad=True) for k in names}
    t = OG.render_lidar(p, lid)
    tot = sum((torch.as_tensor(weights[k]) * t[k]).sum() for k in weights)
    tot.backward()
    h = 1e-6
    for name in names:
        v = rng.normal(size=getattr(s, name).shape)
        base = getattr(s, name)
        fp = _c_lidar(_with_lidar(s, name, base + h * v), lid)
        fm = _c_lidar(_with_lidar(s, name, base - h * v), lid)
        fd = sum(((weights[k] * (fp[k] - fm[k])).sum() for k in weights)) / (2 * h)
        ad = float((p[name].grad.numpy() * v).sum())
        assert ad == pytest.approx(fd, rel=2e-5, abs=1e-6), name


def _with_lidar(s, name, arr):
    d = dict(pos=s.pos, log_scale=s.log_scale, quat=s.quat, opacity=s.opacity, sh=s.sh, intensity=s.intensity,
             ray_drop=s.ray_drop)
    d[name] = arr
    return synth.Surfels(**d)


def test_lidar_loss_worked_example():
    """Three rays, values worked by hand: ray 0 returns at 10 m (rendered
    range 12/1.2 = 10, intensity 0.5 vs 0.3); ray 1 returns at 20 m
    (rendered 18, intensity 0.1 vs 0.2); ray 2 has no return (drop 0.8)."""
    A = torch.tensor([1.2, 0.9, 0.2], dtype=torch.float64)
    out = {"A": A, "B": torch.tensor([12.0, 0.9 * 18.0, 0.5], dtype=torch.float64),
           "I": torch.tensor([0.5, 0.1, 0.0], dtype=torch.float64),
           "drop": torch.tensor([0.1, 0.3, 0.8], dtype=torch.float64)}
    L, lr, li, ld = OG.lidar_loss(out, [10.0, 20.0, 0.0], [0.3, 0.2, 0.0], w_range=1.0, w_int=2.0, w_drop=0.5)
    assert float(lr) == pytest.approx((0.0 + 2.0) / 2)
    assert float(li) == pytest.approx(2.0 * (0.2 + 0.1) / 2)
    assert float(ld) == pytest.approx(0.5 * (-math.log(0.9) - math.log(0.7) - math.log(0.8)) / 3)
    assert float(L) == pytest.approx(float(lr + li + ld))
    # no returns at all: only the drop term, and a sure drop costs ~0
    L0, lr0, li0, ld0 = OG.lidar_loss({k: v[2:] for k, v in out.items()}, [0.0], [0.0])
    assert float(lr0) == 0.0 and float(li0) == 0.0 and float(ld0) == pytest.approx(-0.1 * math.log(0.8))
    one = {"A": torch.zeros(1, dtype=torch.float64), "B": torch.zeros(1, dtype=torch.float64),
           "I": torch.zeros(1, dtype=torch.float64), "drop": torch.ones(1, dtype=torch.float64)}
    assert float(OG.lidar_loss(one, [0.0], [0.0])[0]) == pytest.approx(-0.1 * math.log(1 - 2.0 ** -20))
    # a sure drop where the target has a return costs the clamped -log(2^-20)
    assert float(OG.lidar_loss(one, [5.0], [0.0])[3]) == pytest.approx(0.1 * 20 * math.log(2.0))


def _cyl_scene(seed):
    s = synth.driving_scene(n=200, seed=seed, x_range=(-6.0, 14.0), n_boxes=2)
    f = lambda a: np.asarray(a, np.float64)
    sh = f(s.sh)[:, :4]  # SH degree 1
    return synth.Surfels(f(s.pos), f(s.log_scale) + 0.6, f(s.quat), f(s.opacity), sh, f(s.intensity))


def _cyl_cam():
    return synth.cylindrical(48, 20, 200.0, 50.0, (0.0, 0.0, 1.5), pitch_deg=-10.0)


@pytest.mark.parametrize("seed", [9, 10])
def test_cylindrical_render_vjp_matches_fd_of_c_oracle(seed):
    """Eq. 4 cylindrical render: autograd VJP == central FD of the C oracle."""
    s, cam = _cyl_scene(seed), _cyl_cam()
    rng = np.random.default_rng(seed + 100)
    outs = _c_outputs(s, cam)
    assert (outs["A"] > 0.5).mean() > 0.1
    weights = {k: rng.normal(size=v.shape) for k, v in outs.items()}
    weights["B"] *= 0.05
    weights["D"] *= 0.002
    p = OG.surfel_tensors(s, requires_grad=True)
    t = OG.render_cylindrical(p, cam, bg=(0.1, 0.2, 0.3))
    tot = sum((torch.as_tensor(weights[k]) * t[k]).sum() for k in weights)
    tot.backward()
    h = 1e-6
    for name in ("pos", "log_scale", "quat", "opacity", "sh"):
        v = rng.normal(size=getattr(s, name).shape)
        base = getattr(s, name)
        fp = _c_outputs(_with(s, name, base + h * v), cam)
        fm = _c_outputs(_with(s, name, base - h * v), cam)
        fd = sum(((weights[k] * (fp[k] - fm[k])).sum() for k in weights)) / (2 * h)
        ad = float((p[name].grad.numpy() * v).sum())
        assert ad == pytest.approx(fd, rel=2e-5, abs=1e-6), name


def test_cylindrical_loss_gradient_matches_fd():
    """Full camera loss (L1 + distortion + normal consistency through the
    cylindrical back-projection) through the C render."""
    s, cam = _cyl_scene(12), _cyl_cam()
    rng = np.random.default_rng(6)
    target = rng.uniform(0, 1, (cam.height, cam.width, 3))
    L, g, parts = OG.loss_and_grad(s, cam, target, bg=(0.1, 0.2, 0.3))
    assert parts["normal"] > 0 and parts["dist"] > 0

    def c_loss(ss):
        o = _c_outputs(ss, cam)
        out = {k: torch.as_tensor(o[k]) for k in ("rgb", "A", "B", "D", "normal")}
        return float(OG.loss(out, torch.as_tensor(target), cam)[0])
    assert c_loss(s) == pytest.approx(L, rel=1e-12)
    h = 1e-6
    for name in ("pos", "log_scale", "quat", "opacity", "sh"):
        v = rng.normal(size=getattr(s, name).shape)
        base = getattr(s, name)
        fd = (c_loss(_with(s, name, base + h * v)) - c_loss(_with(s, name, base - h * v))) / (2 * h)
        ad = float((g[name] * v).sum())
        assert ad == pytest.approx(fd, rel=1e-4, abs=1e-7), name


def test_depth_normal_of_a_plane_cylindrical():
    """A plane n.X = c seen by a cylindrical camera: the depth (horizontal
    distance) of pixel (x, y) is c / (d . n) with d = (sin phi, y_n, cos phi);
    its back-projection lies on the plane, so N_d = n at every interior
    pixel and the normal term vanishes for the rendered normal n."""
    W, H = 40, 16
    cam = synth.Cylindrical(W, H, W / math.radians(120.0), 20.0, W / 2, H / 2, np.eye(4), 0.2)
    n = np.array([0.2, -0.3, -1.0])
    n /= np.linalg.norm(n)
    c = -6.0
    ys, xs = np.mgrid[0:H, 0:W]
    phi = (xs + 0.5 - cam.cx) / cam.fx
    d = np.stack([np.sin(phi), (ys + 0.5 - cam.cy) / cam.fy, np.cos(phi)], -1)
    Z = c / (d @ n)
    assert (Z > 0).all()
    out = {"rgb": torch.zeros(H, W, 3, dtype=torch.float64), "A": torch.ones(H, W, dtype=torch.float64),
           "B": torch.as_tensor(Z), "D": torch.as_tensor(Z * Z),
           "normal": torch.as_tensor(np.broadcast_to(n, (H, W, 3)).copy())}
    _, parts = OG.loss(out, torch.zeros(H, W, 3, dtype=torch.float64), cam)
    assert float(parts["normal"]) == pytest.approx(0.0, abs=1e-12)
    # the pinhole back-projection of the same depths is not planar
    pin = synth.Pinhole(W, H, cam.fx, cam.fy, cam.cx, cam.cy, np.eye(4), 0.2)
    _, parts_pin = OG.loss(out, torch.zeros(H, W, 3, dtype=torch.float64), pin)
    assert float(parts_pin["normal"]) > 1e-3


def _loss_example(A_edge=1.0):
    """3x3 image, fx = fy = 1, principal point (1.5, 1.5): the centre pixel's
    ray is the optical axis and pixel (x, y) back-projects its depth d to
    d (x - 1, y - 1, 1).  Every pixel renders rgb 0.5, A = 1, B = 2 (depth 2),
    D = 4 (no spread) except where stated; A of pixel (2, 1) is A_edge."""
    cam = synth.Pinhole(3, 3, 1.0, 1.0, 1.5, 1.5, np.eye(4), 0.2)
    rgb = torch.full((3, 3, 3), 0.5, dtype=torch.float64)
    target = rgb.clone()
    target[0, 0, 0] = 0.2          # |0.5 - 0.2| = 0.3
    target[1, 2, 2] = 1.0          # |0.5 - 1.0| = 0.5
    A = torch.ones(3, 3, dtype=torch.float64)
    A[1, 2] = A_edge
    B = 2.0 * A                    # depth B / A = 2 everywhere
    D = 4.0 * A
    D[1, 1] = 4.5                  # centre: A D - B^2 = 4.5 - 4 = 0.5
    D[0, 2] = 4.09                 # corner: 4.09 - 4 = 0.09
    Nr = torch.zeros(3, 3, 3, dtype=torch.float64)
    Nr[1, 1] = torch.tensor([0.0, 0.0, -0.5], dtype=torch.float64)
    out = {"rgb": rgb, "A": A, "B": B, "D": D, "normal": Nr}
    return out, target, cam


def test_camera_loss_worked_example():
    """The camera loss on a 3x3 image worked by hand:
    L1 = (0.3 + 0.5) / 27 (mean over 3 H W);
    distortion = (0.5 + 0.09) / 9 (mean over the pixels of A D - B^2);
    normal term: only the centre pixel is interior.  Its four neighbours lie
    on the plane z = 2, so dX = X(2,1) - X(0,1) = (4, 0, 0),
    dY = X(1,2) - X(1,0) = (0, 4, 0), N_d = normalise(dY x dX) = (0, 0, -1),
    and 1 - N . N_d = 1 - 0.5 = 0.5, summed and divided by H W = 9.
    L = L1 + 0.1 distortion + 0.05 normal.  A sum in place of a mean, or a
    3 H W / H W slip, changes a term by a factor of 3, 9 or 27."""
    out, target, cam = _loss_example()
    L, parts = OG.loss(out, target, cam)
    assert float(parts["l1"]) == pytest.approx(0.8 / 27, rel=1e-14)
    assert float(parts["dist"]) == pytest.approx(0.59 / 9, rel=1e-14)
    assert float(parts["normal"]) == pytest.approx(0.5 / 9, rel=1e-14)
    assert float(L) == pytest.approx(0.8 / 27 + 0.1 * 0.59 / 9 + 0.05 * 0.5 / 9, rel=1e-14)
    # a neighbour with A below 0.5 masks the centre pixel's normal term
    out, target, cam = _loss_example(A_edge=0.4)
    L, parts = OG.loss(out, target, cam)
    assert float(parts["normal"]) == 0.0
    assert float(parts["dist"]) == pytest.approx((0.5 + 0.09 + (0.4 * 1.6 - 0.8 ** 2)) / 9, rel=1e-14)


def test_camera_loss_worked_example_gradients():
    """Gradients of the worked example in closed form: dL/drgb =
    sign(rgb - target) / 27; dL/dD = 0.1 A / 9; dL/dB = -0.1 2 B / 9 away
    from the pixels whose depth feeds the normal term; dL/dN at the centre =
    -0.05 N_d / 9."""
    out, target, cam = _loss_example()
    leaves = {k: v.clone().requires_grad_(True) for k, v in out.items()}
    L, _ = OG.loss(leaves, target, cam)
    L.backward()
    g = {k: v.grad for k, v in leaves.items()}
    want = torch.zeros(3, 3, 3, dtype=torch.float64)
    want[0, 0, 0] = 1.0 / 27
    want[1, 2, 2] = -1.0 / 27
    assert torch.allclose(g["rgb"], want, rtol=0, atol=1e-15)
    assert torch.allclose(g["D"], 0.1 * out["A"] / 9, rtol=1e-14, atol=0)
    # B also moves the back-projected depth B / A of the normal term; only
    # the centre's four neighbours enter it, so compare the other pixels
    far = torch.ones(3, 3, dtype=torch.bool)
    far[0, 1] = far[1, 0] = far[1, 2] = far[2, 1] = False
    assert torch.allclose(g["B"][far], (-0.1 * 2 * out["B"] / 9)[far], rtol=1e-14, atol=0)
    wantN = torch.zeros(3, 3, 3, dtype=torch.float64)
    wantN[1, 1] = torch.tensor([0.0, 0.0, 0.05 / 9], dtype=torch.float64)
    assert torch.allclose(g["normal"], wantN, rtol=1e-14, atol=1e-17)
