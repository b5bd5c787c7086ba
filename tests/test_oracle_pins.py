"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms of Eqs. 1-3/5 for simple geometry, an independent ray-plane
derivation of the Eq. 2 solution, quadrature of the SH basis, compositing
identities, and the LiDAR/pinhole special case.  A dropped term, a wrong sign
or a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle import grad as OG
from oracle import render as R
from paper_2503_11731_gb300 import synth


def _one(pos, log_scale, quat, opacity, rgb=(0.2, 0.5, 0.9), intensity=0.7):
    return synth.Surfels(np.asarray([pos], np.float64), np.asarray([log_scale], np.float64),
                         np.asarray([quat], np.float64), np.asarray([opacity], np.float64),
                         synth.rgb_to_sh0(np.asarray([rgb], np.float64), np.float64),
                         np.asarray([intensity], np.float64))


def _logit(p):
    return math.log(p / (1 - p))


def _cam(W=33, H=33, f=100.0, pose=None):
    return synth.Pinhole(W, H, f, f, W / 2.0, H / 2.0, np.eye(4) if pose is None else pose, 0.2)


# ---------------------------------------------------------------- SH basis
def test_sh_basis_orthonormal_by_quadrature():
    """Real SH to degree 3 are orthonormal on the sphere (Gauss-Legendre x uniform phi)."""
    xs, ws = np.polynomial.legendre.leggauss(24)
    phis = np.linspace(0, 2 * np.pi, 48, endpoint=False)
    dirs, wts = [], []
    for x, w in zip(xs, ws):
        st = math.sqrt(1 - x * x)
        for ph in phis:
            dirs.append((st * math.cos(ph), st * math.sin(ph), x))
            wts.append(w * 2 * np.pi / len(phis))
    lm = [(l, m) for l in range(4) for m in range(-l, l + 1)]
    Y = np.array([[R.sh_basis(l, m, d) for (l, m) in lm] for d in dirs])
    G = (Y * np.asarray(wts)[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-10


def test_sh_basis_low_orders_closed_form():
    d = np.array([0.3, -0.5, 0.81])
    d /= np.linalg.norm(d)
    x, y, z = d
    assert R.sh_basis(0, 0, d) == pytest.approx(0.5 / math.sqrt(math.pi), abs=1e-14)
    c1 = math.sqrt(3 / (4 * math.pi))
    assert R.sh_basis(1, 0, d) == pytest.approx(c1 * z, abs=1e-14)
    assert R.sh_basis(1, 1, d) == pytest.approx(-c1 * x, abs=1e-14)   # Condon-Shortley phase
    assert R.sh_basis(1, -1, d) == pytest.approx(-c1 * y, abs=1e-14)
    assert R.sh_basis(2, 0, d) == pytest.approx(math.sqrt(5 / (16 * math.pi)) * (3 * z * z - 1), abs=1e-13)
    assert R.sh_basis(2, -2, d) == pytest.approx(math.sqrt(15 / (4 * math.pi)) * x * y, abs=1e-13)


# ---------------------------------------------------- Eq. 2 intersection
def _rot(q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _ray_plane(o, d, mu, Rm, s):
    """Direct ray-plane intersection: x = o + t d with n.(x - mu) = 0."""
    n = Rm[:, 2]
    t = n @ (mu - o) / (n @ d)
    x = o + t * d
    return (Rm[:, 0] @ (x - mu)) / s[0], (Rm[:, 1] @ (x - mu)) / s[1], t, x


def test_eq2_pinhole_matches_direct_ray_plane():
    rng = np.random.default_rng(1)
    pose = synth.camera_pose((1.0, -2.0, 1.5), 20.0, -5.0, f32=False)
    Rc, tc = pose[:3, :3], pose[:3, 3]
    origin = -Rc.T @ tc
    cam = (500.0, 480.0, 320.0, 240.0)
    for _ in range(200):
        mu = origin + Rc.T @ np.array([rng.uniform(-3, 3), rng.uniform(-2, 2), rng.uniform(4, 30)])
        q = rng.standard_normal(4)
        ls = rng.uniform(-2, 0.5, 2)
        px, py = rng.uniform(0, 640), rng.uniform(0, 480)
        r = R.intersect(0, mu, ls, q, pose, cam, px, py)
        # camera ray through the pixel, in world coordinates
        dc = np.array([(px - cam[2]) / cam[0], (py - cam[3]) / cam[1], 1.0])
        d = Rc.T @ dc
        u, v, t, x = _ray_plane(origin, d, mu, _rot(q), np.exp(ls))
        depth = (Rc @ x + tc)[2]
        assert r is not None
        assert np.allclose(r, [u, v, depth], rtol=1e-9, atol=1e-9 * (1 + abs(u) + abs(v)))


def test_eq5_lidar_matches_direct_ray_plane():
    rng = np.random.default_rng(2)
    pose = synth.lidar_pose((0.3, 0.1, 1.8), 15.0, f32=False)
    Rl, tl = pose[:3, :3], pose[:3, 3]
    origin = -Rl.T @ tl
    for _ in range(200):
        az, el = rng.uniform(-np.pi, np.pi), rng.uniform(-0.5, 0.3)
        dl = np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        mu = origin + Rl.T @ (dl * rng.uniform(3, 40) + rng.normal(0, 0.3, 3))
        q = rng.standard_normal(4)
        ls = rng.uniform(-2, 0.5, 2)
        r = R.intersect(1, mu, ls, q, pose, (0, 0, 0, 0), az, el)
        u, v, t, _ = _ray_plane(origin, Rl.T @ dl, mu, _rot(q), np.exp(ls))
        assert r is not None
        assert np.allclose(r, [u, v, t], rtol=1e-9, atol=1e-9 * (1 + abs(u) + abs(v) + abs(t)))
        # both Eq. 5 planes contain the ray
        hu = np.array([math.sin(az), -math.cos(az), 0.0])
        hv = np.array([math.sin(el) * math.cos(az), math.sin(el) * math.sin(az), -math.cos(el)])
        assert abs(hu @ dl) < 1e-15 and abs(hv @ dl) < 1e-15


# ------------------------------------------------------ closed-form weights
def test_single_surfel_on_axis():
    """Facing surfel, pixel on its centre ray: u = v = 0, G = 1, alpha = min(0.99, o)."""
    cam = _cam()
    for o in (0.3, 0.999):
        s = _one((0, 0, 10), (0, 0), (1, 0, 0, 0), _logit(o))
        out = R.render_pinhole(s, cam, pixels=[16 * 33 + 16])
        a = min(0.99, o)
        assert out["rgb"][0] == pytest.approx(a * np.array([0.2, 0.5, 0.9]), abs=1e-12)
        assert out["depth"][0] == pytest.approx(10.0, abs=1e-12)
        assert out["T"][0] == pytest.approx(1 - a, abs=1e-12)
        # normal faces the camera: -z in the camera frame
        assert out["normal"][0] == pytest.approx([0, 0, -a], abs=1e-12)


def test_fronto_parallel_analytic_weight():
    """u = (X - mu_x)/s_u with X = (p_x - c_x) Z / f; G = exp(-(u^2+v^2)/2)."""
    cam = _cam(W=64, H=48, f=100.0)
    Z, su, sv, o = 8.0, 0.6, 0.3, 0.8
    s = _one((0.1, -0.05, Z), (math.log(su), math.log(sv)), (1, 0, 0, 0), _logit(o))
    out = R.render_pinhole(s, cam)
    ys, xs = np.mgrid[0:48, 0:64]
    X = (xs + 0.5 - 32.0) * Z / 100.0
    Y = (ys + 0.5 - 24.0) * Z / 100.0
    u, v = (X - 0.1) / su, (Y + 0.05) / sv
    rho3 = u * u + v * v
    cxp, cyp = 100 * 0.1 / Z + 32, 100 * -0.05 / Z + 24
    rholp = ((xs + 0.5 - cxp) ** 2 + (ys + 0.5 - cyp) ** 2) / 0.5
    rho = np.where(rho3 <= 9, np.where(rholp <= 9, np.minimum(rho3, rholp), rho3), np.where(rholp <= 9, rholp, np.inf))
    a = np.minimum(0.99, o * np.exp(-0.5 * rho))
    a = np.where(a >= 1 / 255, a, 0.0)
    assert np.abs(out["alpha"] - a).max() < 1e-12
    assert np.abs(out["rgb"][..., 1] - 0.5 * a).max() < 1e-12
    inside = a > 0
    # depth: the intersection depth of a fronto-parallel plane is Z everywhere
    assert np.abs(out["depth"][inside] - Z).max() < 1e-12


def test_edge_on_surfel_uses_low_pass_only():
    """Normal along x: the surfel plane x = 0 contains the camera centre, so
    every ray off that plane meets it only at depth 0 (< near); the low-pass
    exp(-|p-c|^2) (sigma^2 = 1/2 px^2) is all that is left.  The principal
    point is offset by 1/4 px so that no pixel centre lies in the plane."""
    cam = synth.Pinhole(33, 33, 100.0, 100.0, 16.75, 16.5, np.eye(4), 0.2)
    q = (math.cos(math.pi / 4), 0, math.sin(math.pi / 4), 0)  # 90 deg about y: normal -> +x
    o = 0.9
    s = _one((0, 0, 10), (-1, -1), q, _logit(o))
    out = R.render_pinhole(s, cam)
    ys, xs = np.mgrid[0:33, 0:33]
    d2 = (xs + 0.5 - 16.75) ** 2 + (ys + 0.5 - 16.5) ** 2
    a = np.where(d2 / 0.5 <= 9, np.minimum(0.99, o * np.exp(-d2)), 0.0)
    a = np.where(a >= 1 / 255, a, 0)
    assert a.max() > 0.5
    assert np.abs(out["alpha"] - a).max() < 1e-12
    # the low-pass contribution takes the centre depth
    assert np.abs(out["depth"][a > 0] - 10.0).max() < 1e-12


def test_two_surfels_composite_in_depth_order():
    cam = _cam()
    o1, o2 = 0.6, 0.7
    near = _one((0, 0, 5), (0, 0), (1, 0, 0, 0), _logit(o1), rgb=(1, 0, 0))
    far = _one((0, 0, 9), (0, 0), (1, 0, 0, 0), _logit(o2), rgb=(0, 0, 1))
    for s in (near.concat(far), far.concat(near)):
        out = R.render_pinhole(s, cam, pixels=[16 * 33 + 16])
        assert out["rgb"][0] == pytest.approx([o1, 0, (1 - o1) * o2], abs=1e-12)
        assert out["depth"][0] == pytest.approx((o1 * 5 + (1 - o1) * o2 * 9) / (o1 + (1 - o1) * o2), abs=1e-12)
        assert out["T"][0] == pytest.approx((1 - o1) * (1 - o2), abs=1e-12)


def test_alpha_skip_and_early_stop_rules():
    cam = _cam()
    pix = [16 * 33 + 16]
    # alpha just below 1/255 is skipped entirely
    s = _one((0, 0, 5), (0, 0), (1, 0, 0, 0), _logit(1 / 255 * 0.999))
    out = R.render_pinhole(s, cam, pixels=pix)
    assert out["alpha"][0] == 0.0 and out["T"][0] == 1.0
    s = _one((0, 0, 5), (0, 0), (1, 0, 0, 0), _logit(1 / 255 * 1.001))
    assert R.render_pinhole(s, cam, pixels=pix)["alpha"][0] > 0
    # a stack of alpha = 0.95: T 1 -> 0.05 -> 2.5e-3 -> 1.25e-4; the 4th would
    # leave 6.25e-6 < 1e-4, so compositing stops before it
    stack = None
    for k in range(6):
        t = _one((0, 0, 5 + k), (0, 0), (1, 0, 0, 0), _logit(0.95))
        stack = t if stack is None else stack.concat(t)
    out = R.render_pinhole(stack, cam, pixels=pix)
    assert out["n_contrib"][0] == 3
    assert out["T"][0] == pytest.approx(0.05 ** 3, rel=1e-12)


def test_opacity_zero_gives_background():
    s = synth.plain_scene(n=300, seed=5)
    s.opacity[:] = -60.0
    cam = synth.plain_camera(64, 40, 50.0)
    out = R.render_pinhole(s, cam, bg=(0.25, 0.5, 0.75))
    assert np.all(out["rgb"] == np.array([0.25, 0.5, 0.75]))
    assert np.all(out["T"] == 1.0) and np.all(out["alpha"] == 0.0)


def test_weights_plus_transmittance_is_one():
    s = synth.plain_scene(n=600, seed=6)
    cam = synth.plain_camera(64, 40, 50.0)
    out = R.render_pinhole(s, cam)
    assert np.abs(out["alpha"] + out["T"] - 1.0).max() < 1e-12
    assert out["alpha"].max() > 0.99  # the scene covers the image


def test_permutation_invariance_bit_exact():
    s = synth.plain_scene(n=500, seed=7)
    cam = synth.plain_camera(48, 32, 40.0)
    perm = np.random.default_rng(3).permutation(s.n)
    a = R.render_pinhole(s, cam)
    b = R.render_pinhole(s.subset(perm), cam)
    for k in ("rgb", "depth", "normal", "alpha", "T"):
        assert np.array_equal(a[k], b[k]), k


# ------------------------------------------------------------------- LiDAR
def test_lidar_fronto_plane_range_closed_form():
    """A big surfel facing the LiDAR at x = 10: range along ray = 10/(cos el cos az)."""
    lid = synth.Lidar(beams=21, columns=361, el_min_deg=-10, el_max_deg=10, world_to_sensor=np.eye(4))
    q = (math.cos(math.pi / 4), 0, math.sin(math.pi / 4), 0)  # normal -> +x
    o = 0.9
    s = _one((10, 0, 0), (math.log(2.0), math.log(2.0)), q, _logit(o), intensity=0.4)
    out = R.render_lidar(s, lid)
    Rm = _rot(q)
    for i in range(21):
        for j in range(361):
            el = math.radians(10 - i)
            az = math.radians(-180 + (j + 0.5) * 360.0 / 361)
            d = np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
            if d[0] <= 0:
                continue
            t = 10.0 / d[0]
            x = t * d
            u, v = Rm[:, 0] @ (x - [10, 0, 0]) / 2.0, Rm[:, 1] @ (x - [10, 0, 0]) / 2.0
            if u * u + v * v > 9:
                continue
            a = min(0.99, o * math.exp(-0.5 * (u * u + v * v)))
            assert out["range"][i, j] == pytest.approx(t, rel=1e-12)
            assert out["intensity"][i, j] == pytest.approx(0.4 * a, rel=1e-12)


def test_lidar_ray_drop_closed_form():
    """One surfel facing the LiDAR with drop probability rho: a ray through
    it returns drop = rho a + (1 - a) (its weight a, the rest escapes); a ray
    that misses every surfel is dropped (drop = 1)."""
    lid = synth.Lidar(beams=11, columns=181, el_min_deg=-5, el_max_deg=5, world_to_sensor=np.eye(4))
    q = (math.cos(math.pi / 4), 0, math.sin(math.pi / 4), 0)  # normal -> +x
    o, rho = 0.8, 0.3
    s = _one((10, 0, 0), (math.log(0.5), math.log(0.5)), q, _logit(o), intensity=0.4)
    s.ray_drop = np.asarray([_logit(rho)], np.float64)
    out = R.render_lidar(s, lid)
    Rm = _rot(q)
    hit = 0
    for i in range(11):
        for j in range(181):
            el = math.radians(5 - i)
            az = math.radians(-180 + (j + 0.5) * 360.0 / 181)
            d = np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
            a = 0.0
            if d[0] > 0:
                x = (10.0 / d[0]) * d
                u, v = Rm[:, 0] @ (x - [10, 0, 0]) / 0.5, Rm[:, 1] @ (x - [10, 0, 0]) / 0.5
                if u * u + v * v <= 9:
                    a = min(0.99, o * math.exp(-0.5 * (u * u + v * v)))
            if a < 1 / 255 and out["alpha"][i, j] == 0.0:
                assert out["drop"][i, j] == 1.0
                continue
            hit += 1
            assert out["drop"][i, j] == pytest.approx(rho * a + 1 - a, abs=1e-12)
    assert hit > 5


def test_lidar_ray_drop_identities():
    """rho = 1 everywhere: every ray is dropped (sum w + T = 1); rho = 0:
    drop = T; the drop attribute never changes range or intensity."""
    s = synth.driving_scene(n=3000, seed=9, x_range=(-10.0, 10.0), n_boxes=3)
    lid = synth.spinning_lidar(16, 180, -25.0, 10.0, (0.0, 0.0, 1.8))
    base = R.render_lidar(s, lid)
    s.ray_drop = np.full(s.n, 60.0, np.float64)
    one = R.render_lidar(s, lid)
    s.ray_drop = np.full(s.n, -60.0, np.float64)
    zero = R.render_lidar(s, lid)
    assert base["alpha"].max() > 0.9
    assert np.abs(one["drop"] - 1.0).max() < 1e-12
    assert np.abs(zero["drop"] - zero["T"]).max() < 1e-12
    assert np.all(base["drop"] == base["T"])
    for k in ("range", "intensity", "alpha", "T"):
        assert np.array_equal(base[k], one[k]) and np.array_equal(base[k], zero[k]), k


def test_lidar_centre_ray_equals_pinhole_centre_pixel():
    """The LiDAR ray at az = 0, el = 0 and a +x-looking pinhole's centre pixel
    are the same ray: same weights, range = depth."""
    rng = np.random.default_rng(4)
    n = 60
    pos = np.stack([rng.uniform(4, 20, n), rng.normal(0, 0.3, n), rng.normal(0, 0.3, n)], 1)
    # roughly fronto-facing (normal near +-x), large enough that G3 always beats the low-pass
    tilt = rng.uniform(-0.5, 0.5, (n, 2))
    qs = []
    for a, b in tilt:
        R1 = _rot((math.cos(math.pi / 4), 0, math.sin(math.pi / 4), 0))
        R2 = _rot((math.cos(a / 2), math.sin(a / 2), 0, 0)) @ _rot((math.cos(b / 2), 0, 0, math.sin(b / 2)))
        Rm = R2 @ R1
        qs.append(synth._quat_from_frame(Rm[:, 0][None], Rm[:, 1][None], Rm[:, 2][None])[0])
    q = np.asarray(qs, np.float64)
    ls = rng.uniform(-0.6, 0.0, (n, 2))
    op = rng.normal(0, 1, n)
    inten = rng.uniform(0, 1, n)
    s = synth.Surfels(pos, ls, q, op, synth.rgb_to_sh0(np.stack([inten] * 3, 1), np.float64), inten)
    lid = synth.Lidar(beams=21, columns=361, el_min_deg=-10, el_max_deg=10, world_to_sensor=np.eye(4))
    lo = R.render_lidar(s, lid, rays=[10 * 361 + 180])
    # camera looking +x: camera x = -y_world, camera y = -z_world, camera z = x_world
    pose = np.eye(4)
    pose[:3, :3] = [[0, -1, 0], [0, 0, -1], [1, 0, 0]]
    f = 1.0 / math.radians(1.0)
    cam = synth.Pinhole(33, 33, f, f, 16.5, 16.5, pose, 0.2)
    co = R.render_pinhole(s, cam, pixels=[16 * 33 + 16])
    assert lo["alpha"][0] > 0.5
    assert lo["alpha"][0] == pytest.approx(co["alpha"][0], abs=1e-12)
    assert lo["range"][0] == pytest.approx(co["depth"][0], rel=1e-12)
    assert lo["intensity"][0] == pytest.approx(co["rgb"][0][0], abs=1e-12)


def test_lidar_azimuth_wrap_low_pass():
    """An edge-on surfel straight behind the sensor (az = +-180 deg) reaches
    columns on both ends of the range image through the wrapped low-pass."""
    lid = synth.Lidar(beams=8, columns=360, el_min_deg=-7, el_max_deg=0, world_to_sensor=np.eye(4))
    # normal along z, centre on the -x axis at el 0 -> the surfel plane contains the rays of row 0
    s = _one((-10, 0, 0), (-3, -3), (1, 0, 0, 0), _logit(0.9), intensity=1.0)
    out = R.render_lidar(s, lid)
    # centre column coordinate: (180 - (-180))/1 - 0.5 = 359.5 -> columns 359 and 0 are 0.5 cells away
    a = 0.9 * math.exp(-0.25)
    assert out["intensity"][0, 0] == pytest.approx(a, rel=1e-9)
    assert out["intensity"][0, 359] == pytest.approx(a, rel=1e-9)
    assert out["intensity"][0, 180] == 0.0


# ---------------------------------------------------------- object placement
def test_object_pose_equals_pretransformed_surfels():
    """A rigid object pose (R_o, t_o) renders like surfels moved by hand, with
    the degree-1 SH coefficients rotated like a vector."""
    rng = np.random.default_rng(8)
    n = 80
    pos = rng.normal(0, 1.0, (n, 3))
    q = rng.standard_normal((n, 4))
    ls = rng.uniform(-2, -0.5, (n, 2))
    op = rng.normal(1, 1, n)
    sh = rng.normal(0, 0.3, (n, 4, 3))
    obj = synth.Surfels(pos, ls, q, op, sh, np.zeros(n), np.zeros(n, np.int32))
    yaw = 0.7
    Ro = np.array([[math.cos(yaw), -math.sin(yaw), 0], [math.sin(yaw), math.cos(yaw), 0], [0, 0, 1]])
    to = np.array([0.5, -0.3, 12.0])
    pose = np.concatenate([Ro, to[:, None]], 1)[None]
    cam = _cam(W=48, H=40, f=60.0)
    a = R.render_pinhole(obj, cam, obj_pose=pose)
    # by hand: mu' = R_o mu + t_o; R' = R_o R; SH l=1 coefficients (Y_1-1,Y_10,Y_11) ~ (-y, z, -x)
    Rm = np.stack([_rot(qq) for qq in q])
    Rn = np.einsum("ab,nbc->nac", Ro, Rm)
    qn = synth._quat_from_frame(Rn[:, :, 0], Rn[:, :, 1], Rn[:, :, 2]).astype(np.float64)
    shn = sh.copy()
    vec = np.stack([-sh[:, 3], -sh[:, 1], sh[:, 2]], 1)  # coefficient vector along (x, y, z)
    vec = np.einsum("ab,nbc->nac", Ro, vec)
    shn[:, 3], shn[:, 1], shn[:, 2] = -vec[:, 0], -vec[:, 1], vec[:, 2]
    moved = synth.Surfels(pos @ Ro.T + to, ls, qn, op, shn, np.zeros(n))
    b = R.render_pinhole(moved, cam)
    assert np.abs(a["rgb"] - b["rgb"]).max() < 1e-5  # quaternion round trip is float32
    assert np.abs(a["alpha"] - b["alpha"]).max() < 1e-5


# ------------------------------------------------------------ torch oracle
def test_torch_oracle_matches_c_oracle():
    """The FP64 tensor restatement used for gradients agrees with the C oracle."""
    s = synth.plain_scene(n=200, seed=9)
    s.sh = np.concatenate([s.sh, np.random.default_rng(1).normal(0, 0.2, (200, 15, 3))], 1).astype(np.float32)
    cam = synth.plain_camera(40, 32, 30.0)
    c = R.render_pinhole(s, cam, bg=(0.1, 0.2, 0.3))
    t = OG.render_pinhole(OG.surfel_tensors(s), cam, bg=(0.1, 0.2, 0.3))
    assert np.abs(t["rgb"].numpy() - c["rgb"]).max() < 1e-10
    assert np.abs(t["A"].numpy() - c["acc"][..., 0]).max() < 1e-10
    assert np.abs(t["B"].numpy() - c["acc"][..., 1]).max() < 1e-8
    assert np.abs(t["D"].numpy() - c["acc"][..., 2]).max() < 1e-7
    assert np.abs(t["normal"].numpy() - c["normal"]).max() < 1e-10
    assert np.array_equal(t["n_contrib"].numpy(), c["n_contrib"])


def test_distortion_identity():
    """A D - B^2 = 1/2 sum_ij w_i w_j (z_i - z_j)^2 (the pairwise definition)."""
    rng = np.random.default_rng(10)
    w = rng.uniform(0, 0.3, 12)
    z = rng.uniform(2, 30, 12)
    pair = 0.5 * sum(w[i] * w[j] * (z[i] - z[j]) ** 2 for i in range(12) for j in range(12))
    A, B, D = w.sum(), (w * z).sum(), (w * z * z).sum()
    assert A * D - B * B == pytest.approx(pair, rel=1e-12)


# ------------------------------------------------- cylindrical camera (Eq. 4)
def test_eq4_cylinder_matches_direct_ray_plane():
    """(u, v) and the depth (the horizontal distance along the cylinder ray)
    equal a direct intersection of the ray d = (sin phi, y_n, cos phi) from
    the camera centre with the surfel plane."""
    rng = np.random.default_rng(12)
    pose = synth.camera_pose((0.5, 1.0, 1.6), 35.0, 3.0, f32=False)
    Rc, tc = pose[:3, :3], pose[:3, 3]
    origin = -Rc.T @ tc
    cam = (300.0, 280.0, 400.0, 120.0)
    for _ in range(200):
        phi, yn = rng.uniform(-2.5, 2.5), rng.uniform(-0.6, 0.6)
        dc = np.array([math.sin(phi), yn, math.cos(phi)])
        mu = origin + Rc.T @ (dc * rng.uniform(3, 30) + rng.normal(0, 0.4, 3))
        q = rng.standard_normal(4)
        ls = rng.uniform(-2, 0.5, 2)
        r = R.intersect(2, mu, ls, q, pose, cam, phi, yn)
        u, v, t, x = _ray_plane(origin, Rc.T @ dc, mu, _rot(q), np.exp(ls))
        xc = Rc @ x + tc
        assert r is not None
        assert np.allclose(r, [u, v, math.hypot(xc[0], xc[2]) * np.sign(t)], rtol=1e-9,
                           atol=1e-9 * (1 + abs(u) + abs(v) + abs(t)))
        assert t == pytest.approx(r[2], rel=1e-9)  # |(sin phi, cos phi)| = 1: the ray parameter is the depth


def test_cylinder_centre_column_equals_pinhole_column():
    """The cylinder column at azimuth 0 and the pinhole column through its
    principal point carry the same rays (0, y_n, 1); for surfels centred on
    the camera's x = 0 plane the low-pass centres coincide too, so the whole
    column renders identically (depth = horizontal distance = z there)."""
    rng = np.random.default_rng(13)
    n = 80
    pos = np.stack([np.zeros(n), rng.uniform(-2, 2, n), rng.uniform(4, 25, n)], 1)
    q = rng.standard_normal((n, 4))
    ls = rng.uniform(-2.0, -0.3, (n, 2))
    op = rng.normal(0.5, 1, n)
    s = synth.Surfels(pos, ls, q, op, synth.rgb_to_sh0(rng.uniform(0, 1, (n, 3)), np.float64),
                      rng.uniform(0, 1, n))
    W, H, fy = 41, 48, 60.0
    cyl = synth.Cylindrical(W, H, 25.0, fy, 20.5, 24.0, np.eye(4), 0.2)   # column 20 at phi = 0
    pin = synth.Pinhole(W, H, 77.0, fy, 20.5, 24.0, np.eye(4), 0.2)
    col = [y * W + 20 for y in range(H)]
    oc = R.render_pinhole(s, cyl, pixels=col)
    op_ = R.render_pinhole(s, pin, pixels=col)
    assert oc["alpha"].max() > 0.3
    for k in ("rgb", "alpha", "T", "normal"):
        assert np.abs(oc[k] - op_[k]).max() <= 1e-12, k
    assert np.abs(oc["depth"] - op_["depth"]).max() <= 1e-9
    # and away from that column the two projections differ
    other = [y * W + 3 for y in range(H)]
    assert np.abs(R.render_pinhole(s, cyl, pixels=other)["alpha"] -
                  R.render_pinhole(s, pin, pixels=other)["alpha"]).max() > 1e-3


# ------------------------------------------------------------------- zones
def test_zone_membership_geometry():
    """3 x 3 zones of 40 m from the origin with 25 % padding: a zone core
    point belongs to its zone only, a point in one padding band to two, near
    a corner to four, beyond the outer padding to none."""
    from oracle import zones as OZ
    g = {"x0": 0.0, "y0": 0.0, "zone_size": 40.0, "padding": 0.25, "nx": 3, "ny": 3}
    pos = np.array([[60.0, 60.0, 0.0],    # core of zone (1, 1) = 4
                    [41.0, 60.0, 0.0],    # x in zones 0 ([-10, 50)) and 1 ([30, 90))
                    [45.0, 45.0, 0.0],    # both axes in two zones
                    [-20.0, 60.0, 0.0],   # x below -10: no zone
                    [129.9, 5.0, 0.0]])   # x in zone 2 ([70, 130)), y in zone 0
    m = OZ.members(g, pos)
    sets = [sorted(z for z in range(9) if k in m[z]) for k in range(len(pos))]
    assert sets == [[4], [3, 4], [0, 1, 3, 4], [], [2]]
    assert OZ.zone_of(g, 60.0, 60.0) == 4 and OZ.zone_of(g, 41.0, 60.0) == 4 and OZ.zone_of(g, -1.0, 5.0) == -1


# ------------------------------------------------- tiled mode = brute force
def _near_plane_scene(seed):
    """Plain scene with a fifth of the surfels pulled to centre depths around
    the near plane (0.2 m), some of them within rounding of it."""
    s = synth.plain_scene(n=1500, seed=seed)
    rng = np.random.default_rng(seed)
    pos = s.pos.astype(np.float64)
    k = rng.choice(s.n, s.n // 5, replace=False)
    pos[k, 2] = rng.uniform(0.05, 1.5, len(k))
    pos[k[:8], 2] = 0.2 * (1 + rng.choice([-1, 1], 8) * 1e-7)
    pos[k, :2] *= 0.05
    return synth.Surfels(pos, s.log_scale.astype(np.float64), s.quat.astype(np.float64),
                         s.opacity.astype(np.float64), s.sh.astype(np.float64), s.intensity.astype(np.float64))


def _tiled_cases():
    plain = synth.plain_scene(n=2000, seed=3)
    drive = synth.driving_scene(n=6000, seed=11, x_range=(-20.0, 30.0), n_boxes=4)
    obj = synth.object_asset(n=3000, seed=4)
    obj.obj_id = np.zeros(obj.n, np.int32) + (np.arange(obj.n) % 2).astype(np.int32)
    poses = synth.object_poses(2, seed=8, x_range=(6.0, 14.0))
    rng = np.random.default_rng(12)
    n = 1500
    ang = rng.uniform(np.pi - 0.3, np.pi + 0.3, n)
    dist = rng.uniform(0.5, 12.0, n)
    seam = synth.Surfels(np.stack([dist * np.cos(ang), dist * np.sin(ang), rng.uniform(-1.5, 1.5, n)], 1),
                         rng.uniform(-3, 0, (n, 2)), synth._unit_quats(rng, n).astype(np.float64),
                         rng.normal(0, 1, n), rng.normal(0, 0.2, (n, 1, 3)), rng.uniform(0, 1, n))
    return [
        ("pinhole plain", plain, synth.plain_camera(96, 64, 80.0), None),
        ("pinhole near plane", _near_plane_scene(5), synth.plain_camera(80, 56, 60.0), None),
        ("pinhole posed objects", obj, synth.pinhole(72, 40, 60.0, (0.0, 0.5, 1.2), yaw_deg=4.0), poses),
        ("cylinder 240 deg", drive, synth.cylindrical(120, 40, 240.0, 50.0, (0.0, 0.0, 1.5), pitch_deg=-6.0), None),
        ("lidar drive", drive, synth.spinning_lidar(16, 180, -25.0, 15.0, (0.0, 0.0, 1.8)), None),
        ("lidar seam", seam, synth.spinning_lidar(12, 150, -20.0, 20.0, (0.0, 0.0, 0.0)), None),
        ("lidar posed objects", obj, synth.spinning_lidar(10, 200, -20.0, 10.0, (0.0, 0.0, 1.8)), poses),
    ]


@pytest.mark.parametrize("case", range(7))
def test_tiled_mode_equals_brute_force(case):
    """Per-tile candidate lists from the oracle's own conservative bound give
    bit-identical outputs (flip values and contributor counts included) to
    checking every surfel for every ray, at several tile sizes: the bound
    misses no surfel that any ray of its tiles could see."""
    name, s, sensor, poses = _tiled_cases()[case]
    render = R.render_lidar if sensor.kind == "lidar" else R.render_pinhole
    brute = render(s, sensor, obj_pose=poses)
    assert brute["alpha"].max() > 0.5, name
    for tile in (4, 8, 16):
        tiled = render(s, sensor, obj_pose=poses, tile=tile)
        for k in brute:
            assert np.array_equal(brute[k], tiled[k]), (name, tile, k)


# ----------------------------------------------- FP32-flippable decisions
def test_order_near_tie_slack():
    """Two facing surfels on the optical axis.  Depths 1 mm apart: composited
    in depth order, no slack.  Depths 1e-7 m apart (below what an FP32
    evaluation of a 10 m depth resolves): still composited in FP64 depth
    order, and the ray's slack is the exact change a swap makes, the weight
    o1 o2 moved between colours that differ by 1 in red and blue (and the
    depth accumulator's o1 o2 dz)."""
    cam = _cam()
    pix = [16 * 33 + 16]
    o1, o2 = 0.6, 0.7
    for dz, tied in ((1e-3, False), (1e-7, True)):
        a = _one((0, 0, 10.0), (0, 0), (1, 0, 0, 0), _logit(o1), rgb=(1, 0, 0))
        b = _one((0, 0, 10.0 + dz), (0, 0), (1, 0, 0, 0), _logit(o2), rgb=(0, 0, 1))
        for s in (a.concat(b), b.concat(a)):
            out = R.render_pinhole(s, cam, pixels=pix)
            assert out["rgb"][0] == pytest.approx([o1, 0, (1 - o1) * o2], abs=1e-12)
            assert out["flip"][0] == 0.0
            if tied:
                assert out["slack"][0] == pytest.approx(o1 * o2 * 1.0, rel=1e-9)
                assert out["slack_z"][0] == pytest.approx(o1 * o2 * dz, rel=1e-6)
                # the swapped order differs from the FP64 order by exactly the slack
                swapped = [o2 * (1 - o1), 0, o2]
                assert np.abs(np.array(swapped) - out["rgb"][0]).max() == pytest.approx(out["slack"][0], rel=1e-9)
            else:
                assert out["slack"][0] == 0.0 and out["slack_z"][0] == 0.0
    # a run of three tied surfels: any order keeps the run's weight
    # W = 1 - (1 - o)^3 and T; each output stays within W times the run's
    # range of it (red 1 / 0 / 0 here: slack W)
    o = 0.5
    run = None
    for k, c in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
        t = _one((0, 0, 10.0 + 4e-7 * k), (0, 0), (1, 0, 0, 0), _logit(o), rgb=c)
        run = t if run is None else run.concat(t)
    out = R.render_pinhole(run, cam, pixels=pix)
    W = 1 - (1 - o) ** 3
    assert out["slack"][0] == pytest.approx(W, rel=1e-9)
    assert out["slack_z"][0] == pytest.approx(W * 8e-7, rel=1e-6)
    import itertools
    base = out["rgb"][0]
    for perm in itertools.permutations(range(3)):
        # every order of the run lies within the slack of the FP64 order
        cols = [((1, 0, 0), (0, 1, 0), (0, 0, 1))[p] for p in perm]
        T, rgb = 1.0, np.zeros(3)
        for c in cols:
            rgb += o * T * np.array(c)
            T *= 1 - o
        assert np.abs(rgb - base).max() <= out["slack"][0] + 1e-12
    # equal colours and normals: a swap changes no colour
    a = _one((0, 0, 10.0), (0, 0), (1, 0, 0, 0), _logit(o1))
    b = _one((0, 0, 10.0 + 1e-7), (0, 0), (1, 0, 0, 0), _logit(o2))
    out = R.render_pinhole(a.concat(b), cam, pixels=pix)
    assert out["slack"][0] == 0.0 and out["slack_z"][0] > 0.0
    # a tie at the stop (the second surfel would end the ray) is a flag: the
    # swapped order composites the other surfel instead; the flag carries the
    # weight at stake, T before the tied run (0.03 here) times the largest
    # value (1)
    stack = None
    for k in range(3):
        t = _one((0, 0, 5.0 + k), (0, 0), (1, 0, 0, 0), _logit(0.97), rgb=(1, 0, 0))
        stack = t if stack is None else stack.concat(t)
    # T after three surfels of 0.97: 2.7e-5 < 1e-4, so the third stops the
    # ray; put a blue surfel within 1e-8 m of the second
    blue = _one((0, 0, 6.0 + 1e-8), (0, 0), (1, 0, 0, 0), _logit(0.97), rgb=(0, 0, 1))
    out = R.render_pinhole(stack.concat(blue), cam, pixels=pix)
    assert out["n_contrib"][0] == 2 and out["flip"][0] == pytest.approx(0.03, rel=1e-6)


def test_near_cull_within_rounding_is_flagged():
    """A surfel tilted 60 degrees about x whose centre depth sits within
    rounding of the near plane (0.2 m), seen by pixels whose rays meet it
    0.03-0.1 m beyond the centre: just in front it is composited, just
    behind it is culled; either way the rays it reaches are flagged with the
    weight it has (or would have)."""
    cam = _cam(W=65, H=65, f=40.0)
    q = (math.cos(math.pi / 6), math.sin(math.pi / 6), 0, 0)
    res = {}
    for sign in (1, -1):
        z = 0.2 * (1 + sign * 1e-7)
        s = _one((0, 0, z), (math.log(0.05), math.log(0.05)), q, _logit(0.9))
        res[sign] = R.render_pinhole(s, cam)
    seen = res[1]["alpha"] > 0
    assert seen.sum() > 20
    assert np.array_equal(res[1]["flip"][seen], res[1]["alpha"][seen])
    assert np.all(res[-1]["alpha"] == 0.0)
    # the two centres differ by 4e-8 m, so the weights agree to about that
    assert np.abs(res[-1]["flip"] - res[1]["flip"]).max() < 1e-6
    assert np.array_equal(res[-1]["flip"] > 0, res[1]["flip"] > 0)
    # a centre 1 % in front of the near plane raises no flag
    s = _one((0, 0, 0.202), (math.log(0.05), math.log(0.05)), q, _logit(0.9))
    far = R.render_pinhole(s, cam)
    assert far["alpha"].max() > 0.5
    on = far["alpha"] > 0
    assert np.all(far["flip"][on] < far["alpha"][on])


def test_identical_key_operands_are_not_a_tie():
    """Two unposed surfels at the same depth z (the identity camera's key
    takes only z) with different x: their FP32 keys are equal whatever the
    evaluation order, so both sides order them by index -- no slack, and the
    lower index composites first.  The same pair one FP32 step apart in depth
    is a near tie and carries the swap's slack."""
    cam = _cam(W=65, H=65, f=40.0)
    pix = [32 * 65 + 32]
    o1, o2 = 0.6, 0.7
    step = float(np.nextafter(np.float32(10.0), np.float32(20.0))) - 10.0
    for dz, tied in ((0.0, False), (step, True)):
        # positions exactly representable in FP32, as a table handed to both sides is
        a = _one((0.015625, 0, 10.0), (0, 0), (1, 0, 0, 0), _logit(o1), rgb=(1, 0, 0))
        b = _one((-0.015625, 0, 10.0 + dz), (0, 0), (1, 0, 0, 0), _logit(o2), rgb=(0, 0, 1))
        out = R.render_pinhole(a.concat(b), cam, pixels=pix)
        assert (out["slack"][0] > 0) == tied
        if not tied:
            # index order: a (index 0) first
            ga, gb = out["rgb"][0][0] / 1.0, out["rgb"][0][2]
            assert ga > gb
            out2 = R.render_pinhole(b.concat(a), cam, pixels=pix)
            assert out2["rgb"][0][2] > out2["rgb"][0][0]  # now b composites first


def test_near_tie_past_the_stop_is_slack():
    """Three red surfels of opacity 0.97 at 5, 6 and 7 m on the optical
    axis: the third ends the ray (T would fall to 2.7e-5 < 1e-4), with
    T = 9e-4 before it.  A blue surfel of opacity 0.5 within 1e-8 m behind
    the third comes after the stop in FP64 order, but an FP32 sort may put
    it first: it then composites 0.5 * 9e-4 of blue, and as much alpha,
    before the third still ends the ray.  That bounded change is the ray's
    slack of every output (slack_c), not a flag; the same surfel 1 mm
    behind is no tie and adds none.  Brute force and the tiled walk agree
    bit for bit."""
    cam = _cam()
    pix = [16 * 33 + 16]
    stack = None
    for k in range(3):
        t = _one((0, 0, 5.0 + k), (0, 0), (1, 0, 0, 0), _logit(0.97), rgb=(1, 0, 0))
        stack = t if stack is None else stack.concat(t)
    T_stop = 0.03 ** 2
    for dz, tied in ((1e-8, True), (1e-3, False)):
        blue = _one((0, 0, 7.0 + dz), (0, 0), (1, 0, 0, 0), _logit(0.5), rgb=(0, 0, 1))
        s = stack.concat(blue)
        out = R.render_pinhole(s, cam, pixels=pix)
        assert out["n_contrib"][0] == 2 and out["flip"][0] == 0.0
        assert out["rgb"][0][2] == pytest.approx(0.0, abs=1e-12)
        if tied:
            assert out["slack_c"][0] == pytest.approx(0.5 * T_stop, rel=1e-6)
            # the swapped order: blue at T_stop, then the third red stops the ray
            T, rgb, A = 1.0, np.zeros(3), 0.0
            for a, c in ((0.97, (1, 0, 0)), (0.97, (1, 0, 0)), (0.5, (0, 0, 1)), (0.97, (1, 0, 0))):
                if T * (1 - a) < 1e-4:
                    break
                rgb += a * T * np.array(c)
                A += a * T
                T *= 1 - a
            assert np.abs(rgb - out["rgb"][0]).max() == pytest.approx(out["slack_c"][0], rel=1e-6)
            assert abs(A - out["alpha"][0]) == pytest.approx(out["slack_c"][0], rel=1e-6)
        else:
            assert out["slack_c"][0] == 0.0
        for tile in (4, 16):
            tiled = R.render_pinhole(s, cam, pixels=pix, tile=tile)
            for k in out:
                assert np.array_equal(out[k], tiled[k]), (dz, tile, k)


def test_low_pass_centre_reach_flags_alpha_threshold():
    """A sub-cell surfel seen by a 1024-column LiDAR only through the
    low-pass fallback: its centre sits at cell (598 + 2^-15, 15.25), so the
    ray of cell (600, 15) has rho_lp = 2 (dx^2 + dy^2) = 8.12.  The centre's
    column is half an FP32 ulp off a representable value: rounding it to
    FP32 alone moves rho_lp by 4 dx 2^-15 = 2.4e-4, and alpha = o exp(-rho_lp
    / 2) by 1.2e-4 relative, six times the flat 2e-5 margin.  With its
    opacity set so that alpha sits 4e-5 (relative) below 1/255, the oracle
    flags the ray with the weight at stake (T / 255 = 1/255); at 5e-3 below,
    beyond the centre's reach, it does not.  Brute force and tiled agree."""
    lid = synth.Lidar(32, 1024, -30.0, 10.0, np.eye(4), -180.0, 0.2)
    d_az = 2 * math.pi / 1024
    d_el = math.radians(40.0) / 31
    h = 2.0 ** -15
    c0, c1 = 598.0 + h, 15.25
    az = math.radians(-180.0) + (c0 + 0.5) * d_az
    el = math.radians(10.0) - c1 * d_el
    rng_ = 9.0
    pos = (rng_ * math.cos(el) * math.cos(az), rng_ * math.cos(el) * math.sin(az), rng_ * math.sin(el))
    dx, dy = 600 - c0, 15 - c1
    rho = 2 * (dx * dx + dy * dy)
    assert rho < 9
    # what FP32 rounding of the centre's column alone does to alpha
    dx32 = 600 - float(np.float32(c0))
    rel = abs(math.exp(-(dx32 * dx32 + dy * dy)) / math.exp(-0.5 * rho) - 1)
    assert rel > 5 * 2e-5
    ray = 15 * 1024 + 600
    for delta, flagged in ((4e-5, True), (5e-3, False)):
        o = (1 - delta) / 255 / math.exp(-0.5 * rho)
        s = _one(pos, (math.log(1e-3), math.log(1e-3)), (1, 0, 0, 0), _logit(o))
        out = R.render_lidar(s, lid, rays=[ray])
        assert out["alpha"][0] == 0.0            # below 1/255 in FP64: skipped
        if flagged:
            assert out["flip"][0] == pytest.approx(1 / 255, rel=1e-9)
        else:
            assert out["flip"][0] == 0.0
        for tile in (4, 8):
            tiled = R.render_lidar(s, lid, rays=[ray], tile=tile)
            for k in out:
                assert np.array_equal(out[k], tiled[k]), (delta, tile, k)


def test_low_pass_centre_reach_camera_column_1900():
    """The same for a camera: a sub-pixel surfel 10 m ahead whose projected
    centre sits at pixel x = 1900 + 2^-14 (half an FP32 ulp there), seen by
    the pixel whose centre is (1901.5, 500.5) only through the low-pass
    disc.  Rounding the centre's column to FP32 moves rho_lp by about
    4 dx 2^-14 = 3.7e-4 and alpha by 1.8e-4 relative; with alpha 4e-5 below
    1/255 the ray is flagged, at 5e-3 below it is not."""
    W, H, f = 2048, 1024, 1000.0
    cam = _cam(W=W, H=H, f=f)
    h = 2.0 ** -14
    c0, c1 = 1900.0 + h, 500.25
    Z = 10.0
    pos = ((c0 - W / 2.0) * Z / f, (c1 - H / 2.0) * Z / f, Z)
    px, py = 1901, 500
    dx, dy = px + 0.5 - c0, py + 0.5 - c1
    rho = 2 * (dx * dx + dy * dy)
    assert rho < 9
    dx32 = px + 0.5 - float(np.float32(c0))
    rel = abs(math.exp(-(dx32 * dx32 + dy * dy)) / math.exp(-0.5 * rho) - 1)
    assert rel > 5 * 2e-5
    pix = [py * W + px]
    for delta, flagged in ((4e-5, True), (5e-3, False)):
        o = (1 - delta) / 255 / math.exp(-0.5 * rho)
        s = _one(pos, (math.log(1e-4), math.log(1e-4)), (1, 0, 0, 0), _logit(o))
        out = R.render_pinhole(s, cam, pixels=pix)
        assert out["alpha"][0] == 0.0
        if flagged:
            assert out["flip"][0] == pytest.approx(1 / 255, rel=1e-9)
        else:
            assert out["flip"][0] == 0.0
        tiled = R.render_pinhole(s, cam, pixels=pix, tile=16)
        for k in out:
            assert np.array_equal(out[k], tiled[k]), (delta, k)
