"""GPU parity of the cylindrical (fisheye) camera of Eq. 4 against the FP64
oracle, through the C ABI: full frames with surfels at every azimuth (behind
the camera, straddling the +-180 deg seam of a full panorama, and above the
camera where the horizontal distance is small), and a sampled frame of the
1.5M-surfel driving scene.  Tolerances as for the pinhole: RGB, alpha,
normal 1e-4 absolute; depth (horizontal distance) 1e-4 relative."""
import numpy as np
import pytest

from oracle import render as OR
from paper_2503_11731_gb300 import synth

from test_gpu_forward import _check_camera, _render

pytestmark = pytest.mark.gpu


def _ring_scene(n, seed, r=(1.5, 30.0), height=(-4.0, 4.0), n_pole=0):
    """Surfels around a camera at the origin (camera frame: y down), all
    azimuths; `n_pole` of them sit over the camera at small horizontal
    distance.  SH degree 1 so the view direction matters."""
    rng = np.random.default_rng(seed)
    m = n - n_pole
    ang = rng.uniform(-np.pi, np.pi, m)
    dist = rng.uniform(r[0], r[1], m)
    pos = np.stack([dist * np.sin(ang), rng.uniform(height[0], height[1], m), dist * np.cos(ang)], 1)
    if n_pole:
        pole = np.stack([rng.uniform(-0.6, 0.6, n_pole), rng.uniform(-4.0, -1.0, n_pole),
                         rng.uniform(-0.6, 0.6, n_pole)], 1)
        pos = np.concatenate([pos, pole], 0)
    return synth.Surfels(pos.astype(np.float32), rng.uniform(-3, 0, (n, 2)).astype(np.float32),
                         synth._unit_quats(rng, n), rng.normal(0, 1, n).astype(np.float32),
                         rng.normal(0, 0.3, (n, 4, 3)).astype(np.float32), rng.uniform(0, 1, n).astype(np.float32))


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_cylindrical_full_frame_parity(gpu_lib, tile):
    """390x123 (ragged), 220 deg horizontal field; every pixel."""
    s = _ring_scene(6000, seed=31, n_pole=300)
    cam = synth.cylindrical(390, 123, 220.0, 70.0, pose=np.eye(4))
    r, out = _render(s, [cam], tile=tile, bg=(0.1, 0.2, 0.3))
    st, nvis, npairs = r.status()
    assert st == 0 and nvis > 0 and npairs > 0
    o = OR.render_pinhole(s, cam, bg=(0.1, 0.2, 0.3))
    _check_camera(out[0], o, max_flag=0.003)  # measured 0.14 %


def test_cylindrical_panorama_seam(gpu_lib):
    """A full 360 deg panorama with close surfels straddling the seam behind
    the camera (azimuth +-180 deg): the image does not wrap, both ends see
    their own part of each surfel."""
    rng = np.random.default_rng(32)
    s = _ring_scene(3000, seed=33, r=(0.8, 12.0))
    k = 1500
    ang = rng.uniform(np.pi - 0.15, np.pi + 0.15, k)
    dist = rng.uniform(0.6, 6.0, k)
    s.pos[:k] = np.stack([dist * np.sin(ang), rng.uniform(-1.5, 1.5, k), dist * np.cos(ang)], 1)
    cam = synth.cylindrical(360, 96, 360.0, 60.0, pose=np.eye(4))
    r, out = _render(s, [cam], tile=(16, 8), max_dup=1 << 21)
    assert r.status()[0] == 0
    o = OR.render_pinhole(s, cam)
    _check_camera(out[0], o, max_flag=0.003)  # measured 0.12 %
    # both ends of the image are covered
    a = out[0]["alpha"]
    assert a[:, :4].max() > 0.5 and a[:, -4:].max() > 0.5


def test_cylindrical_posed_driving_scene_sampled(gpu_lib):
    """1.5M-surfel driving scene (SH degree 3), a 2880x720 surround camera
    (200 deg) beside a pinhole and a LiDAR in one plan; 4,096 sampled
    pixels against the oracle (tiled mode)."""
    s = synth.driving_scene()
    cyl = synth.cylindrical(2880, 720, 200.0, 70.0, (0.0, 0.0, 1.6), yaw_deg=0.0)
    sensors = [synth.driving_camera(), cyl, synth.driving_lidar()]
    r, out = _render(s, sensors)
    st, nvis, npairs = r.status()
    assert st == 0, st
    rng = np.random.default_rng(34)
    pix = rng.choice(2880 * 720, 4096, replace=False)
    o = OR.render_pinhole(s, cyl, pixels=pix, tile=16)
    _check_camera(out[1], o, pix=pix, max_flag=0.025)  # measured 1.54 %
