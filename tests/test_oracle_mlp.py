"""Pins of the anchor-MLP decode oracle (oracle/mlp.py) against facts fixed
by its definition: biases pass through a zero network, a single active
hidden unit gives a closed form, the view inputs are a unit direction and a
distance, and the frustum cull keeps/drops anchors by plain geometry."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp as OM
from paper_2503_11731_gb300 import synth


def _anchors(n=5, k=10, seed=3):
    rng = np.random.default_rng(seed)
    return synth.Anchors(rng.normal(0, 5, (n, 3)) + [0, 0, 20], rng.normal(0, 1, (n, 32)),
                         rng.uniform(0.5, 2.0, n), rng.normal(0, 0.5, (n, k, 3)), rng.uniform(0, 1, (n, k)))


def test_zero_network_passes_biases():
    a = _anchors()
    b2 = np.random.default_rng(1).normal(0, 1, 100)
    out = OM.decode(a, np.zeros((36, 64)), np.zeros(64), np.zeros((64, 100)), b2, (0, 0, 0))
    y = b2.reshape(10, 10)
    sig = 1 / (1 + np.exp(-y[:, 1:4]))
    for i in range(a.n):
        s = slice(10 * i, 10 * i + 10)
        assert np.allclose(out["opacity"][s].numpy(), y[:, 0])
        assert np.allclose(out["rgb"][s].numpy(), sig)
        assert np.allclose(out["log_scale"][s].numpy(), y[:, 4:6] + math.log(a.scale[i]))
        assert np.allclose(out["quat"][s].numpy(), y[:, 6:10])
        assert np.allclose(out["pos"][s].numpy(), a.pos[i] + a.scale[i] * a.offsets[i])
        # degree-0 SH reproduces the colour: 0.5 + Y00 c0 = rgb
        assert np.allclose(0.5 + OM.Y00 * out["sh"][s, 0].numpy(), sig)


def test_lidar_head_zero_network_passes_biases():
    """LiDAR head: opacity y0, intensity sigmoid(y1), ray-drop logit y2, y3
    unused, log-scales y4..5 + ln l_a, quaternion y6..9; no colour."""
    a = _anchors()
    b2 = np.random.default_rng(2).normal(0, 1, 100)
    out = OM.decode(a, np.zeros((36, 64)), np.zeros(64), np.zeros((64, 100)), b2, (0, 0, 0), head="lidar")
    y = b2.reshape(10, 10)
    for i in range(a.n):
        s = slice(10 * i, 10 * i + 10)
        assert np.allclose(out["opacity"][s].numpy(), y[:, 0])
        assert np.allclose(out["intensity"][s].numpy(), 1 / (1 + np.exp(-y[:, 1])))
        assert np.allclose(out["ray_drop"][s].numpy(), y[:, 2])
        assert np.allclose(out["log_scale"][s].numpy(), y[:, 4:6] + math.log(a.scale[i]))
        assert np.allclose(out["quat"][s].numpy(), y[:, 6:10])
        assert np.all(out["sh"][s].numpy() == 0.0)
    # the unused output y3 does not reach any attribute
    b3 = b2.copy()
    b3[3::10] += 5.0
    o3 = OM.decode(a, np.zeros((36, 64)), np.zeros(64), np.zeros((64, 100)), b3, (0, 0, 0), head="lidar")
    for k in ("opacity", "intensity", "ray_drop", "log_scale", "quat", "pos"):
        assert torch.equal(out[k], o3[k]), k


def test_single_hidden_unit_closed_form():
    a = _anchors(n=3)
    W1 = np.zeros((36, 64))
    W1[0, 5] = 2.0          # hidden 5 = relu(2 f0 + 0.5)
    W1[35, 5] = 0.0
    b1 = np.zeros(64)
    b1[5] = 0.5
    W2 = np.zeros((64, 100))
    W2[5, 30] = 1.5         # offset 3, opacity logit
    out = OM.decode(a, W1, b1, W2, np.zeros(100), (0, 0, 0))
    for i in range(a.n):
        h = max(0.0, 2 * a.feature[i, 0] + 0.5)
        assert out["opacity"][10 * i + 3].item() == pytest.approx(1.5 * h, abs=1e-12)
        assert out["opacity"][10 * i + 2].item() == 0.0


def test_view_inputs_are_direction_and_distance():
    a = _anchors(n=4)
    origin = np.array([1.0, -2.0, 0.5])
    out = OM.decode(a, np.zeros((36, 64)), np.zeros(64), np.zeros((64, 100)), np.zeros(100), origin)
    X = out["X"].numpy()
    v = a.pos - origin
    assert np.allclose(X[:, :32], a.feature)
    assert np.allclose(X[:, 35], np.linalg.norm(v, axis=1))
    assert np.allclose(X[:, 32:35], v / np.linalg.norm(v, axis=1, keepdims=True))


def test_frustum_cull_geometry():
    cam = synth.Pinhole(200, 100, 100.0, 100.0, 100.0, 50.0, np.eye(4), 0.2)
    k = 10
    offs = np.zeros((4, k, 3))
    offs[:, 0] = [0.5, 0, 0]                     # max offset 0.5 -> radius 0.5 + 3
    pos = np.array([[0.0, 0.0, 20.0],            # straight ahead: kept
                    [0.0, 0.0, -5.0],            # behind, beyond near - r: culled
                    [100.0, 0.0, 20.0],          # far to the right (x/z = 5 > 1): culled
                    [0.0, 0.0, -3.0]])           # behind but within near - r: kept
    m = OM.cull_mask(pos, np.ones(4), offs, cam)
    assert list(m) == [False, True, True, False]
    a = synth.Anchors(pos, np.zeros((4, 32)), np.ones(4), offs, np.zeros((4, k)))
    out = OM.decode(a, np.zeros((36, 64)), np.zeros(64), np.zeros((64, 100)), np.zeros(100), (0, 0, 0), cam=cam)
    op = out["opacity"].numpy().reshape(4, k)
    assert np.all(op[1] == OM.CULLED_LOGIT) and np.all(op[2] == OM.CULLED_LOGIT)
    assert np.all(op[0] == 0.0) and np.all(op[3] == 0.0)


def test_decode_gradients_flow_to_features_and_weights():
    a = _anchors(n=6)
    W1, b1, W2, b2 = (torch.tensor(x, dtype=torch.float64, requires_grad=True) for x in synth.init_mlp(4))
    f = torch.tensor(a.feature, dtype=torch.float64, requires_grad=True)
    out = OM.decode(a, W1, b1, W2, b2, (0, 0, 0), features=f)
    (out["opacity"].sum() + out["rgb"].sum()).backward()
    for t in (W1, b1, W2, b2, f):
        assert t.grad is not None and torch.isfinite(t.grad).all() and t.grad.abs().max() > 0
