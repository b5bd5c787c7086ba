"""FP64 oracle of the anchor MLP decode (neural Gaussians).

TEST INFRASTRUCTURE, NOT PRODUCT CODE: used only by tests and the
benchmark's CPU-baseline leg; it never imports the CUDA package.

The paper infers each 2DGS attribute set by passing anchor features through
an MLP (Sec. III-A, "Scene Reconstruction": anchors organised as in
Scaffold-GS).  Readings of the points the paper leaves open:
  input   X = [f (32), d (3), |x_a - o| (1)] with d = (x_a - o)/|x_a - o|,
          o the view origin (the camera centre; the rig centre for a rig)
  hidden  H = ReLU(X W1 + b1)                         W1 [36, 64]
  output  Y = H W2 + b2, Y[a] = k offsets x 10 values  W2 [64, 10 k]
  offset j of anchor a, y = Y[a, 10 j : 10 j + 10]:
          opacity logit = y0, colour = sigmoid(y1..y3), log-scale = y4..y5 + ln l_a,
          raw quaternion = y6..y9, centre = x_a + l_a o_{a,j}
  LiDAR   the LiDAR scene's MLP (Sec. III-A infers {mu, R, S, rho, r, alpha}
  head    for the LiDAR scene G^L too) reads the same 10 values per offset
          as: opacity logit y0, intensity r = sigmoid(y1), ray-drop logit
          y2 (rho = sigmoid(y2)), y3 unused, log-scales y4..y5 + ln l_a,
          raw quaternion y6..y9; its table carries no colour (SH 0).
  cull    (optional, one pinhole camera) an anchor whose sphere of radius
          l_a max_j |o_{a,j}| + 3 m lies entirely behind the near plane or
          outside a side plane of the frustum renders nothing (its surfels
          get opacity logit -1e4).
The decoded colour is stored as a degree-0 SH coefficient (c - 0.5)/Y00 so
that the renderer reproduces it.
"""
from __future__ import annotations

import math

import numpy as np
import torch

DT = torch.float64
Y00 = 0.5 / math.sqrt(math.pi)
CULL_MARGIN = 3.0
CULLED_LOGIT = -1.0e4


def cull_mask(pos, scale, offsets, cam):
    """True for anchors the frustum of pinhole `cam` cannot see (FP64)."""
    M = np.asarray(cam.world_to_sensor, np.float64)
    pc = pos @ M[:3, :3].T + M[:3, 3]
    r = scale * np.linalg.norm(offsets, axis=-1).max(-1) + CULL_MARGIN
    z = pc[:, 2]
    out = z < cam.near - r
    # side planes through the camera centre: x/z = (0 - cx)/fx, (W - cx)/fx, y likewise
    for nx, ny in ((cam.fx, 0.0), (-cam.fx, 0.0), (0.0, cam.fy), (0.0, -cam.fy)):
        if nx > 0:
            n = np.array([cam.fx, 0.0, cam.cx])            # inside: fx x + cx z >= 0
        elif nx < 0:
            n = np.array([-cam.fx, 0.0, cam.width - cam.cx])  # inside: -fx x + (W - cx) z >= 0
        elif ny > 0:
            n = np.array([0.0, cam.fy, cam.cy])
        else:
            n = np.array([0.0, -cam.fy, cam.height - cam.cy])
        n = n / np.linalg.norm(n)
        out |= (pc @ n) < -r
    return out


def decode(anchors, W1, b1, W2, b2, origin, cam=None, features=None, head="camera"):
    """FP64 decode.  Returns a dict of tensors (pos [N,3], log_scale [N,2],
    quat [N,4], opacity [N], rgb [N,3], sh [N,1,3], intensity [N], and for
    head="lidar" ray_drop [N] logits) with N = A k, surfel a k + j = offset
    j of anchor a.  The camera head takes the intensity from the anchors,
    the LiDAR head from the network (its rgb is 0.5, sh 0).  Differentiable
    w.r.t. W1, b1, W2, b2 and `features` when they are tensors with
    requires_grad."""
    A, k = anchors.offsets.shape[0], anchors.offsets.shape[1]
    t = lambda a: a if isinstance(a, torch.Tensor) else torch.as_tensor(np.asarray(a, np.float64), dtype=DT)
    x = t(anchors.pos)
    f = t(anchors.feature) if features is None else features
    v = x - t(np.asarray(origin, np.float64))[None, :]
    dist = v.norm(dim=-1, keepdim=True)
    X = torch.cat([f, v / dist, dist], -1)
    H = torch.relu(X @ t(W1) + t(b1))
    Y = (H @ t(W2) + t(b2)).reshape(A, k, 10)
    l = t(anchors.scale)
    pos = x[:, None, :] + l[:, None, None] * t(anchors.offsets)
    opacity = Y[..., 0]
    if cam is not None:
        m = torch.as_tensor(cull_mask(np.asarray(anchors.pos, np.float64), np.asarray(anchors.scale, np.float64),
                                      np.asarray(anchors.offsets, np.float64), cam))
        opacity = torch.where(m[:, None], torch.full_like(opacity, CULLED_LOGIT), opacity)
    log_scale = Y[..., 4:6] + torch.log(l)[:, None, None]
    quat = Y[..., 6:10]
    N = A * k
    out = {"pos": pos.reshape(N, 3), "log_scale": log_scale.reshape(N, 2), "quat": quat.reshape(N, 4),
           "opacity": opacity.reshape(N), "hidden": H, "X": X, "Y": Y}
    if head == "lidar":
        out["rgb"] = torch.full((N, 3), 0.5, dtype=DT)
        out["sh"] = torch.zeros((N, 1, 3), dtype=DT)
        out["intensity"] = torch.sigmoid(Y[..., 1]).reshape(N)
        out["ray_drop"] = Y[..., 2].reshape(N)
    elif head == "camera":
        rgb = torch.sigmoid(Y[..., 1:4])
        out["rgb"] = rgb.reshape(N, 3)
        out["sh"] = ((rgb - 0.5) / Y00).reshape(N, 1, 3)
        out["intensity"] = t(anchors.intensity).reshape(N)
    else:
        raise ValueError(head)
    return out
