"""GPU check of the pixel partition used for multi-GPU training: a camera
cut into row bands (band cameras: same rays, cy shifted, height cut)
renders every band row like the full image (bit-exactly for the first
band; to FP32 rounding of the shifted centre row for the others), and the gradients
of the band losses (L1 + distortion, each band's share of the image mean)
sum to the full image's gradient."""
import numpy as np
import pytest
import torch

from paper_2503_11731_gb300 import distributed as D
from paper_2503_11731_gb300 import synth

pytestmark = pytest.mark.gpu


def test_band_renders_and_gradients_sum_to_full_image(gpu_lib):
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer, camera_backward, camera_loss
    s = synth.driving_scene(n=60_000, seed=71, x_range=(-10.0, 60.0), n_boxes=6)
    cam = synth.pinhole(320, 200, 170.0, (0.0, 0.5, 1.5), 0.0)
    tgt = synth.perturbed(s, seed=72)
    outs = ("rgb", "depth", "normal", "alpha", "trans", "depth_acc", "n_contrib")
    d, dt = DeviceSurfels.from_host(s), DeviceSurfels.from_host(tgt)
    split = (1 << 24, 1 << 24)  # unsplit lists: band rows bit-exact

    def grads_of(c, rows):
        r = Renderer(s.n, [c], tiles=[(16, 8)], outputs=outs, split=split)
        r.render(dt)
        target = r.out[0]["rgb"].clone()
        out = r.render(d)[0]
        g = {k: torch.zeros_like(getattr(d, k)) for k in ("pos", "log_scale", "quat", "opacity", "sh")}
        loss, lo = camera_loss(r, 0, target, w_dist=0.1, w_normal=0.0)
        # the band's mean over its rows, as a share of the image mean
        scale = rows / cam.height
        for t in (lo.rgb, lo.alpha, lo.depth_acc, lo.normal):
            t.mul_(scale)
        camera_backward(r, 0, lo.struct(), d, out=g)
        torch.cuda.synchronize()
        return {k: v.clone() for k, v in out.items()}, float(loss[0]) * scale, g

    full_out, full_loss, full_g = grads_of(cam, cam.height)
    bounds = D.balance_rows(np.linspace(1.0, 4.0, cam.height), 3)
    assert bounds[1] % 8 and bounds[2] % 8  # bands that do not start on a tile row
    loss_sum = 0.0
    g_sum = {k: torch.zeros_like(v) for k, v in full_g.items()}
    for k in range(3):
        y0, y1 = bounds[k], bounds[k + 1]
        bo, bl, bg = grads_of(D.band_camera(cam, y0, y1), y1 - y0)
        for key in ("rgb", "depth", "alpha", "trans", "normal", "depth_acc"):
            a, b = bo[key], full_out[key][..., y0:y1, :]
            if k == 0:  # same pixel frame: identical arithmetic
                assert torch.equal(a, b), (k, key)
            else:  # the centre's row moves by -y0 in FP32: rounding-level differences
                scale = max(1.0, float(b.abs().max())) if key in ("depth", "depth_acc") else 1.0
                assert (a - b).abs().max().item() <= 2e-5 * scale, (k, key)
        loss_sum += bl
        for key in g_sum:
            g_sum[key] += bg[key]
    assert loss_sum == pytest.approx(full_loss, rel=1e-5)
    for key in g_sum:
        err = (g_sum[key] - full_g[key]).abs().max().item()
        assert err <= 1e-4 * full_g[key].abs().max().item(), key
