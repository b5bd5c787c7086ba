"""The pixel-partitioned training step (Sec. III-A, "Paralleled training")
with the library's kernels behind each band: two gloo ranks, both on the one
visible GPU, split the image rows by balanced bands, exchange the surfels
each band needs (sparse all-to-all on the host), and each renders its band
camera, computes its share of the loss and runs the backward through the C
ABI; the gradients go back to their owners.  The owner-summed gradients and
the loss shares must equal a single-process GPU step on the whole image (to
1e-4 of the largest gradient: FP32 atomics and the band cameras' shifted
centre rows), and that step the FP64 oracle's gradient.

The two ranks' kernels never wait on one another: every exchange is a gloo
transfer of host tensors between whole band steps."""
import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2503_11731_gb300 import distributed as D
from paper_2503_11731_gb300 import synth

pytestmark = pytest.mark.gpu

W_DIST = 0.1
KEYS = ("pos", "log_scale", "quat", "opacity", "sh")


def _scene():
    # small enough for the FP64 autograd oracle (every pixel x every surfel)
    s = synth.driving_scene(n=400, seed=91, x_range=(2.0, 30.0), n_boxes=2, sh_degree=1)
    s.log_scale += 0.7  # fewer, larger surfels cover the little image
    tgt = synth.perturbed(s, seed=92)
    cam = synth.pinhole(64, 48, 40.0, (0.0, 0.5, 1.5), 0.0)
    return s, tgt, cam


def _flat(s):
    K = s.sh.shape[1]
    return np.concatenate([s.pos, s.log_scale, s.quat, s.opacity[:, None], s.sh.reshape(-1, 3 * K)], 1).astype(
        np.float32)


def _unflat(x, K):
    x = np.asarray(x, np.float32)
    return synth.Surfels(np.ascontiguousarray(x[:, 0:3]), np.ascontiguousarray(x[:, 3:5]),
                         np.ascontiguousarray(x[:, 5:9]), np.ascontiguousarray(x[:, 9]),
                         np.ascontiguousarray(x[:, 10:10 + 3 * K].reshape(-1, K, 3)),
                         np.zeros(len(x), np.float32))


def _rows(x, cam):
    """Conservative image rows of each surfel: its 3-sigma sphere projected
    by the (unrotated) camera, widened by the low-pass radius; every row
    when the sphere reaches the near plane."""
    pos, ls = x[:, 0:3].numpy().astype(np.float64), x[:, 3:5].numpy().astype(np.float64)
    R, t = cam.world_to_sensor[:3, :3], cam.world_to_sensor[:3, 3]
    m = pos @ R.T + t
    r = 3.0 * np.exp(ls.max(1)) + 1e-6
    z, y = m[:, 2], m[:, 1]
    H = cam.height
    lo = np.zeros(len(z), np.int64)
    hi = np.full(len(z), H - 1, np.int64)
    ok = z - r > cam.near
    ya = cam.cy + cam.fy * np.minimum((y - r) / (z - r), (y - r) / (z + r)) - 3.0
    yb = cam.cy + cam.fy * np.maximum((y + r) / (z - r), (y + r) / (z + r)) + 3.0
    lo[ok] = np.clip(np.floor(ya[ok] - 0.5), 0, H).astype(np.int64)
    hi[ok] = np.clip(np.ceil(yb[ok] - 0.5), -1, H - 1).astype(np.int64)
    return lo, hi


def _gpu_step(s_np, cam, target, rows, H):
    """Loss share and gradients of one camera (a band or the whole image)
    through the library: render, gsr_loss (L1 + 0.1 distortion), the
    per-pixel gradients scaled to the band's share of the image mean, and
    gsr_backward.  Returns (loss share, flat gradient [n, F] on the host)."""
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer, camera_backward, camera_loss
    d = DeviceSurfels.from_host(s_np)
    r = Renderer(s_np.n, [cam], tiles=[(16, 8)], outputs=("rgb", "depth", "normal", "alpha", "trans", "depth_acc",
                                                           "n_contrib"), split=(1 << 24, 1 << 24))
    r.render(d)
    loss, lo = camera_loss(r, 0, target, w_dist=W_DIST, w_normal=0.0)
    scale = rows / H
    for t in (lo.rgb, lo.alpha, lo.depth_acc, lo.normal):
        t.mul_(scale)
    g = {k: torch.zeros_like(getattr(d, k)) for k in KEYS}
    camera_backward(r, 0, lo.struct(), d, out=g)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    n = s_np.n
    flat = torch.cat([g["pos"], g["log_scale"], g["quat"], g["opacity"][:, None], g["sh"].reshape(n, -1)], 1)
    return float(loss[0]) * scale, flat.cpu().double()


def _worker(rank, world, port, q):
    import os
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    s, tgt, cam = _scene()
    K = s.sh.shape[1]
    full_t = _gpu_target(tgt, cam)
    x = torch.tensor(_flat(s))
    ids = torch.arange(s.n)
    mine = ids % world == rank  # surfels owned round-robin
    bounds = D.balance_rows(np.linspace(1.0, 3.0, cam.height), world)

    def band_fn(k, band_ids, band_x):
        y0, y1 = bounds[k], bounds[k + 1]
        loss, g = _gpu_step(_unflat(band_x.numpy(), K), D.band_camera(cam, y0, y1),
                            full_t[:, y0:y1].contiguous(), y1 - y0, cam.height)
        return loss, g.to(band_x.dtype), 0.0

    res = D.partitioned_step(ids[mine], x[mine], lambda p: _rows(p, cam), bounds, band_fn)
    q.put((rank, res.loss, ids[mine].numpy(), res.owned_grad.double().numpy(), bounds, res.received))
    dist.destroy_process_group()


def _gpu_target(tgt, cam):
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer
    r = Renderer(tgt.n, [cam], tiles=[(16, 8)], outputs=("rgb", "alpha"))
    r.render(DeviceSurfels.from_host(tgt))
    torch.cuda.synchronize()
    return r.out[0]["rgb"].clone()


def test_partitioned_step_with_library_kernels(gpu_lib):
    from test_distributed import _free_port
    s, tgt, cam = _scene()
    target = _gpu_target(tgt, cam)
    ref_loss, ref_grad = _gpu_step(s, cam, target, cam.height, cam.height)
    ref_grad = ref_grad.numpy()
    assert np.abs(ref_grad).max() > 0

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.spawn(_worker, args=(2, _free_port(), q), nprocs=2)
    got = [q.get() for _ in range(2)]
    loss = sum(g[1] for g in got)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    grad = np.zeros_like(ref_grad)
    for _, _, ids, g, bounds, received in got:
        grad[ids] = g
        assert 0 < bounds[1] < cam.height
        assert 0 < received < s.n  # each band received only the surfels it needs
    err = np.abs(grad - ref_grad).max() / np.abs(ref_grad).max()
    print("partitioned vs single-process GPU gradient: max error", err, "of the largest; bands", got[0][4])
    assert err <= 1e-4


def test_single_process_gpu_step_matches_fp64_oracle_gradient(gpu_lib):
    """The reference of the partitioned test: the GPU loss and gradient of
    the whole image against the FP64 oracle's (autograd of the plain
    definition), per parameter group to 1e-3 of its largest entry."""
    from oracle import grad as OG
    s, tgt, cam = _scene()
    target = _gpu_target(tgt, cam)
    loss, g = _gpu_step(s, cam, target, cam.height, cam.height)
    p = OG.surfel_tensors(s, requires_grad=True)
    out = OG.render_pinhole(p, cam)
    L, parts = OG.loss(out, target.permute(1, 2, 0).cpu().double(), cam, w_dist=W_DIST, w_norm=0.0)
    L.backward()
    assert loss == pytest.approx(float(L), rel=1e-4)
    n, K = s.n, s.sh.shape[1]
    ref = torch.cat([p["pos"].grad, p["log_scale"].grad, p["quat"].grad, p["opacity"].grad[:, None],
                     p["sh"].grad.reshape(n, -1)], 1).numpy()
    g = g.numpy()
    for name, sl in (("pos", slice(0, 3)), ("log_scale", slice(3, 5)), ("quat", slice(5, 9)), ("opacity", slice(9, 10)),
                     ("sh", slice(10, 10 + 3 * K))):
        scale = np.abs(ref[:, sl]).max()
        err = np.abs(g[:, sl] - ref[:, sl]).max()
        print(name, "max|ref|", scale, "max err", err)
        assert err <= 1e-3 * scale, name
