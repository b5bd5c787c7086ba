"""Pixel-partitioned training on CPU ranks (gloo, world size 2): the row
balancer, the sparse all-to-all, and one partitioned training step whose
loss shares and owner-summed gradients equal the single-process step of the
FP64 oracle (band renders stand in for the GPU renderer here)."""
import math
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2503_11731_gb300 import distributed as D
from paper_2503_11731_gb300 import synth


def test_balance_rows():
    assert D.balance_rows(np.ones(100), 4) == [0, 25, 50, 75, 100]
    # a costly top half: the first bands are thin
    c = np.concatenate([np.full(50, 9.0), np.ones(50)])
    b = D.balance_rows(c, 2)
    assert b[0] == 0 and b[2] == 100 and 27 <= b[1] <= 29
    # every band keeps at least one row, even with all the cost in one row
    c = np.zeros(10)
    c[0] = 1.0
    b = D.balance_rows(c, 4)
    assert b == sorted(b) and len(set(b)) == 5 and b[-1] == 10
    rc = D.RowCost(100, decay=0.0)
    rc.update([0, 20, 100], [4.0, 4.0])
    assert np.allclose(rc.cost[:20], 0.2) and np.allclose(rc.cost[20:], 0.05)
    assert D.balance_rows(rc.cost, 2)[1] == 20


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _a2a_worker(rank, world, port, q):
    _init(rank, world, port)
    rng = np.random.default_rng(rank)
    sizes = [int(rng.integers(0, 4)) for _ in range(world)]
    send = [torch.full((n, 2), float(10 * rank + dst)) for dst, n in enumerate(sizes)]
    got = D.sparse_all_to_all(send)
    q.put((rank, sizes, [g.tolist() for g in got]))
    dist.destroy_process_group()


def test_sparse_all_to_all_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    mp.spawn(_a2a_worker, args=(2, port, q), nprocs=2)
    res = {}
    while not q.empty():
        r, sizes, got = q.get()
        res[r] = (sizes, got)
    for r in (0, 1):
        for p in (0, 1):
            n = res[p][0][r]
            assert res[r][1][p] == [[10.0 * p + r] * 2] * n


# ------------------------------------------------------- partitioned step
W_DIST = 0.1


def _flat(s):
    K = s.sh.shape[1]
    return np.concatenate([s.pos, s.log_scale, s.quat, s.opacity[:, None], s.sh.reshape(-1, 3 * K)], 1)


def _unflat(x, K):
    return {"pos": x[:, 0:3], "log_scale": x[:, 3:5], "quat": x[:, 5:9], "opacity": x[:, 9],
            "sh": x[:, 10:10 + 3 * K].reshape(-1, K, 3)}


def _scene():
    s = synth.plain_scene(n=160, seed=41)
    s.pos[:, 2] = np.clip(s.pos[:, 2], 8.0, 40.0)
    cam = synth.plain_camera(48, 32, 40.0)
    tgt = synth.plain_scene(n=160, seed=42)
    return s, cam, tgt


def _band_loss(params, cam, target, y0, y1, H, W):
    """Loss share of rows [y0, y1): sum |C - C*| / (3 H W) + w sum (A D - B^2) / (H W)."""
    from oracle import grad as OG
    out = OG.render_pinhole(params, D.band_camera(cam, y0, y1))
    l1 = (out["rgb"] - target[y0:y1]).abs().sum() / (3 * H * W)
    dst = (out["A"] * out["D"] - out["B"] ** 2).sum() / (H * W)
    return l1 + W_DIST * dst


def _rows(x, cam):
    """Conservative image rows of each surfel: its 3-sigma sphere projected,
    widened by the low-pass radius (full image if it reaches the near plane)."""
    pos, ls = x[:, 0:3].numpy(), x[:, 3:5].numpy()
    r = 3.0 * np.exp(ls.max(1)) + 1e-6
    z = pos[:, 2]
    H = cam.height
    lo = np.zeros(len(z), np.int64)
    hi = np.full(len(z), H - 1, np.int64)
    ok = z - r > cam.near
    y = pos[:, 1]
    ya = cam.cy + cam.fy * np.minimum((y - r) / (z - r), (y - r) / (z + r)) - 3.0
    yb = cam.cy + cam.fy * np.maximum((y + r) / (z - r), (y + r) / (z + r)) + 3.0
    lo[ok] = np.clip(np.floor(ya[ok] - 0.5), 0, H).astype(np.int64)
    hi[ok] = np.clip(np.ceil(yb[ok] - 0.5), -1, H - 1).astype(np.int64)
    return lo, hi


def _step_worker(rank, world, port, q):
    from oracle import grad as OG
    torch.set_default_dtype(torch.float64)
    _init(rank, world, port)
    s, cam, tgt = _scene()
    K = s.sh.shape[1]
    target = OG.render_pinhole(OG.surfel_tensors(tgt), cam)["rgb"].detach()
    x = torch.tensor(_flat(s), dtype=torch.float64)
    ids = torch.arange(s.n)
    mine = ids % world == rank  # surfels owned round-robin
    bounds = D.balance_rows(np.linspace(1.0, 3.0, cam.height), world)

    def band_fn(k, band_ids, band_x):
        leaf = band_x.clone().requires_grad_(True)
        L = _band_loss(_unflat(leaf, K), cam, target, bounds[k], bounds[k + 1], cam.height, cam.width)
        L.backward()
        return L.detach(), leaf.grad, 0.0

    mlp_g = [torch.full((3,), float(rank + 1))]
    res = D.partitioned_step(ids[mine], x[mine], lambda p: _rows(p, cam), bounds, band_fn, mlp_grads=mlp_g)
    q.put((rank, res.loss, ids[mine].numpy(), res.owned_grad.numpy(), mlp_g[0].numpy(), bounds, res.received))
    dist.destroy_process_group()


def test_partitioned_step_equals_single_process():
    from oracle import grad as OG
    torch.set_default_dtype(torch.float64)
    s, cam, tgt = _scene()
    K = s.sh.shape[1]
    target = OG.render_pinhole(OG.surfel_tensors(tgt), cam)["rgb"].detach()
    x = torch.tensor(_flat(s), dtype=torch.float64, requires_grad=True)
    L = _band_loss(_unflat(x, K), cam, target, 0, cam.height, cam.height, cam.width)
    L.backward()
    ref_loss, ref_grad = float(L.detach()), x.grad.numpy()
    torch.set_default_dtype(torch.float32)
    assert np.abs(ref_grad).max() > 0

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.spawn(_step_worker, args=(2, _free_port(), q), nprocs=2)
    got = [q.get() for _ in range(2)]
    loss = sum(g[1] for g in got)
    assert loss == pytest.approx(ref_loss, rel=1e-12)
    grad = np.zeros_like(ref_grad)
    for _, _, ids, g, mlp, bounds, received in got:
        grad[ids] = g
        assert np.array_equal(mlp, [3.0, 3.0, 3.0])  # all-reduced MLP gradients
        assert 0 < bounds[1] < cam.height
        assert 0 < received < s.n  # each band received only the surfels it needs
    assert np.abs(grad - ref_grad).max() <= 1e-10 * np.abs(ref_grad).max()
