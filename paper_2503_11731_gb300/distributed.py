"""Pixel-partitioned training across ranks (Sec. III-A, "Paralleled
training", after Grendel-GS): each rank renders a contiguous band of image
rows, the bands are balanced by measured rendering time, the surfels a band
needs travel to its rank by a sparse all-to-all, and their gradients travel
back to the ranks that own them; shared MLP parameters are all-reduced.

Host logic over torch.distributed (point-to-point sends and receives, which
the NCCL and gloo backends both provide).  A rank renders its band with a
band camera -- the same pinhole with the image cut to rows [y0, y1): cy
shifted by -y0, height y1 - y0 -- so every pixel keeps its ray and the GPU
renderer needs nothing new.  The per-rank render/loss/backward is a
callable, the library's kernels on a GPU.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch
import torch.distributed as dist


def balance_rows(row_cost, n_parts: int):
    """Bounds b_0 = 0 < b_1 < ... < b_n = H of n contiguous row bands whose
    summed costs are as equal as row granularity allows: b_k is the row at
    which the running cost first reaches k/n of the total (each band at
    least one row)."""
    c = np.cumsum(np.asarray(row_cost, np.float64))
    H = len(c)
    if n_parts < 1 or n_parts > H:
        raise ValueError("need 1 <= n_parts <= rows")
    total = c[-1]
    bounds = [0]
    for k in range(1, n_parts):
        b = int(np.searchsorted(c, total * k / n_parts, side="left")) + 1 if total > 0 else (H * k) // n_parts
        b = max(b, bounds[-1] + 1)
        b = min(b, H - (n_parts - k))
        bounds.append(b)
    bounds.append(H)
    return bounds


def band_camera(cam, y0: int, y1: int):
    """The pinhole `cam` restricted to image rows [y0, y1)."""
    return dataclasses.replace(cam, height=int(y1 - y0), cy=float(cam.cy - y0))


class RowCost:
    """Per-row rendering cost, updated from each band's measured time
    (spread evenly over its rows) as an exponential moving average."""

    def __init__(self, height: int, decay: float = 0.5):
        self.cost = np.ones(height, np.float64)
        self.decay = decay

    def update(self, bounds, band_ms):
        new = self.cost.copy()
        for k in range(len(bounds) - 1):
            y0, y1 = bounds[k], bounds[k + 1]
            new[y0:y1] = band_ms[k] / (y1 - y0)
        self.cost = self.decay * self.cost + (1 - self.decay) * new


def needed_by_band(row_lo, row_hi, bounds):
    """For each band, a boolean mask of the surfels whose image rows
    [row_lo, row_hi] (inclusive; row_hi < row_lo = not visible) meet it."""
    row_lo, row_hi = np.asarray(row_lo), np.asarray(row_hi)
    vis = row_hi >= row_lo
    return [vis & (row_lo < bounds[k + 1]) & (row_hi >= bounds[k]) for k in range(len(bounds) - 1)]


def sparse_all_to_all(send, group=None):
    """send[q] = tensor for rank q (same dtype and trailing shape on every
    rank, any leading size, possibly 0); returns recv[p] = what rank p sent
    here.  Sizes are exchanged first (all_gather), then the payloads by
    point-to-point sends and receives."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = send[0].device
    n = torch.tensor([t.shape[0] for t in send], dtype=torch.int64, device=dev)
    all_n = [torch.empty_like(n) for _ in range(world)]
    dist.all_gather(all_n, n, group=group)
    tail = tuple(send[0].shape[1:])
    recv = [torch.empty((int(all_n[p][rank]),) + tail, dtype=send[0].dtype, device=dev) for p in range(world)]
    recv[rank] = send[rank].clone()
    ops = []
    for q in range(world):
        if q == rank:
            continue
        if send[q].shape[0] > 0:
            ops.append(dist.P2POp(dist.isend, send[q].contiguous(), q, group))
        if recv[q].shape[0] > 0:
            ops.append(dist.P2POp(dist.irecv, recv[q], q, group))
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()
    return recv


@dataclasses.dataclass
class StepResult:
    loss: float          # this rank's share of the loss (the shares sum to the image loss)
    owned_grad: torch.Tensor  # d(loss)/d(owned parameters), every band's contribution summed
    band_ms: float
    received: int        # surfels this rank's band needed (its share of the sparse exchange)


def partitioned_step(owned_ids, owned_params, row_range, bounds, band_fn, group=None, mlp_grads=None):
    """One training step of this rank.

    owned_ids [m] (int64, global surfel ids), owned_params [m, F] (the
    parameters this rank owns), row_range(params) -> (row_lo, row_hi) of
    each surfel on the full image, bounds = balance_rows(...) (the same on
    every rank), band_fn(k, ids, params) -> (loss, d loss / d params, ms) for
    band k given the surfels it received (ids ascending: the plan's
    composite ties break by surfel index, so a band's list order is the
    full image's).  mlp_grads: tensors all-reduced (summed) across ranks.
    """
    rank = dist.get_rank(group)
    lo, hi = row_range(owned_params)
    need = needed_by_band(lo, hi, bounds)
    send_ids = [owned_ids[torch.as_tensor(m)] for m in need]
    send_par = [owned_params[torch.as_tensor(m)] for m in need]
    got_ids = sparse_all_to_all(send_ids, group)
    got_par = sparse_all_to_all(send_par, group)
    ids = torch.cat(got_ids)
    par = torch.cat(got_par)
    order = torch.argsort(ids)
    loss, g, ms = band_fn(rank, ids[order], par[order])
    # gradients back to the owners, in the order each sent its surfels
    g_unsorted = torch.empty_like(g)
    g_unsorted[order] = g
    back = list(torch.split(g_unsorted, [t.shape[0] for t in got_ids]))
    ret = sparse_all_to_all(back, group)
    owned_grad = torch.zeros_like(owned_params)
    for q, m in enumerate(need):
        owned_grad[torch.as_tensor(np.nonzero(m)[0])] += ret[q]
    if mlp_grads:
        for t in mlp_grads:
            dist.all_reduce(t, group=group)
    return StepResult(float(loss), owned_grad, float(ms), int(ids.shape[0]))
