"""Large scenes: zones and the double-buffered zone streamer, over the C ABI
(gsr_zone_* / gsr_streamer_*; marshalling only).

A scene larger than one zone is packed once on the host: every zone's
surfels (its padded square) contiguous in pinned memory.  While the vehicle
drives, the streamer keeps two device buffers: frames draw from the front
one while the next zone is copied into the back one on a copy stream, and
crossing into that zone swaps them (the render stream waits for the copy's
event, the copy stream for the render stream to release the old front).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import gsr
from .frame import DeviceSurfels, _ptr, _stream_handle


def _table(d: DeviceSurfels) -> gsr.SurfelTable:
    return gsr.SurfelTable(_ptr(d.pos), _ptr(d.log_scale), _ptr(d.quat), _ptr(d.opacity), _ptr(d.sh),
                           _ptr(d.intensity), _ptr(d.ray_drop))


class ZoneScene:
    """A host surfel table (synth.Surfels-like, float32) cut into zones of a
    gsr.ZoneGrid and packed per zone into pinned host memory."""

    def __init__(self, s, grid: gsr.ZoneGrid, pin=True):
        self.grid = grid
        self.sh_degree = int(round(np.sqrt(s.sh.shape[1]))) - 1
        f = lambda a: np.ascontiguousarray(a, np.float32)
        self.src = {k: f(getattr(s, k)) for k in ("pos", "log_scale", "quat", "opacity", "sh", "intensity")}
        rd = getattr(s, "ray_drop", None)
        self.src["ray_drop"] = None if rd is None else f(rd)
        self.offsets, self.members = gsr.zone_members(grid, self.src["pos"])
        self.zones = []
        K = (self.sh_degree + 1) ** 2
        for z in range(grid.nx * grid.ny):
            m = np.ascontiguousarray(self.members[self.offsets[z]:self.offsets[z + 1]])
            n = len(m)
            t = lambda *shape: torch.empty(*shape, dtype=torch.float32, pin_memory=pin)
            pk = {"pos": t(n, 3), "log_scale": t(n, 2), "quat": t(n, 4), "opacity": t(n), "sh": t(n, K, 3),
                  "intensity": t(n), "ray_drop": t(n) if self.src["ray_drop"] is not None else None}
            out = gsr.SurfelTable(*[_ptr(pk[k]) for k in ("pos", "log_scale", "quat", "opacity", "sh",
                                                           "intensity", "ray_drop")])
            gsr._check(gsr.lib().gsr_zone_pack(ctypes.byref(self._host_struct()),
                                               m.ctypes.data_as(ctypes.c_void_p), n, ctypes.byref(out)),
                       "gsr_zone_pack")
            self.zones.append(pk)

    def _host_struct(self) -> gsr.Surfels:
        p = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
        src = self.src
        return gsr.Surfels(int(src["pos"].shape[0]), self.sh_degree, p(src["pos"]), p(src["log_scale"]),
                           p(src["quat"]), p(src["opacity"]), p(src["sh"]), p(src["intensity"]), None,
                           p(src["ray_drop"]), 0)

    def zone_struct(self, z) -> gsr.Surfels:
        pk = self.zones[z]
        return gsr.Surfels(int(pk["pos"].shape[0]), self.sh_degree, _ptr(pk["pos"]), _ptr(pk["log_scale"]),
                           _ptr(pk["quat"]), _ptr(pk["opacity"]), _ptr(pk["sh"]), _ptr(pk["intensity"]), None,
                           _ptr(pk["ray_drop"]), 0)

    def size(self, z) -> int:
        return int(self.offsets[z + 1] - self.offsets[z])

    @property
    def max_zone(self) -> int:
        return int(np.diff(self.offsets).max())

    def zone_of(self, x, y) -> int:
        return gsr.zone_of(self.grid, x, y)

    def zones_near(self, x, y):
        """Zones whose padded square holds (x, y) (the ones worth having resident)."""
        s, p = self.grid.zone_size, self.grid.padding
        i = (x - self.grid.x0) / s
        j = (y - self.grid.y0) / s
        out = []
        for jj in range(self.grid.ny):
            for ii in range(self.grid.nx):
                if ii - p <= i < ii + 1 + p and jj - p <= j < jj + 1 + p:
                    out.append(jj * self.grid.nx + ii)
        return out


class ZoneStreamer:
    """Two device buffers of `capacity` surfels fed from a ZoneScene on a
    copy stream (gsr_streamer)."""

    def __init__(self, scene: ZoneScene, capacity=None, device="cuda"):
        self.scene = scene
        cap = scene.max_zone if capacity is None else int(capacity)
        K = (scene.sh_degree + 1) ** 2
        z = lambda *shape: torch.zeros(*shape, device=device)
        has_rd = scene.src["ray_drop"] is not None
        self.bufs = [DeviceSurfels(z(cap, 3), z(cap, 2), z(cap, 4), z(cap), z(cap, K, 3), z(cap),
                                   ray_drop=z(cap) if has_rd else None) for _ in range(2)]
        self.copy_stream = torch.cuda.Stream(device=device)
        self.s = gsr.streamer_init(cap, scene.sh_degree, [_table(b) for b in self.bufs],
                                   ctypes.c_void_p(self.copy_stream.cuda_stream))
        self.capacity = cap

    def prefetch(self, zone):
        """Start copying `zone` into the back buffer (no-op if it is resident)."""
        gsr.streamer_prefetch(self.s, zone, self.scene.zone_struct(zone))

    def acquire(self, zone, stream=None) -> DeviceSurfels:
        """The zone's device table, ready for work enqueued on `stream` from now on."""
        gsr.streamer_acquire(self.s, zone, _stream_handle(stream))
        return self.bufs[self.s.front]

    def resident(self):
        return [self.s.zone[0], self.s.zone[1]]

    def close(self):
        gsr.streamer_destroy(self.s)
