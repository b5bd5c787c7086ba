"""GPU test of the double-buffered zone streamer (gsr_streamer_*): a camera
and a LiDAR driving across four 40 m zones (25 % padding) render, frame by
frame, exactly what a synchronously uploaded copy of the current zone
renders; the next zone is prefetched on the copy stream while the vehicle
is in its padding band, and the buffers swap when it crosses."""
import numpy as np
import pytest
import torch

from paper_2503_11731_gb300 import gsr, synth

pytestmark = pytest.mark.gpu


def _resident_copy(zs, z, capacity):
    """The zone's packed surfels on the device, the tail culled (reference)."""
    from paper_2503_11731_gb300.frame import DeviceSurfels
    pk = zs.zones[z]
    n = zs.size(z)
    K = pk["sh"].shape[1]
    d = DeviceSurfels(torch.zeros(capacity, 3, device="cuda"), torch.zeros(capacity, 2, device="cuda"),
                      torch.zeros(capacity, 4, device="cuda"), torch.full((capacity,), -1e4, device="cuda"),
                      torch.zeros(capacity, K, 3, device="cuda"), torch.zeros(capacity, device="cuda"))
    for k in ("pos", "log_scale", "quat", "opacity", "sh", "intensity"):
        getattr(d, k)[:n] = pk[k].to("cuda")
    return d


def _sensors(x):
    return [synth.pinhole(320, 180, 170.0, (x, 0.0, 1.5), 0.0), synth.spinning_lidar(32, 360, -25.0, 15.0,
                                                                                     (x, 0.0, 1.8))]


def test_streamed_zones_render_like_resident_copies(gpu_lib):
    from paper_2503_11731_gb300.frame import Renderer
    from paper_2503_11731_gb300.stream import ZoneScene, ZoneStreamer
    s = synth.driving_scene(n=200_000, seed=61, x_range=(-20.0, 140.0), n_boxes=10)
    zs = ZoneScene(s, gsr.zone_grid(-20.0, -20.0, 40.0, 0.25, 4, 1))
    st = ZoneStreamer(zs)
    outs = ("rgb", "depth", "alpha", "range", "intensity")
    tiles = [(16, 8), (8, 8)]
    r = Renderer(st.capacity, _sensors(0.0), tiles=tiles, outputs=outs)
    ref = Renderer(st.capacity, _sensors(0.0), tiles=tiles, outputs=outs)
    swaps, prefetched = 0, set()
    front = None
    for x in np.arange(-10.0, 130.0, 7.5):
        z = zs.zone_of(x, 0.0)
        if z not in st.resident():
            st.prefetch(z)  # not predicted: copy now, the acquire waits for it
        d = st.acquire(z)
        swaps += front is not None and st.s.front != front
        front = st.s.front
        r.move(_sensors(x))
        got = r.render(d)
        # the next zone ahead, once the vehicle is in its padding band
        for nz in zs.zones_near(x, 0.0):
            if nz != z and nz not in st.resident():
                st.prefetch(nz)
                prefetched.add(nz)
        ref.move(_sensors(x))
        want = ref.render(_resident_copy(zs, z, st.capacity))
        torch.cuda.synchronize()
        assert r.status()[0] == 0 and ref.status()[0] == 0
        for a, b in zip(got, want):
            for k in a:
                assert torch.equal(a[k], b[k]), (x, z, k)
    assert swaps >= 3 and prefetched >= {1, 2, 3}
    st.close()
