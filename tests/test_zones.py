"""CPU checks of the zone partition of large scenes (host C++ in the
library) against the brute-force oracle: membership bit-exact (ascending
indices per zone), the zone of a point, the packing of a zone's surfels,
and argument errors of the streamer that need no device."""
import ctypes

import numpy as np
import pytest

from oracle import zones as OZ
from paper_2503_11731_gb300 import build as B
from paper_2503_11731_gb300 import gsr, synth


@pytest.fixture(scope="module")
def L():
    B.build()
    return gsr.lib()


def _grid_dict(g):
    return {"x0": g.x0, "y0": g.y0, "zone_size": g.zone_size, "padding": g.padding, "nx": g.nx, "ny": g.ny}


def _points(rng, n):
    pos = np.stack([rng.uniform(-110, 190, n), rng.uniform(-40, 80, n), rng.normal(0, 1, n)], 1)
    # points exactly on padded-square edges (integers here: -80 + (i -+ 0.25) 40)
    edges = np.array([-90.0, -70.0, -50.0, -30.0, -10.0, 10.0, 30.0, 50.0, 70.0, 90.0, 110.0, 130.0, 150.0])
    k = n // 4
    pos[:k, 0] = rng.choice(edges, k)
    pos[k:2 * k, 1] = rng.choice(edges, k)
    return pos.astype(np.float32)


def test_zone_members_match_oracle(L):
    g = gsr.zone_grid(-80.0, -20.0, 40.0, 0.25, 6, 2)
    pos = _points(np.random.default_rng(1), 20_000)
    offsets, members = gsr.zone_members(g, pos)
    ref = OZ.members(_grid_dict(g), pos)
    assert len(offsets) == 13
    for z in range(12):
        got = members[offsets[z]:offsets[z + 1]]
        assert np.array_equal(got, ref[z]), z
    # multiplicity: a surfel belongs to at most four zones
    mult = np.bincount(members, minlength=len(pos))
    assert mult.max() == 4 and (mult == 0).any() and (mult == 1).any()


def test_zone_of_matches_oracle(L):
    g = gsr.zone_grid(-80.0, -20.0, 40.0, 0.25, 6, 2)
    pos = _points(np.random.default_rng(2), 3000)
    for x, y in pos[:, :2]:
        assert gsr.zone_of(g, x, y) == OZ.zone_of(_grid_dict(g), float(x), float(y))
    assert gsr.zone_of(gsr.zone_grid(0.0, 0.0, 0.0, 0.25, 1, 1), 1.0, 1.0) == -1  # bad grid


def test_zone_pack_gathers_members(L):
    from paper_2503_11731_gb300.stream import ZoneScene
    s = synth.driving_scene(n=5000, seed=3, x_range=(-20.0, 60.0), n_boxes=2)
    s.ray_drop = np.random.default_rng(4).normal(size=s.n).astype(np.float32)
    g = gsr.zone_grid(-20.0, -20.0, 40.0, 0.25, 2, 1)
    zs = ZoneScene(s, g, pin=False)
    ref = OZ.members(_grid_dict(g), s.pos)
    for z in range(2):
        m = ref[z]
        assert zs.size(z) == len(m)
        for k in ("pos", "log_scale", "quat", "opacity", "sh", "intensity", "ray_drop"):
            src = np.asarray(getattr(s, k), np.float32)
            assert np.array_equal(zs.zones[z][k].numpy(), src[m]), (z, k)
    # a zone near a point: its padded square holds it
    assert zs.zones_near(19.0, 0.0) == [0, 1] and zs.zones_near(0.0, 0.0) == [0]


def test_zone_argument_errors(L):
    g = gsr.zone_grid(0.0, 0.0, 40.0, 0.75, 2, 2)  # padding beyond 0.5
    n = ctypes.c_int64(0)
    counts = np.zeros(4, np.int64)
    pos = np.zeros((1, 3), np.float32)
    assert L.gsr_zone_count(ctypes.byref(g), pos.ctypes.data_as(ctypes.c_void_p), 1,
                            counts.ctypes.data_as(ctypes.c_void_p)) == gsr.ERR_INVALID_ARG
    g = gsr.zone_grid(0.0, 0.0, 40.0, 0.25, 2, 2)
    bad = np.array([0, 0, 0, 0, 0], np.int64)  # offsets too small for the members
    pos = np.array([[10.0, 10.0, 0.0]], np.float32)
    mem = np.zeros(4, np.int64)
    assert L.gsr_zone_members(ctypes.byref(g), pos.ctypes.data_as(ctypes.c_void_p), 1,
                              bad.ctypes.data_as(ctypes.c_void_p), mem.ctypes.data_as(ctypes.c_void_p)) \
        == gsr.ERR_INVALID_ARG
    st = gsr.Streamer()
    bufs = (gsr.SurfelTable * 2)()
    assert L.gsr_streamer_init(ctypes.byref(st), -1, 0, bufs, None) == gsr.ERR_INVALID_ARG
    assert L.gsr_streamer_init(ctypes.byref(st), 10, 0, bufs, None) == gsr.ERR_INVALID_ARG  # null buffers
