"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every symbol include/gsr.h declares, its struct layouts match the binding,
and host-only calls (plan, workspace size, argument errors) behave.  No
kernel is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2503_11731_gb300 import build as B
from paper_2503_11731_gb300 import gsr, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return gsr.lib()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(gsr_\w+)\s*\(", txt, re.M))
    return names


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    assert set(gsr.SIGNATURES) <= names


def test_struct_layouts_match(L):
    for i, st in enumerate(gsr._STRUCTS):
        assert L.gsr_struct_size(i) == ctypes.sizeof(st), st.__name__


def test_plan_and_workspace_host_only(L):
    cam = synth.plain_camera()
    lid = synth.driving_lidar()
    p = gsr.plan_init(8000, [gsr.sensor(cam), gsr.sensor(lid)], (16, 16))
    assert p.tiles_x[0] == 16 and p.tiles_y[0] == 10
    assert p.tiles_x[1] == 113 and p.tiles_y[1] == 8
    assert p.tile_base[1] == 160 and p.tile_base[2] == 160 + 904
    ws = gsr.workspace_size(p)
    assert ws >= 2 * 8000 * 80 and ws % 256 == 0
    offs = [p.off[i] for i in range(19)]
    assert offs == sorted(offs) and all(o % 256 == 0 for o in offs)


def test_argument_errors(L):
    cam = gsr.sensor(synth.plain_camera())
    with pytest.raises(gsr.GsrError) as e:
        gsr.plan_init(10, [cam], (12, 16))
    assert e.value.code == gsr.ERR_UNSUPPORTED
    bad = gsr.sensor(synth.plain_camera())
    bad.fx = 0.0
    with pytest.raises(gsr.GsrError) as e:
        gsr.plan_init(10, [bad])
    assert e.value.code == gsr.ERR_INVALID_ARG
    # a cylindrical image must stay within azimuths [-pi, pi]
    wide = gsr.sensor(synth.cylindrical(400, 100, 200.0, 60.0))
    wide.fx = 400 / 7.0
    with pytest.raises(gsr.GsrError) as e:
        gsr.plan_init(10, [wide])
    assert e.value.code == gsr.ERR_INVALID_ARG
    assert gsr.plan_init(10, [gsr.sensor(synth.cylindrical(400, 100, 360.0, 60.0))]).sensors[0].kind == gsr.CYLINDRICAL
    p = gsr.plan_init(10, [cam])
    # undersized / misaligned workspace is rejected before any launch
    buf = (ctypes.c_uint8 * 1024)()
    s = gsr.Surfels()
    s.n = 10
    rc = L.gsr_preprocess(ctypes.byref(p), ctypes.byref(s), None, ctypes.cast(buf, ctypes.c_void_p), 1024, None)
    assert rc == gsr.ERR_WORKSPACE
    # a part outside the plan's surfel range is rejected before any launch
    # (the workspace address is never dereferenced on this path)
    fake_ws, nbytes = ctypes.c_void_p(1 << 20), gsr.workspace_size(p)
    for first, n in ((-1, 4), (7, 4), (0, 11)):
        s.n = n
        rc = L.gsr_preprocess_part(ctypes.byref(p), ctypes.byref(s), None, first, fake_ws, nbytes, None)
        assert rc == gsr.ERR_INVALID_ARG, (first, n)
    rc = L.gsr_bin_sort(ctypes.byref(p), None, 0, None)
    assert rc == gsr.ERR_INVALID_ARG
    assert gsr.status_string(gsr.ERR_CAPACITY) == "GSR_ERR_CAPACITY"


def test_autotune_workspace_and_batch_depth_host_only(L):
    cam, lid = gsr.sensor(synth.driving_camera()), gsr.sensor(synth.driving_lidar())
    p = gsr.plan_init(100_000, [cam, lid], (16, 16))
    cams, lids = ((16, 16), (8, 8), (32, 8)), ((8, 8), (4, 8))
    sp = gsr.autotune_space(cams, lids, (64, 256))
    need = gsr.autotune_workspace_size(p, sp)
    for ct in cams:
        for lt in lids:
            q = gsr.plan_init(100_000, [gsr.sensor(synth.driving_camera(), tile=ct),
                                        gsr.sensor(synth.driving_lidar(), tile=lt)], (16, 16))
            assert gsr.workspace_size(q) <= need
    # the staging depth does not change the workspace; odd depths are rejected
    assert gsr.workspace_size(gsr.plan_init(100_000, [cam, lid], (16, 16), batch_depth=512)) == gsr.workspace_size(p)
    for bd in (16, 100, 1024):
        with pytest.raises(gsr.GsrError) as e:
            gsr.plan_init(100_000, [cam, lid], (16, 16), batch_depth=bd)
        assert e.value.code == gsr.ERR_UNSUPPORTED
    # bad spaces and part lists are rejected before any launch
    bad = gsr.autotune_space(cams, lids, (64,), reps=0)
    n = ctypes.c_size_t()
    assert L.gsr_autotune_workspace_size(ctypes.byref(p), ctypes.byref(bad), ctypes.byref(n)) == gsr.ERR_INVALID_ARG
    part = gsr.Surfels()
    part.n = 99_999   # parts must cover the plan exactly
    res = gsr.AutotuneResult()
    rc = L.gsr_autotune(ctypes.byref(p), ctypes.byref(part), 1, None, ctypes.byref(sp), ctypes.c_void_p(1 << 20),
                        need, None, None, ctypes.byref(res), None)
    assert rc == gsr.ERR_INVALID_ARG
