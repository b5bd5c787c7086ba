"""gsr_loss_noalloc: the reconstruction loss for callers that cannot allocate
device memory (no plan, no workspace; scratch in the library's own fixed
device array).  Its results must equal those of gsr_loss, the entry point
that uses a caller-allocated workspace, call after call.

This file is named to be collected last, so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2503_11731_gb300 import gsr, synth

pytestmark = pytest.mark.gpu


def _buffers(H, W, seed):
    """Seeded camera outputs and a target, as the loss consumes them."""
    rng = np.random.default_rng(seed)
    dev = lambda a: torch.as_tensor(a.astype(np.float32), device="cuda").contiguous()
    A = rng.uniform(0.3, 1.0, (H, W))
    z = rng.uniform(5.0, 6.0, (H, W))
    return {"rgb": dev(rng.uniform(0, 1, (3, H, W))), "alpha": dev(A),
            "depth_acc": dev(np.stack([A * z, A * z * z * 1.01])),
            "normal": dev(rng.normal(0, 0.5, (3, H, W))), "target": dev(rng.uniform(0, 1, (3, H, W)))}


def _grads(H, W):
    return {"rgb": torch.zeros(3, H, W, device="cuda"), "alpha": torch.zeros(H, W, device="cuda"),
            "depth_acc": torch.zeros(2, H, W, device="cuda"), "normal": torch.zeros(3, H, W, device="cuda"),
            "loss": torch.zeros(4, device="cuda")}


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _structs(b, g):
    fwd = gsr.CameraOut(_p(b["rgb"]), None, _p(b["normal"]), _p(b["alpha"]), None, _p(b["depth_acc"]), None, None)
    cg = gsr.CameraGrad(_p(g["rgb"]), _p(g["alpha"]), _p(g["depth_acc"]), _p(g["normal"]))
    return fwd, cg


def test_loss_noalloc_matches_workspace_loss_twice():
    if not torch.cuda.is_available():
        pytest.fail("gpu test selected but no CUDA device is visible")
    from paper_2503_11731_gb300 import build
    build.build()
    L = gsr.lib()
    H, W = 160, 256
    cam = synth.Pinhole(W, H, 200.0, 190.0, 128.0, 80.0, np.eye(4), 0.2)
    sensor = gsr.sensor(cam)
    plan = gsr.plan_init(1, [sensor])
    ws_bytes = gsr.workspace_size(plan)
    ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device="cuda")
    ws_ptr = ctypes.c_void_p((ws.data_ptr() + 255) & ~255)
    weights = gsr.LossWeights(0.1, 0.05, 0.5)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((1, 2)):  # two calls in a row, different inputs
        b = _buffers(H, W, seed)
        g_ws, g_na = _grads(H, W), _grads(H, W)
        fwd, cg = _structs(b, g_ws)
        rc = L.gsr_loss(ctypes.byref(plan), ws_ptr, ws_bytes, 0, ctypes.byref(fwd), _p(b["target"]),
                        ctypes.byref(weights), _p(g_ws["loss"]), ctypes.byref(cg), stream)
        assert rc == gsr.OK, gsr.status_string(rc)
        fwd, cg = _structs(b, g_na)
        rc = L.gsr_loss_noalloc(ctypes.byref(sensor), ctypes.byref(fwd), _p(b["target"]), ctypes.byref(weights),
                                _p(g_na["loss"]), ctypes.byref(cg), stream)
        assert rc == gsr.OK, gsr.status_string(rc)
        torch.cuda.synchronize()
        assert float(g_ws["loss"][0]) > 0
        for k in g_ws:
            a, n = g_ws[k].cpu().numpy(), g_na[k].cpu().numpy()
            np.testing.assert_allclose(n, a, rtol=1e-6, atol=1e-9 * max(1.0, float(np.abs(a).max())),
                                       err_msg=f"call {call}: {k}")


def test_loss_noalloc_rejects_frames_beyond_its_limit():
    if not torch.cuda.is_available():
        pytest.fail("gpu test selected but no CUDA device is visible")
    L = gsr.lib()
    cam = synth.Pinhole(2048, 1025, 1000.0, 1000.0, 1024.0, 512.0, np.eye(4), 0.2)  # 2,099,200 px > limit
    assert cam.width * cam.height > gsr.NOALLOC_MAX_PIXELS
    sensor = gsr.sensor(cam)
    dummy = torch.zeros(4, device="cuda")
    fwd = gsr.CameraOut(_p(dummy), None, _p(dummy), _p(dummy), None, _p(dummy), None, None)
    cg = gsr.CameraGrad(_p(dummy), _p(dummy), _p(dummy), _p(dummy))
    rc = L.gsr_loss_noalloc(ctypes.byref(sensor), ctypes.byref(fwd), _p(dummy), ctypes.byref(gsr.LossWeights(0.1, 0.05, 0.5)),
                            _p(dummy), ctypes.byref(cg), None)
    assert rc == gsr.ERR_TOO_LARGE
    assert gsr.status_string(rc) == "GSR_ERR_TOO_LARGE"
