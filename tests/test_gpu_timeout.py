"""The device-side give-up path: a bounded wait that runs out records
GSR_ERR_TIMEOUT in the plan's status word, the kernel returns, and the
context stays usable (the next frame renders bit-identically to one before
the timeout).  The wait is made to run out on an mbarrier armed for bytes
that no copy delivers, so nothing is in flight when it gives up."""
import pytest
import torch

from paper_2503_11731_gb300 import gsr, synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_with_timeout_status(gpu_lib):
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer, _stream_handle
    s = synth.plain_scene(n=2000, seed=4)
    cam = synth.plain_camera(96, 64, 80.0)
    r = Renderer(s.n, [cam])
    d = DeviceSurfels.from_host(s)
    before = {k: v.clone() for k, v in r.render(d)[0].items()}
    assert r.status()[0] == gsr.OK
    gsr.selftest_wait_timeout(r.plan, r.ws_ptr, r.ws_bytes, 64, _stream_handle())
    st, _, _ = r.status()
    assert st == gsr.ERR_TIMEOUT
    # a frame after the timeout: the preprocess clears the status word and
    # the frame is the same as before
    after = r.render(d)[0]
    torch.cuda.synchronize()
    assert r.status()[0] == gsr.OK
    for k in before:
        assert torch.equal(before[k], after[k]), k
    # arguments out of range are refused on the host
    with pytest.raises(gsr.GsrError):
        gsr.selftest_wait_timeout(r.plan, r.ws_ptr, r.ws_bytes, 0, _stream_handle())
