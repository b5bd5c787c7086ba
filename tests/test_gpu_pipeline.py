"""Streamed frames (FramePipeline): uploads and read-backs on their own
streams overlap the neighbouring frames, and the objects' preprocess runs
alongside the decode inside each frame's first graph; every frame's outputs
are bit-identical to a serial render of that frame's inputs (here: object
poses that change every frame, per-frame pinned host buffers, no
synchronisation between the frames)."""
import numpy as np
import pytest
import torch

from paper_2503_11731_gb300 import gsr, synth

pytestmark = pytest.mark.gpu


def test_pipeline_frames_equal_serial_frames(gpu_lib):
    from paper_2503_11731_gb300.frame import DeviceSurfels, Renderer
    from paper_2503_11731_gb300.neural import DeviceAnchors, FramePipeline, NeuralFrame, NeuralModel
    bg = synth.driving_scene(n=40_000, seed=91, x_range=(0.0, 40.0), n_boxes=4)
    anchors, _ = synth.anchors_from_surfels(bg, k=10, seed=92)
    objs = None
    for k in range(3):
        a = synth.object_asset(2_000, seed=93 + k)
        a.obj_id = np.full(a.n, k, np.int32)
        objs = a if objs is None else objs.concat(a)
    sensors = [synth.pinhole(256, 160, 200.0, (0.0, 0.0, 1.5)),
               synth.spinning_lidar(32, 512, -25.0, 10.0, (0.0, 0.0, 1.8))]
    n = anchors.n * anchors.k + objs.n
    r = Renderer(n, sensors, tiles=[(16, 8), (8, 8)], max_dup=1 << 22,
                 outputs=("rgb", "depth", "alpha", "range", "intensity"))
    poses = [synth.object_poses(3, seed=100 + f, x_range=(6.0, 30.0)).reshape(-1, 12).astype(np.float32)
             for f in range(3)]
    pose_t = torch.as_tensor(poses[0], device="cuda")
    nf = NeuralFrame(NeuralModel(*synth.init_mlp(7)), DeviceAnchors(anchors), r, DeviceSurfels.from_host(objs),
                     pose_t, (0.0, 0.0, 1.6), gsr.DECODE_BF16_TENSOR)
    keys = [(i, k) for i, o in enumerate(r.out) for k in o]
    # serial frames, one per pose set
    ref = []
    for P in poses:
        pose_t.copy_(torch.as_tensor(P))
        nf.render()
        torch.cuda.synchronize()
        ref.append({(i, k): r.out[i][k].cpu().clone() for i, k in keys})
    assert not torch.equal(ref[0][(0, "rgb")], ref[1][(0, "rgb")])  # the poses move the objects
    # streamed: three frames enqueued back to back
    host_in = [torch.as_tensor(P).pin_memory() for P in poses]
    host_out = [[torch.empty(r.out[i][k].shape, dtype=r.out[i][k].dtype).pin_memory() for i, k in keys]
                for _ in poses]
    pipe = FramePipeline(nf, [(pose_t, host_in[0])],
                         [(r.out[i][k], host_out[0][j]) for j, (i, k) in enumerate(keys)])
    torch.cuda.synchronize()
    for f in range(3):
        pipe.frame(host_inputs=[host_in[f]], host_outputs=host_out[f])
    pipe.finish()
    torch.cuda.synchronize()
    for f in range(3):
        for j, key in enumerate(keys):
            assert torch.equal(host_out[f][j], ref[f][key]), (f, key)
