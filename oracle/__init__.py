"""FP64 CPU oracle of the 2D-Gaussian surfel sensor renderer.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only the test suite, the smoke check
and the CPU-baseline leg of the benchmark import this package.  It shares no
code with the CUDA path (`paper_2503_11731_gb300`), and never imports it.

* `render_pinhole`, `render_lidar` -- brute-force forward render (C, FP64,
  OpenMP) of Eqs. 1-3 and 5 with the compositing rules of 3DGS/2DGS.
* `grad` -- the same forward definition in PyTorch FP64 CPU ops, used with
  autograd for the reconstruction loss and its gradient on small cases.
* `mlp` -- the anchor MLP decode (Scaffold-GS style) in PyTorch FP64.
"""
from .render import build_oracle, render_pinhole, render_lidar, num_threads  # noqa: F401
