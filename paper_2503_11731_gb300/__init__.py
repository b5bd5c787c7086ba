"""GB300-native 2D-Gaussian surfel sensor renderer (arXiv 2503.11731, Sec. III-A).

Modules:
  gsr     -- ctypes binding of the C ABI (include/gsr.h), loads _lib/libgsr.so
  frame   -- device buffers and a Renderer over the C ABI (PyTorch for memory/streams)
  build   -- nvcc build of libgsr.so for sm_103a
  synth   -- seeded synthetic scenes and sensor rigs (inputs only)

Importing the package loads nothing; `gsr.lib()` fails loudly when the CUDA
library is missing.
"""
