"""GB300-native bus injections and power-flow Jacobians (Ybus and element-wise
methods of arXiv 2302.10736), FP64 CUDA kernels for sm_103a behind a C ABI.

Submodules:
  pfgrid  - thin ctypes binding of libpfgrid.so (the C ABI in include/pfgrid.h)
  synth   - seeded synthetic grid / voltage / contingency generator (inputs only)
  _build  - in-tree compilation of the native parts
"""
__version__ = "0.1.0"
