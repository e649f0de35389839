"""GB300 (sm_103a) implementation of the F-AMS two-stage pressure solver for
porous media with embedded discrete fractures (arXiv 1705.05784).

Submodules:
  fams    - ctypes binding of the C ABI in include/fams.h (loads lib/libfams.so)
  build   - compiles lib/libfams.so with nvcc
  inputs  - seeded synthetic problem generators (no method arithmetic)
  tune    - schedule autotuner (precision variant x GMRES restart, timed on
            a workload, cached by the workload's signature)

Importing the package loads nothing; ``from paper_1705_05784_gb300 import fams``
loads the CUDA library and fails loudly if it has not been built.
"""
