"""GB300-native STAMP hot path: SVGD over differentiable planar block pushing.

The CUDA library is reached through :mod:`paper_2310_01775_gb300.stamp` (a
ctypes binding of the C ABI in ``include/stamp.h``); importing that module
fails loudly when the library has not been built.  :mod:`.workloads` holds
the seeded synthetic inputs.
"""
