"""GB300 (sm_103a) NOHAP/OUCS3 compressible Navier-Stokes hot path.

The compute lives in libnopcs.so (hand-written CUDA behind the C ABI of
include/nopcs.h); this package only marshals arguments (nopcs.py) and builds
the library (build.py).
"""
