"""GB300-native fused track propagation + Kalman update (p2r / p2z).

The compute path is the CUDA library ``libfit.so`` (sources in ``csrc/``,
C-ABI in ``include/fit.h``); ``fit`` is its thin ctypes binding and
``inputs`` draws seeded synthetic workloads.  Importing the package loads
nothing; the first call into ``fit`` loads the library and raises if it is
missing.
"""
