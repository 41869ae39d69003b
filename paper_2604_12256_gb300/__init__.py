"""GB300-native full state-vector quantum circuit simulator.

The simulation runs in hand-written CUDA kernels for sm_103a behind the C ABI
declared in ``include/svsim.h`` (``libsvsim.so``); :mod:`.svsim` is the thin
ctypes binding with the same names.  :mod:`.circuits` holds the seeded
synthetic workload generators.

The native library is loaded lazily (on first use of :mod:`.svsim`), so the
generators import without a GPU.
"""
__all__ = ["circuits", "svsim", "build"]
