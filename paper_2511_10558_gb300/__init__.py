"""Batched stiff astrochemistry on GB300: BDF integration of many 0-D cells.

Submodules are imported on demand: ``synth`` (seeded inputs, no GPU needed)
and ``carbox`` (the ctypes binding over the CUDA library; it raises if the
library is not built).
"""
