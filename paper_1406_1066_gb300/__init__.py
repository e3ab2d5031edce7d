"""GB300-native Matlab-compatible sparse assembly (Engblom & Lukarski, arXiv:1406.1066).

The compute path is the CUDA library ``libfsparse.so`` (sources in ``csrc/``,
public C header ``include/fsparse.h``).  ``paper_1406_1066_gb300.fsparse`` is
the thin ctypes binding with the same names; importing this package itself
loads nothing.
"""
__all__ = ["fsparse", "inputs"]
