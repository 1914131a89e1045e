"""GB300-native two-point correlation pair counting (Alonso 2012, CUTE).

The compute path lives in the CUDA library ``libcute_gb.so`` (csrc/), reached
through the ctypes binding in :mod:`paper_1210_1833_gb300.cute`.  The binding
is imported on first use so that :mod:`paper_1210_1833_gb300.synthetic` can be
used without a built library; any call into the library fails loudly when it
is missing.
"""
__all__ = ["synthetic"]
