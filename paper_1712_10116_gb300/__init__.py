"""GB300-native momentum-conserving FMM + HHS N-body solver (Zhu 2017, arXiv:1712.10116).

The compute path is the CUDA library ``libtaichi_gb.so`` (C ABI declared in
``include/taichi_gb.h``); :mod:`paper_1712_10116_gb300.binding` is a thin ctypes layer over
it that marshals PyTorch device tensors.  Importing this package loads nothing; the library
is loaded on first use and a missing library raises immediately (there is no CPU fallback).
"""

__all__ = ["binding", "ics"]
