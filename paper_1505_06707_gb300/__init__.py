"""GB300 library for the exterior-complex-scaled split-operator FFT method of
Serov & Sergeeva (arXiv:1505.06707).

The compute path is the C-ABI library ``_lib/libsoft.so`` (hand-written CUDA
for sm_103a, declared in ``include/soft.h``); ``soft`` is a thin ctypes
binding with the same names.  PyTorch only supplies device memory and
streams.  There is no CPU fallback: loading fails loudly if the library is
missing or no GPU is present when a call needs one."""
from .soft import *  # noqa: F401,F403
