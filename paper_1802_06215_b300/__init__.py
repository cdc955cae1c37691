"""B300-native GPU leaf expansion for HyP-DESPOT (arXiv:1802.06215).

The CUDA library libdsp.so (C ABI in include/dsp.h) runs the data-parallel
hot path; `_dsp` is its ctypes binding, `batch` packs job batches into device
memory, `inputs` draws seeded synthetic workloads.
"""
from . import _dsp  # noqa: F401
