"""GB300-native transpose-algorithm multidimensional FFT on a virtual process grid.

Implements the hot path of Dalcin, Mortensen & Keyes, "Fast parallel
multidimensional FFT using advanced MPI" (arXiv:1804.09536): batched 1-D FFTs
along one axis at a time with global redistributions between them, the
virtual ranks laid out in one GPU's memory and every redistribution fused
into the FFT passes' loads and stores.  The compute runs in the CUDA kernels
of ``libtfft.so`` behind the C ABI of ``include/tfft.h``.
"""
from ._lib import (TFFT_BACKWARD, TFFT_FORWARD, TfftError, load)  # noqa: F401


def __getattr__(name):
    if name == "Plan":
        from .plan import Plan
        return Plan
    raise AttributeError(name)
