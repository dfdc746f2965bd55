"""GB300 (sm_103a) NNFFT: the nonuniform FFT with nonequispaced spatial and
frequency data (type 3) with sinh-type windows, and the fast sinc transform,
after Kircheis, Potts and Tasche.

The transforms run in the CUDA library built from ``csrc/`` (C ABI in
``include/nnfft.h``); ``nnfft`` is its ctypes binding.  The library is loaded
on first use, so importing this package needs neither a GPU nor a build.
"""
from .nnfft import (NNFFTError, Plan, gauss_legendre, library_path, load_library, params,
                    sinc, sinc_release, sinc_sync)

__all__ = ["NNFFTError", "Plan", "gauss_legendre", "library_path", "load_library", "params",
           "sinc", "sinc_release", "sinc_sync"]
