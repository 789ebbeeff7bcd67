"""GB300-native 2D radix-2 decimation-in-time FFT of images.

The transforms run in hand-written sm_103a CUDA kernels behind the C ABI of
``include/fft2d.h`` (``_lib/libfft2d.so``); this package is its thin Python
binding.  Importing it fails loudly when the library has not been built.
"""
from .fft2d import *  # noqa: F401,F403
from .fft2d import FFT2DError, Plan, lib, LIB_PATH  # noqa: F401
