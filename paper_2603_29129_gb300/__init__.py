"""GB300-native FP64-accurate FFT by the Ozaki scheme over 32-bit NTTs.

The compute path lives in ``libozfft.so`` (hand-written CUDA for sm_103a behind
a C ABI, declared in ``include/ozfft.h``); :mod:`.ozfft` is its ctypes binding.
Importing this package does not load the library; the first call does, and it
raises if the library is missing (there is no CPU fallback).
"""
__all__ = ["ozfft", "autograd", "synth"]
