"""GB300-native FFT apply of the null-space-free reduced Maxwell operator.

The compute path lives in the CUDA/C++ library ``_lib/libfame.so`` (C ABI
declared in ``include/fame.h``); ``fame`` is its thin ctypes binding and
``workloads`` holds the seeded synthetic inputs.  Importing the package loads
nothing; the library is loaded on first use and a missing library raises.
"""
