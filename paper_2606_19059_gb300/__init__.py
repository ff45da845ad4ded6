"""GB300-native spectral Ewald summation for the triply periodic Stokeslet.

The compute path is the CUDA library ``libewald_gb300.so`` (sources in
``csrc/``, C ABI in ``include/ewald_gb300.h``); ``ewald`` is its ctypes
binding and ``workloads`` the seeded synthetic inputs.
"""
