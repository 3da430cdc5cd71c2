"""GB300-native dense-inverse apply for the 2-D variable-coefficient Poisson
equation (Dourbal & Pekker): u = L_eps^-1 b for many right-hand sides.

The compute path lives in a CUDA shared library (``csrc/``, C ABI declared in
``include/pide.h``); ``binding`` marshals arguments to it with ctypes and
``workloads`` draws seeded synthetic inputs.
"""
