"""GB300-native FDP=H space-time BIEM hot path (Sato & Ando, arXiv 1903.02118).

The compute path lives in ``libfdph.so`` (CUDA for sm_103a, C ABI in
``include/fdph.h``); ``fdph`` is its ctypes binding and ``inputs`` draws the
seeded synthetic workloads.  Importing the package does not load the library;
``fdph.lib()`` does, and raises if it has not been built.
"""
