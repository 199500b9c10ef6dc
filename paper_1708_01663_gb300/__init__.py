"""GB300-native hot path of CISOR (relaxed-FISTA nonlinear diffraction tomography).

The compute lives in ``libcisor.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/cisor.h``); ``paper_1708_01663_gb300.cisor`` is the thin
ctypes binding with the same names.  Importing this package loads nothing:
``synth`` (seeded inputs) is usable without a GPU, and the library is loaded
when ``cisor`` is imported.
"""
