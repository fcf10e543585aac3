"""GB300 (sm_103a) BGV encrypted comparison.

The computation lives in the CUDA library ``lib/libfhe_gb300.so`` (C ABI in
``include/fhe.h``); ``fhe`` is its Python binding and ``synth`` the seeded
input generator.  Build the library with ``build.build()``.
"""
