"""CFIE hot path for 2-D high-frequency obstacle scattering on GB300 (sm_103a).

The compute runs in the CUDA library ``libcfie.so`` (built from ``csrc/`` by
``build.py``); ``cfie`` is its ctypes binding.  Importing this package does not
load the library; ``paper_1408_1578_gb300.cfie`` does, and fails loudly if it
is missing.
"""
