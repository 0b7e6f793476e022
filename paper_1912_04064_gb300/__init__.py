"""GB300-native patch-decomposed (SDMD) particle-in-cell hot path.

The compute path is the C-ABI library ``libpic.so`` (hand-written sm_103a
CUDA kernels); :mod:`.pic` is its thin ctypes binding and
:mod:`.workloads` the seeded synthetic input generators.
"""
