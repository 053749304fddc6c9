"""GB300-native CompaSO hot path (Hadzhiyska et al. 2021, arXiv:2110.11408).

Kernel density, L0 friends-of-friends and the competitive spherical-overdensity
assignment (L1, then L2 inside each L1 halo) as CUDA kernels for sm_103a behind
a C ABI (``include/cso.h``); ``paper_2110_11408_gb300.cso`` is the thin ctypes
binding with the same entry-point names, ``synth`` draws seeded inputs.
"""
