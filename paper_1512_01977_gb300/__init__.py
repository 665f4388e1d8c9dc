"""GB300-native axisymmetric multiphase lattice Boltzmann engine (arXiv:1512.01977).

The update runs in hand-written sm_103a CUDA kernels behind a C ABI
(include/lbm_axi.h); this package is the thin Python binding over it.
"""
