"""GB300-native (sm_103a) channel-flow Poisson / z-implicit Helmholtz solver.

The hot path of Diez, Peeters & Costa (arXiv 2502.06296) on one GPU: a packed
real FFT along x (App. A), a TMA-staged complex FFT along y, one Thomas sweep per
wavenumber pair along the stretched z (Eq. 12), and the reworked parallel cyclic
reduction of Algorithm 2 for the z-implicit Helmholtz solve (Eq. 11).

Submodules: ``chanfs`` (ctypes binding of the C-ABI library ``libchanfs.so``,
loaded on first use) and ``synth`` (seeded synthetic inputs).
"""
