"""GB300-native (sm_103a) bmDCA hot path: Gibbs sweeps, chain statistics,
Boltzmann update with the Pearson check, sequence weights, data frequencies,
energy scoring and mutant scans (adabmDCA 2.0, arXiv 2501.18456).

The compute lives in libbmdca.so (C ABI, include/bmdca.h).  Submodules:
  bmdca   -- ctypes binding, same names as the C entry points
  train   -- the host-side bmDCA training loop on top of the binding
  synth   -- seeded synthetic inputs (planted Potts models, MSAs)
  _build  -- nvcc build of libbmdca.so

Importing the package loads nothing; the library is opened on first use.
"""

__version__ = "0.1"
