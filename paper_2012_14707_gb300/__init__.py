"""GB300-native slip-wall D2Q9 MRT lattice Boltzmann solver.

The compute path lives in the CUDA library `liblbm.so` built from `csrc/`;
`lbm` is its thin ctypes binding.  `cases` generates seeded inputs.  Import
the submodules explicitly: importing the package loads nothing.
"""
