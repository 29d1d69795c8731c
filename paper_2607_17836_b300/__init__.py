"""B300-native one-way coupled Eulerian-Lagrangian particle hot path.

The compute path lives in ``libelpath.so`` (hand-written sm_103a CUDA kernels
behind a C ABI, see ``include/elpath.h``); :mod:`.elpath` is the thin ctypes
binding, :mod:`.inputs` the seeded synthetic workloads.  Importing the package
loads nothing; the library is opened on first use and a missing library is an
error, never a fallback.
"""
