"""GB300-native coupled viscoelastic lattice Boltzmann step (arXiv 2508.16997).

The compute path is the C-ABI library ``liblbve.so`` (hand-written sm_103a CUDA
kernels); :mod:`.lbve` is its thin ctypes binding.  Importing this package
does not load the library; the first call into :mod:`.lbve` does, and fails
loudly if it is missing.
"""
__all__ = ["lbve", "workloads", "build"]
