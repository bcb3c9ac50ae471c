"""GB300-native moment-encoded lattice Boltzmann (arXiv 2602.05295 hot path).

Submodules: ``melbm`` (ctypes binding of the CUDA library, ``include/melbm.h``),
``autograd`` (torch.autograd.Function over the adjoint), ``workloads`` (seeded
synthetic inputs) and ``build`` (compiles the library with nvcc).
"""
