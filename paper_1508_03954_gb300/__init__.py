"""GB300-native additive multilevel Helmholtz solver (complex scaled grids,
tripartitioned regular levels).  ``mg`` is the ctypes binding of the CUDA
library, ``build`` compiles it, ``workloads`` generates seeded inputs."""
__all__ = ["mg", "build", "workloads"]
