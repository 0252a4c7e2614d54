"""GB300 (sm_103a) implementation of the MRT finite-difference lattice
Boltzmann step of Chen, Xu, Zhang & Li (arXiv:1106.0785).

Layout:
  csrc/          CUDA kernels and the C ABI (libmrtlb.so)
  build.py       in-tree nvcc build of libmrtlb.so
  mrtlb.py       ctypes binding with the C names (include/mrtlb.h)
  simulation.py  PyTorch-facing wrapper (device buffers, stream)
  d2v16.py       the paper's velocity set and M as handed to mrtlb_create
  workloads.py   seeded synthetic inputs for the paper's workloads
"""
from .mrtlb import Config, MrtlbError  # noqa: F401
