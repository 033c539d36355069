"""GB300 (sm_103a) implementation of the pseudo-potential (Shan-Chen) multiphase
lattice Boltzmann step of arXiv:1906.11027, behind the C ABI of include/lbm.h.

``lbm`` is the thin ctypes binding; ``_build`` compiles the CUDA library in-tree;
``inputs`` holds the seeded synthetic workload generators.
"""
