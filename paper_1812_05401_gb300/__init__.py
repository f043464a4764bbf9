"""GB300-native volume-penalization lattice Boltzmann solver (arXiv 1812.05401).

- ``vplbm``: ctypes binding of the C ABI in include/vplbm.h (libvplbm.so, CUDA).
- ``inputs``: seeded synthetic workloads.
- ``diag``: post-processing of force series and fields (C_D, C_L, St, L2 error).
- ``serve``: continuous-batching serving loop over grouped launches.
- ``build``: in-tree nvcc build of libvplbm.so for sm_103a.

Importing the package loads nothing; the CUDA library loads on first use.
"""
