"""GB300-native exact-diagonalization impurity solver (Sec. 4 of arXiv:2305.18643).

The compute path is libed.so (CUDA C++ for sm_103a, C ABI in include/ed.h); the submodule
``ed`` is its ctypes binding, ``build`` compiles it and ``workloads`` holds the seeded
synthetic cluster generators.
"""
