"""GB300-native substage of the low-Mach, variable-density pseudospectral method (arXiv:2206.09878).

The compute path is liblmvd.so (hand-written CUDA for sm_103a behind the C-ABI in include/lmvd.h);
``paper_2206_09878_gb300.lmvd`` is its ctypes binding, ``build`` compiles it in-tree and
``rt_inputs`` generates seeded Rayleigh-Taylor-shaped initial states.
"""
