"""GB300-native IgA + p-multigrid + MGRIT heat solver (arXiv 2107.05337).

The compute path is the C-ABI library ``libigamgrit.so`` built from
``csrc/`` (hand-written CUDA for sm_103a); ``binding`` wraps it with ctypes.
Importing this package does not load the library; ``binding.lib()`` does, and
raises if it is missing -- there is no CPU fallback.
"""
