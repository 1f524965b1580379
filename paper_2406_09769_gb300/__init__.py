"""GB300-native density-matrix tree approximation of tensor networks.

The compute path lives in the C-ABI library ``libtn_dmtree.so`` (sm_103a CUDA,
declared in include/tn_dmtree.h).  ``binding`` is a thin ctypes layer with the
same names as the C entry points; ``build`` compiles the library in-tree.
Importing this package does not load the library.
"""
