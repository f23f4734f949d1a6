"""GB300 (sm_103a) rectangular MRT lattice Boltzmann step behind a C ABI.

``rmrtlb`` is the ctypes binding of ``include/rmrtlb.h``; ``build`` compiles
the CUDA library in-tree.  Importing the package loads nothing.
"""
