"""GB300 (sm_103a) rectangular MRT lattice Boltzmann step behind a C ABI.

``rmrtlb`` is the ctypes binding of ``include/rmrtlb.h``; ``build`` compiles
the CUDA library in-tree; ``slab`` cuts one grid into slabs over ranks;
``warmstart`` trains and applies the learned warm start; ``runlog`` writes
the JSON-lines record of a run.  Importing the package loads nothing.
"""
