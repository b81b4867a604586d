"""GB300 (sm_103a) Galerkin-FFT homogenization of lattice cells.

The compute path is libhom.so (hand-written CUDA, C ABI in include/hom.h);
``paper_2110_00733_gb300.hom`` is its ctypes binding (hom_create, hom_solve,
hom_effective_stiffness, hom_fields and the step entry points used by the
parity tests).  ``paper_2110_00733_gb300.build`` compiles the library in-tree.
"""
__all__ = ["build", "hom"]
