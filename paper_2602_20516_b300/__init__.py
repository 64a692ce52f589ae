"""B300-native (sm_103a) HMC hot path for two-flavour Wilson fermions in SU(3)
lattice gauge theory (arXiv:2602.20516): Wilson-Dirac stencil, CG, forces,
link update and HMC behind the C-ABI library ``liblgt.so``.

Importing the package loads nothing; ``paper_2602_20516_b300.lgt`` loads the
CUDA library and raises if it is missing.
"""
__all__ = ["lgt", "synth"]
