"""GB300-native pseudo-potential D2Q9 lattice Boltzmann library.

Implements the per-timestep update of Kupershtokh et al.'s large-density-ratio
single-component model as analysed by Hu, Li & Uddin (arXiv:1412.5170):
Carnahan-Starling psi (Eqs. 7, 29-30), hybrid psi/psi^2 force (Eq. 6), Guo /
exact-difference / Shan-Chen forcing (Eqs. 20-23), BGK or MRT collision
(Eqs. 1, 34-36), periodic pull streaming.

The compute path is the CUDA library ``liblbm.so`` built from ``csrc/`` for
sm_103a; ``lbm`` below is its thin ctypes binding.  Importing this package
does not load the library; ``paper_1412_5170_gb300.lbm`` does, and raises if
it is missing (there is no CPU fallback).
"""

__all__ = ["lbm", "synth"]
