"""GB300-native PRC-LBM: the fused stream-and-collide update of the
preconditioned rectangular central-moment lattice Boltzmann method
(arXiv:2208.03562) as hand-written sm_103a CUDA behind a C ABI.

Importing the package loads nothing native; ``paper_2208_03562_gb300.lbm``
loads the CUDA library and fails loudly when it is missing.
"""
__all__ = ["inputs"]
