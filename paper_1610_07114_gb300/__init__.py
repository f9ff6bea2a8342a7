"""GB300-native thermal cascaded lattice Boltzmann method (Fei & Luo, arXiv:1610.07114).

The compute path is the C-ABI library libtclbm.so (hand-written sm_103a CUDA);
`paper_1610_07114_gb300.tclbm` is its ctypes binding.  Importing this package does
not load the library; the binding does, and fails loudly when it is missing.
"""

__all__ = ["workloads", "tclbm"]
