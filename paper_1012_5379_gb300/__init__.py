"""GB300-native GMRES(3)-smoothed multigrid for the complex-stretched-grid Helmholtz
preconditioner inside an outer FP64 flexible GMRES (arXiv:1012.5379).

The compute path is the C-ABI library ``libhelm.so`` (hand-written sm_103a CUDA);
``paper_1012_5379_gb300.helm`` is its ctypes binding.  Importing this package loads
nothing; the binding loads the library on first use and raises if it is missing.
"""
__all__ = ["helm", "inputs"]
