"""GB300 (sm_103a) library for certified dual bounds of the perspective relaxation
of k-sparse, box-constrained, ridge-regularised GLMs (arXiv 2502.09502).

``paper_2502_09502_gb300.ksc`` is the ctypes binding of the C ABI in
``include/ksc.h``; ``paper_2502_09502_gb300.build`` compiles the CUDA library.
"""
__all__ = ["build", "ksc"]
