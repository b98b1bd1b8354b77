"""B300 (sm_103a) sparse Krylov solves with adjoint gradients.

A CUDA library (``libsla.so``, C ABI in include/sla.h) with hand-written
kernels for CSR SpMV, Jacobi-preconditioned CG and BiCGStab, and the linear
adjoint backward of arXiv 2601.13994 (Eq. 2-3), plus a thin Python layer:

* ``paper_2601_13994_b300.sla``     -- tensors in, kernels run, tensors out
* ``paper_2601_13994_b300.inputs``  -- seeded synthetic workloads
* ``paper_2601_13994_b300.build``   -- compiles the CUDA sources for sm_103a

The library is loaded on first use; a missing build raises immediately.
"""
__version__ = "0.1.0"
