"""B300 (sm_103a) sparse Krylov solves with adjoint gradients.

A CUDA library (``libsla.so``, C ABI in include/sla.h) with hand-written
kernels for CSR SpMV, Jacobi-preconditioned CG and BiCGStab, and the linear
adjoint backward of arXiv 2601.13994 (Eq. 2-3), plus a thin Python layer:

* ``paper_2601_13994_b300.sla``       -- tensors in, kernels run, tensors out:
  SpMV, CG (standard, cooperative or pipelined), BiCGStab, the adjoint
  backward, batched and multi-right-hand-side solves, LOBPCG ``eigsh`` with
  the Hellmann-Feynman eigenvalue gradient (Eq. 4), the autograd Functions
* ``paper_2601_13994_b300.learned``   -- the learned M = G G^T preconditioner
* ``paper_2601_13994_b300.nonlinear`` -- Newton solves with the one-solve
  adjoint (Sec. 3.2)
* ``paper_2601_13994_b300.inverse``   -- the inverse coefficient problem (Sec. 4.6)
* ``paper_2601_13994_b300.inputs``    -- seeded synthetic workloads
* ``paper_2601_13994_b300.build``     -- compiles the CUDA sources for sm_103a

The library is loaded on first use; a missing build raises immediately.
"""
__version__ = "0.1.0"
