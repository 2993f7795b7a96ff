"""CPU FP64 oracle for the tensor-product (KSVD) preconditioned DG solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference arm of ``bench.py`` may import anything here.  The
product path (the CUDA library and its Python binding) never imports, links or
runs this package, and this package never imports the product path.

Plain, slow, obviously-correct NumPy/SciPy code following Pazner & Persson,
"Approximate tensor-product preconditioners for very high order discontinuous
Galerkin methods":

* ``basis``    - 1D Lagrange basis on Gauss-Legendre nodes, quadrature,
                 evaluation/differentiation matrices (Sec. 3.1-3.2).
* ``dg``       - explicit element-by-element assembly of M - dt*J for linear
                 advection with upwind flux (Sec. 3.4.1, Eq. jac-entries,
                 Table tab:dg-ops) and a sum-factorised matvec (Alg. 1).
* ``ksvd``     - Van Loan-Pitsianis rearrangement and the Kronecker SVD by a
                 dense SVD (Sec. 4.1, Eq. NKP), 3D nested form (Sec. 4.3).
* ``precond``  - dense-LU application of P^-1, the paper's Schur/Sylvester
                 application (Alg. 2d-apply, 3d-apply), exact block Jacobi.
* ``gmres``    - restarted right-preconditioned GMRES and flexible GMRES.

Parity status of each function is stated in its module header.
"""
