"""CPU oracle for the matrix-free neo-Hookean operators (test infrastructure only).

This package is a plain, slow, FP64 NumPy statement of what the GPU library computes.  It
shares no code with the CUDA path and is used only by `tests/`, by the smoke check and by
the CPU-baseline leg of the benchmark; the product path never imports it.

Modules
-------
tables    1D Gauss-Lobatto-Legendre nodes, Gauss-Legendre quadrature, Lagrange basis
          (Section 2.2: Q_p elements, (p+1)^d Gauss points).
mesh      structured unit-cube hexahedral Q_p mesh, DoF numbering, Dirichlet sets.
material  compressible neo-Hookean energy Psi (Eq. hypref), first Piola stress
          P = dPsi/dF (Eq. F), tangent moduli L = dP/dF formed explicitly (Eq. L).
fem       residual (Eq. F), tangent application W_i = K(u; du, phi_i) (Eq. DF,
          Section 2.4) by the direct O((p+1)^6) route with an explicit L per point,
          element matrices, assembled global matrices, energy and the operator diagonal.
solver    Newton with load steps and direct linear solves on tiny meshes (Section 2.2).
unet      FP64 reference of the convolutional U-Net preconditioner (forward, backward).
"""
