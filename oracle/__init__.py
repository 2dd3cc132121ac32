"""Plain, slow FP64 CPU oracle for the SIPG operator of Krank, Fehn, Wall and
Kronbichler (arXiv:1607.01323).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py`` may import it. The product
path (the CUDA library and its Python binding) never imports, links or calls
anything here, and nothing here imports the product path.

What it computes is the plain definition of the discrete operators:

* ``basis``   -- 1D Gauss-Lobatto nodes (the nodal basis, Sec. 3.1) and Gauss
  rules with k+1 points (Sec. 5), Lagrange polynomials by the product formula.
* ``mesh``    -- structured hexahedral meshes, the analytic maps (affine box and
  the tanh wall-normal grading of Sec. 7.1) and their iso-parametric degree-k
  interpolation (Sec. 5).
* ``sipg``    -- element and face matrices of the symmetric interior-penalty
  Laplacian (Sec. 3.2 (ii)) and of the viscous Helmholtz operator in Laplace
  form (Sec. 3.2 (iii), Sec. 4.4), built by dense quadrature: every basis
  function is evaluated at every quadrature point, with no sum factorisation;
  the full 3x3 Jacobian of the mapping is used at every point, so nothing here
  assumes the separable structure that the GPU kernels exploit.
* ``solvers`` -- textbook CG / PCG / flexible CG and the Chebyshev iteration
  (Sec. 5.1).
* ``adjoint`` -- gradient of J = 1/2 |u - u_t|_M^2 with respect to a per-cell
  viscosity, from the assembled derivative dA/dnu_e.

Parity status: pinned. The pins live in ``tests/test_oracle_*.py``
(closed-form quadrature rules, penalty closed forms, symmetry, nullspace,
positive definiteness, brute force with a (k+3)-point rule, Galerkin
consistency for polynomial solutions, optimal L2 convergence, M M^-1 = I and
finite-difference gradients).
"""
