"""CPU oracle for the generalized shifted Green's-function solver.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, FP64 restatement of
what the solver computes, written from the paper (Hoshi et al., SC16,
arXiv:1609.08377, Sec. II-III) so that the CUDA path can be checked against it.
Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
it; the library itself never does, and it shares no code with the library.

Modules:
  dense   -- O1: dense complex LU of (z B - A) per shift (definition of G,
             Eq. EQ-SHIFT-EQ-J and EQ-EIG-X=GB); O2: the generalized
             eigendecomposition closed form (Eq. EQ-EIG-GREEN).
  krylov  -- O3: naive B-inner-product Lanczos with tridiagonal solves per
             shift (Sec. III-B, shared Krylov subspace for all shifts);
             O3': plain COCG on z B - A, one shift at a time;
             lanczos_batch: O3 over a batch of columns, whose sparse
             products, CG solves and pivoted tridiagonal solves run in
             plain C with OpenMP (o3_batch.c, built by build_c.py).
  density -- Fermi function (Eq. EQ-FD-FUNC) and the density matrix on the
             pattern by quadrature of Eq. EQ-DM-GREEN-FN; per-shift traces,
             the chemical potential for an electron count (bisection) and
             the ICOHP connectivity C_IJ (Sec. VII).
  projection-- the real-space projection of one column (Sec. III-B): the
             kappa-atom region, the restricted pencil, multiple Arnoldi on it.
  marnoldi-- the multiple Arnoldi projection of one column (Sec. III-B,
             Eq. EQ-LS-MULTIPLE): Ritz pairs of the pencil on
             K(A; e_j) + K(A; B^-1 e_j), G^(j) and rho^(j) by the analytic
             energy integral.
  mlp     -- the iteration-count regressor used by the column scheduler
             (forward, backward and Adam), in FP64.
  features-- per-column scheduler features.
"""
