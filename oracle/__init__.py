"""Plain, slow, FP64 CPU oracle for the two-sided Lanczos sign function and its
derivative (Puhr & Buividovich, "A method to compute derivatives of functions of
large complex matrices", Lattice 2016).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
benchmark's CPU-baseline / reference legs may import it.  It shares no code with the
CUDA path: it has its own gamma matrices, Gell-Mann table, stencil, Krylov recurrences
and matrix functions.  Every function cites the passage of the paper it follows, or
states the textbook definition it writes out where the paper only names the object.

Modules:
  dirac       -- H(mu) = gamma5 Dw(mu) (Eq. (1.1)), its adjoint and its derivatives
                 along mu and along su(3)/U(1) link directions; dense assembly.
  sign        -- exact matrix sign (ordered Schur + Sylvester; spectral; Newton) and
                 the Frechet derivative (Mathias block, Eq. (2.5); Sylvester route).
  tsl         -- the two-sided Lanczos approximation (Sec. 2) of sgn(A)x and, through
                 Eq. (2.6), of d_t sgn(A)x; the error estimate eps_A (Sec. 4).
  nested      -- the nested (one level) two-sided Lanczos evaluation of sgn(T_k) e_1 (Sec. 4).
  free_field  -- closed forms for U = 1 in momentum space (pins dirac and sign).
  deflation   -- standard (Eq. (3.1)) and generalised (Eqs. (3.2)-(3.4)) deflation.
  adjoint     -- the bilinear S = Re<y|sgn H|x> and its gradient (fermionic force).
"""
