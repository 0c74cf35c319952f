"""Oracle: the nested two-sided Lanczos approximation of the projected sign sgn(T_k) e_1.

Test infrastructure only (see the package docstring).

Sec. 4 evaluates the sign function with a nested version of the two-sided Lanczos method, one
level of nesting, inner Krylov subspace of size 100; the description of the nesting is in a
cited reference that is not at hand.  The reading used here:

  * the outer process (Sec. 2, oracle.tsl) yields the k x k tridiagonal T_k, and
    sgn(A) x ~ |x| V_k sgn(T_k) e_1;
  * the inner process is the same two-sided Lanczos recurrence, m steps from v_1 = w_1 = e_1, on
        M = T_k / c + c T_k^{-1},
    a function of T_k with the same sign: Re(z/c + c/z) = Re(z) (1/c + c/|z|^2) has the sign
    of Re z, so sgn(M) = sgn(T_k).  The map folds the eigenvalue magnitudes about c (|z| and
    c^2/|z| land on the same circle), halving the logarithmic range of magnitudes that the
    inner Krylov polynomial has to resolve; c = sqrt(|lambda|_min |lambda|_max) is the
    geometric centre of the spectrum of T_k.  Without the map the inner process on T_k from
    e_1 would only reproduce the leading m x m block of T_k (the outer process at depth m);
  * sgn(T_k) e_1 ~ V'_m sgn(T'_m) e_1 with the inner m x m projected matrix T'_m, whose sign is
    taken by the ordered Schur method (oracle.sign).
"""
import numpy as np

from .sign import sign_schur
from .tsl import tsl


def nested_scale(T):
    """c = sqrt(|lambda|_min |lambda|_max) over the eigenvalues of T (dense)."""
    lam = np.abs(np.linalg.eigvals(np.asarray(T, dtype=complex)))
    return float(np.sqrt(lam.min() * lam.max()))


def nested_operator(T, c, sign=1.0):
    """M = T / c + sign * c T^{-1} (sign = -1 only to plant a mistake in the tests)."""
    T = np.asarray(T, dtype=complex)
    return T / c + sign * c * np.linalg.inv(T)


def nested_sign_e1(T, m, c=None, sign=1.0, **kw):
    """sgn(T) e_1 by m steps of the inner two-sided Lanczos process on M = T/c + c T^{-1} from
    e_1.  Returns (approximation [k], inner record of oracle.tsl.tsl)."""
    T = np.asarray(T, dtype=complex)
    k = T.shape[0]
    c = nested_scale(T) if c is None else c
    M = nested_operator(T, c, sign)
    Mh = M.conj().T
    e1 = np.zeros(k, complex)
    e1[0] = 1.0
    r = tsl(lambda v: M @ v, lambda v: Mh @ v, e1, e1, min(m, k), **kw)
    s = sign_schur(r["T"])[:, 0]
    return r["V"].T @ s, r
