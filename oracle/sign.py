"""Oracle: the matrix sign function and its Frechet derivative, dense FP64.

Test infrastructure only (see the package docstring).

Definitions (Sec. 2):
  * f(A) = X f(J) X^{-1} through the Jordan form (Eqs. (2.1)-(2.4)); for a
    diagonalisable A the spectral form X diag(f(lambda)) X^{-1}.  For the sign function
    sgn(lambda) = sign(Re lambda); it is undefined on the imaginary axis, the branch cut
    named in Sec. 3.
  * The derivative of f(A(t)) along t is the top-right block of f applied to the block
    matrix B = [[A, dA], [0, A]] (Mathias' theorem, Eq. (2.5)).

Three independent evaluations of sgn are given (ordered Schur + Sylvester, spectral,
scaled Newton) and two of the derivative (Mathias block, Sylvester equations in the
block-diagonalised sign basis).  The tests pin them against each other, against the
free-field closed form and against finite differences.
"""
import numpy as np
import scipy.linalg as sla


def sign_schur(A):
    """sgn(A) from the ordered complex Schur form A = Q T Q^H (eigenvalues with
    Re > 0 first): sgn(T) = [[I, Z], [0, -I]] with T11 Z - Z T22 = 2 T12, which is
    the unique Z making sgn(T) commute with T.  (Schur method, Higham 2008 ch. 5.)"""
    A = np.asarray(A, dtype=complex)
    n = A.shape[0]
    T, Q, sdim = sla.schur(A, output="complex", sort="rhp")
    S = np.zeros((n, n), complex)
    p = sdim
    S[:p, :p] = np.eye(p)
    S[p:, p:] = -np.eye(n - p)
    if 0 < p < n:
        Z = sla.solve_sylvester(T[:p, :p], -T[p:, p:], 2 * T[:p, p:])
        S[:p, p:] = Z
    return Q @ S @ Q.conj().T


def sign_eig(A):
    """Spectral form X diag(sign(Re lambda)) X^{-1} (diagonalisable A only)."""
    lam, X = np.linalg.eig(np.asarray(A, dtype=complex))
    return (X * np.sign(lam.real)) @ np.linalg.inv(X)


def sign_newton(A, tol=1e-14, max_iter=100):
    """Scaled Newton iteration X <- (m X + (m X)^{-1}) / 2 with Frobenius-norm scaling
    m = sqrt(||X^{-1}||_F / ||X||_F) (Higham 2008 ch. 5)."""
    X = np.asarray(A, dtype=complex).copy()
    for _ in range(max_iter):
        Xi = np.linalg.inv(X)
        m = np.sqrt(np.linalg.norm(Xi) / np.linalg.norm(X))
        Xn = 0.5 * (m * X + Xi / m)
        if np.linalg.norm(Xn - X) <= tol * np.linalg.norm(Xn):
            return Xn
        X = Xn
    return X


def frechet_mathias(A, E, sign=sign_schur):
    """d_t sgn(A(t)) with dA/dt = E: the top-right n x n block of sgn([[A, E], [0, A]]) (Eq. (2.5))."""
    A = np.asarray(A, dtype=complex)
    n = A.shape[0]
    B = np.block([[A, E], [np.zeros_like(A), A]])
    return sign(B)[:n, n:]


def frechet_sylvester(A, E):
    """Frechet derivative L of sgn at A along E from differentiating S^2 = 1 and
    A S = S A:  S L + L S = 0 and A L - L A = S E - E S.  In a basis W that
    block-diagonalises A = W diag(A+, A-) W^{-1} (spectra right/left of the imaginary
    axis) this leaves only the off-diagonal blocks, each a Sylvester equation:
      A+ L+- - L+- A- =  2 E+-,   A- L-+ - L-+ A+ = -2 E-+."""
    A = np.asarray(A, dtype=complex)
    n = A.shape[0]
    T, Q, p = sla.schur(A, output="complex", sort="rhp")
    # decouple the Schur blocks: [[I, Y], [0, I]]^{-1} T [[I, Y], [0, I]] is block diagonal
    # when T11 Y - Y T22 = -T12.
    Y = sla.solve_sylvester(T[:p, :p], -T[p:, p:], -T[:p, p:])
    M = np.eye(n, dtype=complex)
    M[:p, p:] = Y
    Minv = np.eye(n, dtype=complex)
    Minv[:p, p:] = -Y
    W = Q @ M
    Winv = Minv @ Q.conj().T
    Ap, Am = T[:p, :p], T[p:, p:]
    Et = Winv @ np.asarray(E, dtype=complex) @ W
    Lt = np.zeros((n, n), complex)
    Lt[:p, p:] = sla.solve_sylvester(Ap, -Am, 2 * Et[:p, p:])
    Lt[p:, :p] = sla.solve_sylvester(Am, -Ap, -2 * Et[p:, :p])
    return W @ Lt @ Winv
