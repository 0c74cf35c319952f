"""Oracle: the bilinear S = Re <y| sgn(H(mu)) |x> and its gradient (the fermionic force named
in Secs. 1 and 5 as a use of the method).

Test infrastructure only (see the package docstring).

Direction derivatives.  Along a link direction U_nu(x) -> exp(i t Omega) U_nu(x) the kernel
changes by E = dH/dt and dS/dt = Re y^H L_sgn(H, E) x, where L_sgn is the Frechet derivative
(Eq. (2.5)).  For a function analytic on the spectrum, tr(L(A, E) B) = tr(E L(A, B)), so all
directions follow from one matrix
    G = L_sgn(H, x y^H):   dS/dt = Re tr(E G).
Force components.  For the generator lambda_a/2 on link (x, nu) the kernel derivative E is the
hopping part of H through that link with U -> i (lambda_a/2) U (forward hop) and U^dag ->
-i U^dag (lambda_a/2) (backward hop); the force is the array F[nu][x][a] = dS/dw^a_nu(x).

Two routes are given:
  * grad_dense: G from the dense Sylvester Frechet route (oracle.sign), contracted with each
    link's E exactly.
  * grad_tsl: the Krylov approximation G ~ |x||y| V_1 X W_2^H, with V_1, T_1 from the TSL of
    Sec. 2 started at x, W_2, T_2 from the TSL started at y, and X the top-right block of
    sgn([[T_1, e_1 e_1^T], [0, T_2]]) (Eq. (2.5) applied to the projected block matrix, the
    reading used for the adjoint), evaluated with the dense Schur sign.
"""
import numpy as np

from . import dirac as od
from .sign import frechet_sylvester, sign_schur
from .tsl import tsl


def link_E(lat, U, nu, s, a, mu):
    """Dense dH/dw^a_nu(s) for the generator lambda_a/2 on the single link (s, nu)."""
    om = np.zeros((4, lat.V, 8))
    om[nu, s, a] = 1.0
    Y = od.link_derivative(U, omega=om)
    return od.dense_dH_dir(lat, U, Y, mu)


def force_from_G(lat, U, G, mu):
    """F[nu][s][a] = Re tr(E_{nu,s,a} G) for every link and generator, with E assembled per
    link from its two hops (independent of the stencil code: explicit block algebra)."""
    g, g5 = od.gammas()
    lam = od.gell_mann()
    I4 = np.eye(4)
    F = np.zeros((4, lat.V, 8))
    fwd = [1.0, 1.0, 1.0, np.exp(mu)]
    bwd = [1.0, 1.0, 1.0, np.exp(-mu)]
    for nu in range(4):
        for s in range(lat.V):
            sp, sgn = lat.neighbour(s, nu, +1)
            for a in range(8):
                dU = 1j * (lam[a] / 2) @ U[nu][s]               # d U_nu(s)
                dUd = dU.conj().T                                # d U_nu(s)^dag
                # forward hop s <- s+nu: block (s, sp) = -1/2 f+ sgn gamma5 (1 - g) (x) dU
                Bf = -0.5 * fwd[nu] * sgn * np.kron(g5 @ (I4 - g[nu]), dU)
                # backward hop sp <- s: block (sp, s) = -1/2 f- sgn gamma5 (1 + g) (x) dU^dag
                Bb = -0.5 * bwd[nu] * sgn * np.kron(g5 @ (I4 + g[nu]), dUd)
                # tr(E G) = sum_{ij} E_ij G_ji
                val = np.sum(Bf * G[12 * sp:12 * sp + 12, 12 * s:12 * s + 12].T)
                val += np.sum(Bb * G[12 * s:12 * s + 12, 12 * sp:12 * sp + 12].T)
                F[nu, s, a] = val.real
    return F


def dmu_from_G(lat, U, G, mu):
    """dS/dmu = Re tr(dH/dmu G)."""
    return np.real(np.sum(od.dense_dH_dmu(lat, U, mu) * G.T))


def bilinear(lat, U, x, y, mu):
    """S = Re <y| sgn(H) |x> with the dense Schur sign."""
    return np.real(np.vdot(y, sign_schur(od.dense_H(lat, U, mu)) @ x))


def grad_dense(lat, U, x, y, mu):
    """(S, F [4][V][8], dS/dmu) from G = L_sgn(H, x y^H) by the Sylvester route."""
    H = od.dense_H(lat, U, mu)
    x = np.asarray(x).ravel()
    y = np.asarray(y).ravel()
    G = frechet_sylvester(H, np.outer(x, y.conj()))
    S = np.real(np.vdot(y, sign_schur(H) @ x))
    return S, force_from_G(lat, U, G, mu), dmu_from_G(lat, U, G, mu)


def G_tsl(apply_A, apply_Ah, x, y, k):
    """G ~ |x||y| V_1 X W_2^H (see the module docstring).  Returns (G, S_tsl, record)."""
    x = np.asarray(x, dtype=complex).ravel()
    y = np.asarray(y, dtype=complex).ravel()
    nx, ny = np.linalg.norm(x), np.linalg.norm(y)
    r1 = tsl(apply_A, apply_Ah, x / nx, x / nx, k)
    r2 = tsl(apply_A, apply_Ah, y / ny, y / ny, k)
    k1, k2 = r1["T"].shape[0], r2["T"].shape[0]
    M = np.zeros((k1 + k2, k1 + k2), complex)
    M[:k1, :k1] = r1["T"]
    M[k1:, k1:] = r2["T"]
    M[0, k1] = 1.0
    X = sign_schur(M)[:k1, k1:]
    G = nx * ny * (r1["V"].T @ X @ r2["W"].conj())
    S1 = sign_schur(r1["T"])[:, 0]
    S = np.real(np.vdot(y, nx * (r1["V"].T @ S1)))
    return G, S, (r1, r2, X)


def grad_tsl(lat, U, x, y, mu, k):
    """(S, F, dS/dmu) from the Krylov approximation of G at depth k."""
    A = lambda v: od.apply_H(lat, U, v, mu).ravel()        # noqa: E731
    Ah = lambda v: od.apply_Hdag(lat, U, v, mu).ravel()    # noqa: E731
    G, S, rec = G_tsl(A, Ah, x, y, k)
    return S, force_from_G(lat, U, G, mu), dmu_from_G(lat, U, G, mu)
