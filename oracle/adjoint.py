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


# ---- deflated adjoint ---------------------------------------------------------------------
# With the eigenpairs (lambda_i, R_i, L_i) of Sec. 3 (L_i R_j = delta_ij) the spectral projectors
# Pi = sum_i R_i L_i and Pbar = 1 - Pi commute with A, and in an eigenbasis the Frechet derivative
# is L_f(A, C) = X (F o X^{-1} C X) X^{-1} with F_ij = f[lambda_i, lambda_j], the divided
# differences (f'(lambda_i) on the diagonal; for sgn they vanish unless the signs differ).  Split
# by Pi / Pbar, with C = x y^H, c_i = L_i x, d_j = y^H R_j, x' = Pbar x, y' = Pbar^H y:
#   Pi G Pi     = sum_ij R_i F_ij c_i d_j L_j
#   Pi G Pbar   = sum_i  R_i c_i u_i^H,   u_i = g_i(A^H) y',  g_i(z) = (sgn lambda_i - sgn z) / (conj lambda_i - z)
#   Pbar G Pi   = sum_j  v_j d_j L_j,     v_j = h_j(A) x',    h_j(z) = (sgn z - sgn lambda_j) / (z - lambda_j)
#   Pbar G Pbar = L_f(A, x' y'^H)        (the undeflated Krylov route on the deflated sources)
# (z - lambda_j) is singular on the whole space (its null vector R_j lies in the deflated range),
# so v_j and u_i are projected by Pbar / Pbar^H after the solve: the exact ones lie in the
# complement, and the projection removes what rounding puts along the null directions.

def sign_divided_differences(lam):
    """F_ij = (sgn lambda_i - sgn lambda_j) / (lambda_i - lambda_j), 0 where the signs agree
    (sgn = sign of the real part; the diagonal, f' = 0 off the imaginary axis, is 0)."""
    lam = np.asarray(lam)
    s = np.sign(lam.real)
    F = np.zeros((len(lam), len(lam)), complex)
    for i in range(len(lam)):
        for j in range(len(lam)):
            if s[i] != s[j]:
                F[i, j] = (s[i] - s[j]) / (lam[i] - lam[j])
    return F


def G_deflated_parts(lam, R, L, x, y):
    """The deflated-space quantities: (c, d, F, x', y')."""
    x = np.asarray(x, dtype=complex).ravel()
    y = np.asarray(y, dtype=complex).ravel()
    c = L @ x
    d = y.conj() @ R
    xp = x - R @ c
    yp = y - L.conj().T @ d.conj()
    return c, d, sign_divided_differences(lam), xp, yp


def G_deflated_dense(A, lam, R, L, x, y):
    """G = L_sgn(A, x y^H) assembled from the four blocks with every function of A dense (the
    block identity itself, to be compared with the plain Sylvester route)."""
    c, d, F, xp, yp = G_deflated_parts(lam, R, L, x, y)
    n = A.shape[0]
    S = sign_schur(A)
    G = R @ (F * np.outer(c, d)) @ L
    I = np.eye(n)
    for i in range(len(lam)):
        si = np.sign(lam[i].real)
        u = np.linalg.solve(np.conj(lam[i]) * I - A.conj().T, si * yp - S.conj().T @ yp)
        v = np.linalg.solve(A - lam[i] * I, S @ xp - si * xp)
        u = u - L.conj().T @ (R.conj().T @ u)      # Pbar^H u
        v = v - R @ (L @ v)                        # Pbar v
        G += np.outer(R[:, i] * c[i], u.conj()) + np.outer(v * d[i], L[i])
    G += frechet_sylvester(A, np.outer(xp, yp.conj()))
    return G


def G_deflated_tsl(apply_A, apply_Ah, lam, R, L, x, y, k):
    """The same blocks with the Krylov approximations at depth k: the Pbar G Pbar block by G_tsl
    on (x', y'), and v_j, u_i from the same two Lanczos runs through the projected functions
    h_j(T_1) e_1 and g_i(T_2) e_1 (the right run is on A from x', the left one on A^H from y').
    Returns (G, S) with S = Re <y|sgn(A)|x> deflated by Eq. (3.1)."""
    c, d, F, xp, yp = G_deflated_parts(lam, R, L, x, y)
    Gk, Sk, (r1, r2, X) = G_tsl(apply_A, apply_Ah, xp, yp, k)
    nx, ny = np.linalg.norm(xp), np.linalg.norm(yp)
    T1, T2 = r1["T"], r2["T"]
    s1, s2 = sign_schur(T1)[:, 0], sign_schur(T2.conj().T)[:, 0]
    e1 = np.zeros(T1.shape[0]); e1[0] = 1.0
    f1 = np.zeros(T2.shape[0]); f1[0] = 1.0
    G = R @ (F * np.outer(c, d)) @ L + Gk
    for i in range(len(lam)):
        si = np.sign(lam[i].real)
        v = nx * (r1["V"].T @ np.linalg.solve(T1 - lam[i] * np.eye(len(e1)), s1 - si * e1))
        # the left run: W_2^H A = T_2 W_2^H, so A^H W_2 = W_2 T_2^H
        u = ny * (r2["W"].T @ np.linalg.solve(np.conj(lam[i]) * np.eye(len(f1)) - T2.conj().T, si * f1 - s2))
        u = u - L.conj().T @ (R.conj().T @ u)
        v = v - R @ (L @ v)
        G += np.outer(R[:, i] * c[i], u.conj()) + np.outer(v * d[i], L[i])
    y_ = np.asarray(y, dtype=complex).ravel()
    S = np.real(np.vdot(y_, R @ (np.sign(lam.real) * c))) + Sk + np.real(np.vdot(y_ - yp, nx * (r1["V"].T @ s1)))
    return G, S
