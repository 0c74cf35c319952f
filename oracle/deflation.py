"""Oracle: deflation of the sign function (Sec. 3).

Test infrastructure only (see the package docstring).

Standard deflation, Eq. (3.1): with right/left eigenvectors R_i, L_i of A (L_i R_j = delta_ij)
for the l eigenvalues closest to zero,
    sgn(A) x = sum_{i<=l} sgn(lambda_i) R_i (L_i x) + sgn(A) Pbar_l x,   Pbar_l = 1 - sum R_i L_i.

Generalised deflation for the block matrix B = [[A, E], [0, A]] (Eqs. (3.2)-(3.4)): B has 2x2
Jordan blocks J_i = [[lambda_i, 1], [0, lambda_i]]; the columns of the transformation X
(Eq. (3.3)) are X_{2i-1} = (R_i, 0), X_{2i} = (dR_i, R_i) / dlambda_i, the rows of X^{-1} are
Xbar_{2i-1} = (L_i, dL_i), Xbar_{2i} = dlambda_i (0, L_i), with dlambda_i = L_i E R_i.  For
the sign the d_t f(lambda_i) terms of Eq. (3.4) vanish:
    sgn(B) psi = sgn(B) Pbar_{2l} psi + sum_{i<=l} sgn(lambda_i) (X_{2i-1} Xbar_{2i-1} + X_{2i} Xbar_{2i}) psi.
Products X_{2i} Xbar_{2i} are formed directly, so dlambda_i cancels (reading: a vanishing
dlambda_i is harmless).  For psi = (t, b):
    sum_i (X_{2i-1} Xbar_{2i-1} + X_{2i} Xbar_{2i}) psi
        = ( sum_i R_i (L_i t + dL_i b) + dR_i (L_i b),  sum_i R_i (L_i b) ).

Eigenvector derivatives (normalisation L_j dR_j = 0, so dL_j R_j = 0):
    dR_j = sum_{i != j} R_i (L_i E R_j) / (lambda_j - lambda_i),
    dL_j = sum_{i != j} (L_j E R_i) L_i / (lambda_j - lambda_i),
given here from the full eigen-decomposition (eigen_derivatives_full) and from the
projected-resolvent form of the end of Sec. 3 (eigen_derivatives_projected), read as
    sum_{i != j, all} R_i L_i/(lambda_j - lambda_i)
        = sum_{i <= l, i != j} R_i L_i/(lambda_j - lambda_i) + Pbar_l (lambda_j - A)^{-1} Pbar_l,
where the right-hand Pbar_l makes the singular shifted solve well defined.
"""
import numpy as np
import scipy.linalg as sla

from .sign import sign_schur


def eigenpairs(A, l):
    """The l eigenpairs of the dense A closest to zero by |lambda| (ties by index):
    (lam [l], R [n][l] columns, L [l][n] rows) with L R = 1 (rows of R^{-1} of the full basis)."""
    lam, Rfull = np.linalg.eig(np.asarray(A, dtype=complex))
    Lfull = np.linalg.inv(Rfull)
    order = np.argsort(np.abs(lam), kind="stable")
    idx = order[:l]
    return lam[idx], Rfull[:, idx], Lfull[idx, :], (lam, Rfull, Lfull)


def deflated_source(R, L, x):
    """Pbar_l x = x - sum_i R_i (L_i x)."""
    return x - R @ (L @ x)


def sign_deflated(sign_apply, lam, R, L, x):
    """Eq. (3.1) with an arbitrary approximation sign_apply(v) ~ sgn(A) v on the complement."""
    c = L @ x
    return R @ (np.sign(lam.real) * c) + sign_apply(x - R @ c)


def eigen_derivatives_full(full, E, idx_l):
    """(dlam [l], dR [n][l], dL [l][n]) for the eigenpairs idx_l from the full decomposition."""
    lam, Rf, Lf = full
    n = len(lam)
    dlam = np.empty(len(idx_l), complex)
    dR = np.empty((n, len(idx_l)), complex)
    dL = np.empty((len(idx_l), n), complex)
    ER = E @ Rf
    LE = Lf @ E
    for a, j in enumerate(idx_l):
        dlam[a] = Lf[j] @ ER[:, j]
        w = np.zeros(n, complex)
        mask = np.arange(n) != j
        w[mask] = 1.0 / (lam[j] - lam[mask])
        dR[:, a] = Rf @ (w * (Lf @ ER[:, j]))
        dL[a, :] = ((LE[j] @ Rf) * w) @ Lf
    return dlam, dR, dL


def eigen_derivatives_projected(A, E, lam, R, L):
    """The same derivatives from only the l eigenpairs plus shifted solves on the deflated
    complement (the projected-resolvent reading of the end of Sec. 3)."""
    n, l = R.shape
    P = np.eye(n) - R @ L                       # Pbar_l
    dlam = np.array([L[i] @ (E @ R[:, i]) for i in range(l)])
    dR = np.empty((n, l), complex)
    dL = np.empty((l, n), complex)
    for j in range(l):
        rj = E @ R[:, j]
        lj = L[j] @ E
        sR = np.zeros(n, complex)
        sL = np.zeros(n, complex)
        for i in range(l):
            if i != j:
                sR += R[:, i] * (L[i] @ rj) / (lam[j] - lam[i])
                sL += (lj @ R[:, i]) * L[i] / (lam[j] - lam[i])
        M = lam[j] * np.eye(n) - A
        # Pbar (lambda_j - A)^{-1} Pbar on the complement: least-squares solve of the
        # (singular) system restricted to range(Pbar), then projected
        z = np.linalg.lstsq(M, P @ rj, rcond=None)[0]
        sR += P @ z
        zl = np.linalg.lstsq(M.T, (lj @ P), rcond=None)[0]
        sL += zl @ P
        dR[:, j] = sR
        dL[j, :] = sL
    return dlam, dR, dL


def eigen_derivatives_tsl(apply_A, apply_Ah, apply_E, apply_Eh, lam, R, L, k):
    """The eigenvector derivatives with the shifted solves on the deflated complement done by
    the TSL approximation of the resolvent (oracle.tsl.tsl_resolvent) at depth k:
        dR_j = sum_{i != j} R_i (L_i E R_j)/(lambda_j - lambda_i) + Pbar z_j,
               z_j ~ (lambda_j - A)^{-1} Pbar E R_j,
        dL_j^H = sum_{i != j} conj((L_j E R_i)/(lambda_j - lambda_i)) L_i^H + Pbar^H z'_j,
               z'_j ~ (conj(lambda_j) - A^H)^{-1} Pbar^H E^H L_j^H.
    Returns (dlam [l], dR [n][l], dL [l][n])."""
    from .tsl import tsl_resolvent
    n, l = R.shape
    Lk = L.conj().T                                    # kets of the left eigenvectors
    ER = np.array([apply_E(R[:, j]) for j in range(l)]).T
    ELk = np.array([apply_Eh(Lk[:, j]) for j in range(l)]).T
    C = L @ ER                                         # C[i, j] = L_i E R_j
    dlam = np.diag(C).copy()
    dR = np.empty((n, l), complex)
    dL = np.empty((l, n), complex)
    for j in range(l):
        b = ER[:, j] - R @ (L @ ER[:, j])
        z, _ = tsl_resolvent(apply_A, apply_Ah, b, lam[j], k)
        z = z - R @ (L @ z)
        bl = ELk[:, j] - Lk @ (R.conj().T @ ELk[:, j])
        zl, _ = tsl_resolvent(apply_Ah, apply_A, bl, np.conj(lam[j]), k)
        zl = zl - Lk @ (R.conj().T @ zl)
        sR = z.copy()
        sL = zl.copy()
        for i in range(l):
            if i != j:
                sR += R[:, i] * C[i, j] / (lam[j] - lam[i])
                sL += Lk[:, i] * np.conj(C[j, i] / (lam[j] - lam[i]))
        dR[:, j] = sR
        dL[j, :] = sL.conj()
    return dlam, dR, dL


def jordan_vectors(lam, R, L, dlam, dR, dL):
    """Columns X_{2i-1}, X_{2i} and rows Xbar_{2i-1}, Xbar_{2i} of Eq. (3.3) (2n-vectors)."""
    n, l = R.shape
    X = np.zeros((2 * n, 2 * l), complex)
    Xb = np.zeros((2 * l, 2 * n), complex)
    for i in range(l):
        X[:n, 2 * i] = R[:, i]
        X[:n, 2 * i + 1] = dR[:, i] / dlam[i]
        X[n:, 2 * i + 1] = R[:, i] / dlam[i]
        Xb[2 * i, :n] = L[i]
        Xb[2 * i, n:] = dL[i]
        Xb[2 * i + 1, n:] = dlam[i] * L[i]
    return X, Xb


def block_projections(R, L, dR, dL, psi):
    """(P_{2l} psi, Pbar_{2l} psi) for psi = (t, b), in the product form that is independent
    of dlambda."""
    n = R.shape[0]
    t, b = psi[:n], psi[n:]
    cb = L @ b
    top = R @ (L @ t + dL @ b) + dR @ cb
    bot = R @ cb
    P = np.concatenate([top, bot])
    return P, psi - P


def sign_block_deflated(sign_block_apply, lam, R, L, dR, dL, psi):
    """Eq. (3.4) for the sign: sgn(B) Pbar psi + sum_i sgn(lambda_i) (X_{2i-1}Xbar_{2i-1} + X_{2i}Xbar_{2i}) psi.
    sign_block_apply(v) ~ sgn(B) v on the deflated complement."""
    n = R.shape[0]
    t, b = psi[:n], psi[n:]
    s = np.sign(lam.real)
    cb = L @ b
    top = R @ (s * (L @ t + dL @ b)) + dR @ (s * cb)
    bot = R @ (s * cb)
    _, Pbar = block_projections(R, L, dR, dL, psi)
    return np.concatenate([top, bot]) + sign_block_apply(Pbar)


def sign_block_exact(A, E):
    """sgn(B) for B = [[A, E], [0, A]] by the dense Schur oracle (Eq. (2.5))."""
    B = np.block([[A, E], [np.zeros_like(A), A]])
    return sign_schur(B)
