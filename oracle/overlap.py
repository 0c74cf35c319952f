"""Oracle: the massless overlap operator at finite density, Eq. (1.1) with lattice spacing 1,

    D_ov = 1 + gamma5 sgn(H(mu)),      H(mu) = gamma5 Dw(mu),

and its derivative along a direction of H, d D_ov = gamma5 d sgn(H) (the Frechet derivative of
Eq. (2.5)).  Test infrastructure only (see the package docstring).  Dense FP64, from the ordered
Schur sign and the Sylvester Frechet route of oracle.sign.
"""
import numpy as np

from . import dirac as od
from .sign import frechet_sylvester, sign_schur


def gamma5_full(lat):
    """gamma5 on the whole lattice: diag(1, 1, -1, -1) on spin, identity on site and colour."""
    _, g5 = od.gammas()
    return np.kron(np.eye(lat.V), np.kron(g5, np.eye(3)))


def overlap_dense(lat, U, mu):
    """D_ov (Eq. (1.1)) as a dense matrix."""
    H = od.dense_H(lat, U, mu)
    return np.eye(lat.n) + gamma5_full(lat) @ sign_schur(H)


def overlap_derivative_dense(lat, U, mu, E):
    """d D_ov along the direction with dH = E: gamma5 L_sgn(H, E)."""
    H = od.dense_H(lat, U, mu)
    return gamma5_full(lat) @ frechet_sylvester(H, E)


def overlap_apply(lat, U, mu, x, E=None):
    """(D_ov x, d D_ov x) for one source x [V][4][3] (the second None without E)."""
    x = np.asarray(x).ravel()
    y = overlap_dense(lat, U, mu) @ x
    dy = None if E is None else overlap_derivative_dense(lat, U, mu, E) @ x
    return y, dy
