"""Oracle: the massless overlap operator at finite density, Eq. (1.1) with lattice spacing 1,

    D_ov = 1 + gamma5 sgn(H(mu)),      H(mu) = gamma5 Dw(mu),

and its derivative along a direction of H, d D_ov = gamma5 d sgn(H) (the Frechet derivative of
Eq. (2.5)); the massive operator D(m) = (1 - m/2) D_ov + m, and the conserved axial current
Tr(D^{-1} dD gamma5) of the paper's conclusion with its per-vector stochastic estimates.  Test
infrastructure only (see the package docstring).  Dense FP64, from the ordered Schur sign and the
Sylvester Frechet route of oracle.sign.
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


def massive_overlap_dense(lat, U, mu, mass):
    """D(m) = (1 - m/2) D_ov + m, the overlap operator with a bare mass m (lattice spacing 1; the
    paper works at m = 0, where D(0) = D_ov of Eq. (1.1))."""
    return (1.0 - 0.5 * mass) * overlap_dense(lat, U, mu) + mass * np.eye(lat.n)


def axial_current_trace(lat, U, mu, E, mass=0.0):
    """Tr(D(m)^{-1} dD(m) gamma5) along the direction with dH = E (the conserved axial current of
    the paper's conclusion, summed over the links the direction moves), with dD(m) = (1 - m/2) d D_ov.
    Exact: the inverse and the trace of dense matrices."""
    D = massive_overlap_dense(lat, U, mu, mass)
    dD = (1.0 - 0.5 * mass) * overlap_derivative_dense(lat, U, mu, E)
    return np.trace(np.linalg.inv(D) @ dD @ gamma5_full(lat))


def axial_current_estimates(lat, U, mu, E, eta, mass=0.0):
    """The per-vector estimates eta_s^dag D(m)^{-1} dD(m) gamma5 eta_s of the trace above (an
    unbiased estimator when E[eta eta^dag] = 1, as for Z2 noise); eta: [nsrc][V][4][3].  Each one
    by a dense solve, not through the inverse."""
    D = massive_overlap_dense(lat, U, mu, mass)
    dD = (1.0 - 0.5 * mass) * overlap_derivative_dense(lat, U, mu, E)
    g5 = gamma5_full(lat)
    eta = np.asarray(eta).reshape(len(eta), -1)
    return np.array([np.vdot(e, np.linalg.solve(D, dD @ (g5 @ e))) for e in eta])
