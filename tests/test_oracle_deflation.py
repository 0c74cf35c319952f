"""Pins of the oracle's deflation (Sec. 3): Eq. (3.1) and the generalised deflation of
Eqs. (3.2)-(3.4) reproduce the exact sign exactly when the complement is treated exactly;
the Jordan vectors of Eq. (3.3) are biorthogonal and complete; B X = X J; the eigenvector
derivatives agree between the full eigen-sum, the projected-resolvent form and finite
differences."""
import numpy as np
import pytest

import synthetic as syn
from oracle import deflation as odf
from oracle import dirac as od
from oracle import sign as osg


@pytest.fixture(scope="module")
def case():
    dims, mu = (4, 2, 2, 2), 0.3
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.4, 3)
    A = od.dense_H(lat, U, mu)
    E = od.dense_dH_dmu(lat, U, mu)
    x = syn.gaussian_source(dims, 5).ravel()
    return lat, U, A, E, x, mu


def test_standard_deflation_exact(case):
    lat, U, A, E, x, mu = case
    S = osg.sign_schur(A)
    lam, R, L, full = odf.eigenpairs(A, 12)
    assert np.abs(L @ R - np.eye(12)).max() < 1e-10
    y = odf.sign_deflated(lambda v: S @ v, lam, R, L, x)
    assert np.linalg.norm(y - S @ x) < 1e-11
    # the deflated source has no component along the deflated eigenvectors
    assert np.abs(L @ odf.deflated_source(R, L, x)).max() < 1e-12


def test_eigen_derivatives_three_ways(case):
    lat, U, A, E, x, mu = case
    l = 6
    lam, R, L, full = odf.eigenpairs(A, l)
    order = np.argsort(np.abs(full[0]), kind="stable")[:l]
    d1 = odf.eigen_derivatives_full(full, E, order)
    d2 = odf.eigen_derivatives_projected(A, E, lam, R, L)
    for a, b in zip(d1, d2):
        assert np.abs(a - b).max() < 1e-9 * max(1.0, np.abs(a).max())
    dlam, dR, dL = d1
    # dlambda by central differences in mu
    h = 1e-6
    lp = np.linalg.eigvals(od.dense_H(lat, U, mu + h))
    lm = np.linalg.eigvals(od.dense_H(lat, U, mu - h))
    for i in range(l):
        fd = (lp[np.argmin(np.abs(lp - lam[i]))] - lm[np.argmin(np.abs(lm - lam[i]))]) / (2 * h)
        assert abs(fd - dlam[i]) < 1e-5 * max(1.0, abs(dlam[i]))
    # normalisation and the differentiated eigen-equations
    for i in range(l):
        assert abs(L[i] @ dR[:, i]) < 1e-10
        assert np.linalg.norm(A @ dR[:, i] + E @ R[:, i] - lam[i] * dR[:, i] - dlam[i] * R[:, i]) < 1e-9
        assert np.linalg.norm(dL[i] @ A + L[i] @ E - lam[i] * dL[i] - dlam[i] * L[i]) < 1e-9


def test_jordan_structure_and_generalised_deflation(case):
    lat, U, A, E, x, mu = case
    n = lat.n
    l = 6
    lam, R, L, full = odf.eigenpairs(A, l)
    dlam, dR, dL = odf.eigen_derivatives_projected(A, E, lam, R, L)
    X, Xb = odf.jordan_vectors(lam, R, L, dlam, dR, dL)
    assert np.abs(Xb @ X - np.eye(2 * l)).max() < 1e-9                   # biorthogonality
    B = np.block([[A, E], [np.zeros_like(A), A]])
    J = np.zeros((2 * l, 2 * l), complex)
    for i in range(l):
        J[2 * i, 2 * i] = J[2 * i + 1, 2 * i + 1] = lam[i]
        J[2 * i, 2 * i + 1] = 1.0
    assert np.abs(B @ X - X @ J).max() < 1e-9                              # Eq. (3.2)
    SB = odf.sign_block_exact(A, E)
    psi = np.concatenate([np.zeros(n), x])
    P, Pbar = odf.block_projections(R, L, dR, dL, psi)
    assert np.abs(P - X @ (Xb @ psi)).max() < 1e-10                       # product form = X Xbar
    y = odf.sign_block_deflated(lambda v: SB @ v, lam, R, L, dR, dL, psi)  # Eq. (3.4) for sgn
    assert np.linalg.norm(y - SB @ psi) < 1e-10
    # a general (non-sparse) block source as well
    psi2 = np.concatenate([syn.gaussian_source(lat.dims, 6).ravel(), x])
    y2 = odf.sign_block_deflated(lambda v: SB @ v, lam, R, L, dR, dL, psi2)
    assert np.linalg.norm(y2 - SB @ psi2) < 1e-10
    # completeness with all eigenpairs: sum_i X_i Xbar_i = 1 (Sec. 3)
    lamf, Rf, Lf = full
    ordf = np.arange(n)
    dlf, dRf, dLf = odf.eigen_derivatives_full(full, E, ordf)
    Xf, Xbf = odf.jordan_vectors(lamf, Rf, Lf, dlf, dRf, dLf)
    assert np.abs(Xf @ Xbf - np.eye(2 * n)).max() < 1e-8
