"""Pins of the oracle's matrix sign and Frechet derivative (Sec. 2, Eqs. (2.3)-(2.5)):
three independent sign algorithms, the involution and commutation identities, the
Hermitian case against eigh, the free-field closed form, and central differences."""
import numpy as np
import pytest

import synthetic as syn
from oracle import dirac as od
from oracle import free_field as ff
from oracle import sign as osg


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_three_sign_algorithms_agree(seed):
    A = _rand(30, seed)
    S = osg.sign_schur(A)
    assert np.abs(S - osg.sign_eig(A)).max() < 1e-11
    assert np.abs(S - osg.sign_newton(A)).max() < 1e-11
    assert np.abs(S @ S - np.eye(30)).max() < 1e-11
    assert np.abs(A @ S - S @ A).max() < 1e-11


def test_sign_of_wilson_kernel_identities():
    dims = (4, 2, 2, 2)
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.4, 3)
    H = od.dense_H(lat, U, 0.3)
    S = osg.sign_schur(H)
    assert np.abs(S @ S - np.eye(lat.n)).max() < 1e-11
    assert np.abs(H @ S - S @ H).max() < 1e-11
    # mu = 0: H is Hermitian, sgn(H) from its eigendecomposition
    H0 = od.dense_H(lat, U, 0.0)
    w, Q = np.linalg.eigh(H0)
    assert np.abs(osg.sign_schur(H0) - (Q * np.sign(w)) @ Q.conj().T).max() < 1e-11


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_free_field_sign_and_mu_derivative(mu):
    dims = (4, 2, 2, 2)
    lat = od.Lattice(dims)
    U = np.tile(np.eye(3, dtype=complex), (4, lat.V, 1, 1))
    x = syn.gaussian_source(dims, 4).ravel()
    H = od.dense_H(lat, U, mu)
    assert np.abs(osg.sign_schur(H) @ x - ff.free_sign(lat, x, mu).ravel()).max() < 1e-12
    L = osg.frechet_sylvester(H, od.dense_dH_dmu(lat, U, mu))
    assert np.abs(L @ x - ff.free_sign_dmu(lat, x, mu).ravel()).max() < 1e-12


def test_frechet_routes_agree_with_finite_differences():
    A = _rand(20, 5)
    E = _rand(20, 6)
    L1 = osg.frechet_mathias(A, E)
    L2 = osg.frechet_sylvester(A, E)
    h = 1e-5
    L3 = (osg.sign_schur(A + h * E) - osg.sign_schur(A - h * E)) / (2 * h)
    scale = np.abs(L1).max()
    assert np.abs(L1 - L2).max() < 1e-10 * scale
    assert np.abs(L1 - L3).max() < 1e-6 * scale


def test_mathias_block_structure():
    """Eq. (2.5): the diagonal blocks of f(B) equal f(A) and the lower-left block vanishes."""
    A = _rand(15, 7)
    E = _rand(15, 8)
    B = np.block([[A, E], [np.zeros_like(A), A]])
    SB = osg.sign_schur(B)
    S = osg.sign_schur(A)
    assert np.abs(SB[:15, :15] - S).max() < 1e-10
    assert np.abs(SB[15:, 15:] - S).max() < 1e-10
    assert np.abs(SB[15:, :15]).max() < 1e-10


def test_derivative_of_wilson_sign_vs_mu_differences():
    dims = (4, 2, 2, 1)
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.4, 12)
    mu, h = 0.3, 1e-5
    L = osg.frechet_mathias(od.dense_H(lat, U, mu), od.dense_dH_dmu(lat, U, mu))
    fd = (osg.sign_schur(od.dense_H(lat, U, mu + h)) - osg.sign_schur(od.dense_H(lat, U, mu - h))) / (2 * h)
    assert np.abs(L - fd).max() < 1e-6 * np.abs(L).max()
