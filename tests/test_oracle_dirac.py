"""Pins of the oracle's Dirac operator (Sec. 1, Eq. (1.1)) against facts other than itself:
the Clifford algebra, the su(3) algebra, the free-field closed form in momentum space,
gamma5-hermiticity, gauge covariance and finite differences."""
import numpy as np
import pytest
import scipy.linalg as sla

import synthetic as syn
from oracle import dirac as od
from oracle import free_field as ff


def test_clifford_algebra():
    g, g5 = od.gammas()
    I4 = np.eye(4)
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2 * (m == n) * I4)
        assert np.allclose(g5 @ g[m] + g[m] @ g5, 0)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


def test_gell_mann_algebra():
    lam = od.gell_mann()
    for a in range(8):
        assert np.allclose(lam[a], lam[a].conj().T)
        assert abs(np.trace(lam[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(lam[a] @ lam[b]) - 2 * (a == b)) < 1e-14
    # [lambda_1, lambda_2] = 2 i f_123 lambda_3 with f_123 = 1; f_458 = sqrt(3)/2
    assert np.allclose(lam[0] @ lam[1] - lam[1] @ lam[0], 2j * lam[2])
    assert np.allclose(lam[3] @ lam[4] - lam[4] @ lam[3], 2j * (0.5 * lam[2] + np.sqrt(3) / 2 * lam[7]))


DIMS = [(4, 2, 3, 2), (3, 2, 1, 2), (2, 2, 2, 2)]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("mu", [0.0, 0.3, -0.45])
def test_stencil_matches_dense_assembly(dims, mu):
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.4, 1)
    x = syn.gaussian_source(dims, 2).ravel()
    H = od.dense_H(lat, U, mu)
    assert np.abs(H @ x - od.apply_H(lat, U, x, mu).ravel()).max() < 1e-14
    assert np.abs(H.conj().T @ x - od.apply_Hdag(lat, U, x, mu).ravel()).max() < 1e-14
    E = od.dense_dH_dmu(lat, U, mu)
    assert np.abs(E @ x - od.apply_dH_dmu(lat, U, x, mu).ravel()).max() < 1e-14
    assert np.abs(E.conj().T @ x - od.apply_dH_dmu_dag(lat, U, x, mu).ravel()).max() < 1e-14
    Y = od.link_derivative(U, omega=syn.su3_direction(dims, 3))
    Ed = od.dense_dH_dir(lat, U, Y, mu)
    assert np.abs(Ed @ x - od.apply_dH_dir(lat, U, Y, x, mu).ravel()).max() < 1e-14
    assert np.abs(Ed.conj().T @ x - od.apply_dH_dir_dag(lat, U, Y, x, mu).ravel()).max() < 1e-14


@pytest.mark.parametrize("dims", [(4, 4, 2, 2), (6, 2, 3, 4)])
@pytest.mark.parametrize("mu", [0.0, 0.3])
@pytest.mark.parametrize("apbc", [True, False])
def test_free_field_closed_form(dims, mu, apbc):
    lat = od.Lattice(dims, antiperiodic_t=apbc)
    U = np.tile(np.eye(3, dtype=complex), (4, lat.V, 1, 1))
    x = syn.gaussian_source(dims, 7)
    assert np.abs(od.apply_H(lat, U, x, mu) - ff.free_H(lat, x, mu)).max() < 1e-14


def test_free_field_spectrum():
    lat = od.Lattice((4, 2, 2, 2))
    U = np.tile(np.eye(3, dtype=complex), (4, lat.V, 1, 1))
    def key(z):
        z = np.asarray(z)
        return z[np.lexsort((np.round(z.imag, 8), np.round(z.real, 8)))]
    lam = key(np.linalg.eigvals(od.dense_H(lat, U, 0.3)))
    ref = key(np.repeat(ff.free_spectrum(lat, 0.3), 6))
    assert np.abs(lam - ref).max() < 1e-12


def test_gamma5_hermiticity():
    dims = (4, 2, 2, 2)
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.5, 4)
    assert np.abs(od.dense_H(lat, U, 0.37).conj().T - od.dense_H(lat, U, -0.37)).max() < 1e-15
    H0 = od.dense_H(lat, U, 0.0)
    assert np.abs(H0 - H0.conj().T).max() < 1e-15


def test_gauge_covariance():
    dims = (4, 2, 3, 2)
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.4, 5)
    g = syn.gauge_field(dims, 1.0, 6)[0]            # one SU(3) matrix per site
    x = syn.gaussian_source(dims, 8)
    Ug = np.empty_like(U)
    for nu in range(4):
        for s in range(lat.V):
            sp, _ = lat.neighbour(s, nu, +1)
            Ug[nu, s] = g[s] @ U[nu, s] @ g[sp].conj().T
    gx = np.einsum("sab,sib->sia", g, x)
    lhs = od.apply_H(lat, Ug, gx, 0.3)
    rhs = np.einsum("sab,sib->sia", g, od.apply_H(lat, U, x, 0.3))
    assert np.abs(lhs - rhs).max() < 1e-14


def test_derivative_operators_vs_finite_differences():
    dims = (4, 2, 2, 2)
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.4, 9)
    mu, h = 0.3, 1e-5
    E = od.dense_dH_dmu(lat, U, mu)
    fd = (od.dense_H(lat, U, mu + h) - od.dense_H(lat, U, mu - h)) / (2 * h)
    assert np.abs(E - fd).max() < 1e-9
    om = syn.su3_direction(dims, 10)
    Om = od.su3_tangent(om)
    Y = od.link_derivative(U, omega=om)
    Ep = np.einsum("dsij,dsjk->dsik", np.array([[sla.expm(1j * h * Om[d, s]) for s in range(lat.V)] for d in range(4)]), U)
    Em = np.einsum("dsij,dsjk->dsik", np.array([[sla.expm(-1j * h * Om[d, s]) for s in range(lat.V)] for d in range(4)]), U)
    fd = (od.dense_H(lat, Ep, mu) - od.dense_H(lat, Em, mu)) / (2 * h)
    assert np.abs(od.dense_dH_dir(lat, U, Y, mu) - fd).max() < 1e-9
    th = syn.u1_direction(dims, 11)
    Yu = od.link_derivative(U, theta=th)
    Up = np.exp(1j * h * th)[:, :, None, None] * U
    Um = np.exp(-1j * h * th)[:, :, None, None] * U
    fd = (od.dense_H(lat, Up, mu) - od.dense_H(lat, Um, mu)) / (2 * h)
    assert np.abs(od.dense_dH_dir(lat, U, Yu, mu) - fd).max() < 1e-9


def test_synthetic_gauge_is_su3():
    U = syn.gauge_field((2, 2, 2, 2), 0.4, 1)
    assert np.abs(np.einsum("dsij,dskj->dsik", U, U.conj()) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
