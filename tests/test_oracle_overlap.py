"""Pins of the overlap oracle (Eq. (1.1)) against facts it must satisfy, independent of how it
is coded: the Ginsparg-Wilson relation (holds for any mu once sgn^2 = 1), the circle spectrum at
mu = 0, the differentiated Ginsparg-Wilson relation, and central differences in mu."""
import numpy as np

import synthetic as syn
from oracle import dirac as od
from oracle import overlap as oo

DIMS = (2, 2, 2, 2)


def _setup(mu):
    lat = od.Lattice(DIMS)
    U = syn.gauge_field(DIMS, 0.4, 3)
    return lat, U, oo.overlap_dense(lat, U, mu), oo.gamma5_full(lat)


def test_ginsparg_wilson_relation():
    """gamma5 D + D gamma5 = D gamma5 D for D = 1 + gamma5 S, S^2 = 1 (mu = 0.3 and 0)."""
    for mu in (0.3, 0.0):
        lat, U, D, g5 = _setup(mu)
        lhs = g5 @ D + D @ g5
        rhs = D @ g5 @ D
        assert np.abs(lhs - rhs).max() < 1e-11 * np.abs(D).max()
        # a planted mistake breaks it: 1 + sgn(H), the gamma5 dropped (g5 (D - 1) = sgn(H))
        D_bad = np.eye(lat.n) + g5 @ (D - np.eye(lat.n))
        assert np.abs(g5 @ D_bad + D_bad @ g5 - D_bad @ g5 @ D_bad).max() > 1e-3


def test_circle_spectrum_at_zero_mu():
    """At mu = 0, H is Hermitian, gamma5 sgn(H) is unitary, and the spectrum of D_ov lies on
    the circle |z - 1| = 1."""
    lat, U, D, g5 = _setup(0.0)
    ev = np.linalg.eigvals(D)
    assert np.abs(np.abs(ev - 1.0) - 1.0).max() < 1e-10


def test_derivative_ginsparg_wilson_and_fd():
    """d D satisfies the differentiated relation, and equals central differences of D in mu."""
    mu, h = 0.3, 1e-4
    lat, U, D, g5 = _setup(mu)
    E = od.dense_dH_dmu(lat, U, mu)
    dD = oo.overlap_derivative_dense(lat, U, mu, E)
    lhs = g5 @ dD + dD @ g5
    rhs = dD @ g5 @ D + D @ g5 @ dD
    assert np.abs(lhs - rhs).max() < 1e-9 * np.abs(dD).max()
    fd = (oo.overlap_dense(lat, U, mu + h) - oo.overlap_dense(lat, U, mu - h)) / (2 * h)
    assert np.abs(fd - dD).max() < 1e-6 * np.abs(dD).max()


def test_apply_matches_matrix():
    lat, U, D, g5 = _setup(0.3)
    x = syn.gaussian_source(DIMS, 5, nsrc=1)[0]
    E = od.dense_dH_dmu(lat, U, 0.3)
    y, dy = oo.overlap_apply(lat, U, 0.3, x, E)
    assert np.allclose(y, D @ x.ravel(), rtol=0, atol=1e-13)
    assert np.allclose(dy, oo.overlap_derivative_dense(lat, U, 0.3, E) @ x.ravel(), rtol=0, atol=1e-12)
