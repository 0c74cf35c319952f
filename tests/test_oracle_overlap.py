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


def test_axial_current_pins():
    """The conserved axial current Tr(D^{-1} dD gamma5) and its estimates, pinned by consequences
    of the Ginsparg-Wilson relation (m = 0: D^{-1} gamma5 + gamma5 D^{-1} = gamma5), the special
    mass m = 2 (D = 2, dD = 0) and the unit-vector sum of the estimator; a U(1) link direction."""
    mu = 0.3
    lat, U, D, g5 = _setup(mu)
    theta = syn.u1_direction(DIMS, 9)
    E = od.dense_dH_dir(lat, U, od.link_derivative(U, theta=theta), mu)
    dD = oo.overlap_derivative_dense(lat, U, mu, E)
    # Tr(gamma5 dD_ov) = d Tr sgn(H) = 0: the index does not change along a smooth direction
    assert abs(np.trace(g5 @ dD)) < 1e-10 * np.abs(dD).sum()
    J = oo.axial_current_trace(lat, U, mu, E)
    Di = np.linalg.inv(D)
    # GW: Tr(D^{-1} dD g5) = Tr(dD g5) - Tr(dD D^{-1} g5) = -Tr(D^{-1} g5 dD)
    Jr = np.trace(Di @ g5 @ dD)
    assert abs(J + Jr) < 1e-9 * max(abs(J), 1e-3)
    # a planted mistake (the gamma5 of dD_ov = gamma5 d sgn(H) dropped) breaks it
    dS = g5 @ dD
    Jb, Jrb = np.trace(Di @ dS @ g5), np.trace(Di @ g5 @ dS)
    assert abs(Jb + Jrb) > 1e-3 * abs(Jb)
    # m = 2: D(2) = 2 and dD(2) = 0
    assert np.allclose(oo.massive_overlap_dense(lat, U, mu, 2.0), 2 * np.eye(lat.n), atol=1e-12)
    assert abs(oo.axial_current_trace(lat, U, mu, E, 2.0)) < 1e-14
    # the estimator over all unit vectors sums to the trace (m = 0 and m = 0.2)
    for m in (0.0, 0.2):
        I = np.eye(lat.n).reshape(lat.n, lat.V, 4, 3)
        est = oo.axial_current_estimates(lat, U, mu, E, I, m)
        assert abs(est.sum() - oo.axial_current_trace(lat, U, mu, E, m)) < 1e-9 * np.abs(est).sum()
