"""Pins of the oracle's bilinear gradient (the fermionic force): the trace-identity route
against per-link Frechet derivatives and central finite differences along random link
directions and in mu; the Krylov route converges to it."""
import numpy as np
import scipy.linalg as sla

import synthetic as syn
from oracle import adjoint as oad
from oracle import dirac as od
from oracle import sign as osg


def _setup(dims=(2, 2, 2, 2), seed=3):
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.4, seed)
    x = syn.gaussian_source(dims, 5).ravel()
    y = syn.gaussian_source(dims, 6).ravel()
    return lat, U, x, y, 0.3


def test_force_matches_per_link_frechet():
    lat, U, x, y, mu = _setup()
    S, F, dmu = oad.grad_dense(lat, U, x, y, mu)
    H = od.dense_H(lat, U, mu)
    rng = np.random.default_rng(0)
    for _ in range(6):
        nu, s, a = rng.integers(4), rng.integers(lat.V), rng.integers(8)
        E = oad.link_E(lat, U, nu, s, a, mu)
        ref = np.real(np.vdot(y, osg.frechet_sylvester(H, E) @ x))
        assert abs(F[nu, s, a] - ref) < 1e-10 * max(1.0, abs(ref))


def test_force_and_mu_derivative_vs_finite_differences():
    lat, U, x, y, mu = _setup()
    S, F, dmu = oad.grad_dense(lat, U, x, y, mu)
    h = 1e-5
    om = syn.su3_direction(lat.dims, 9)
    Om = od.su3_tangent(om)
    expo = lambda t: np.array([[sla.expm(1j * t * Om[d, s]) for s in range(lat.V)] for d in range(4)])  # noqa: E731
    Sp = oad.bilinear(lat, np.einsum("dsij,dsjk->dsik", expo(h), U), x, y, mu)
    Sm = oad.bilinear(lat, np.einsum("dsij,dsjk->dsik", expo(-h), U), x, y, mu)
    assert abs((Sp - Sm) / (2 * h) - np.sum(om * F)) < 1e-7
    Sp = oad.bilinear(lat, U, x, y, mu + h)
    Sm = oad.bilinear(lat, U, x, y, mu - h)
    assert abs((Sp - Sm) / (2 * h) - dmu) < 1e-7
    assert abs(S - oad.bilinear(lat, U, x, y, mu)) < 1e-13


def test_krylov_route_converges():
    lat, U, x, y, mu = _setup((4, 2, 2, 2))
    S, F, dmu = oad.grad_dense(lat, U, x, y, mu)
    errs = []
    for k in (80, 300):
        St, Ft, dmut = oad.grad_tsl(lat, U, x, y, mu, k)
        errs.append(np.linalg.norm(Ft - F) / np.linalg.norm(F))
    assert errs[1] < 0.01 * errs[0]
    assert errs[1] < 1e-3
