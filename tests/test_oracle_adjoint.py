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


def test_deflated_adjoint_blocks():
    """The deflated adjoint: the four-block assembly of G = L_sgn(H, x y^H) from l eigenpairs
    (divided differences on the deflated space, the two mixed blocks through the functions
    (sgn z - sgn lambda) / (z - lambda), the Krylov route on the deflated sources) equals the plain
    Sylvester Frechet derivative, exactly with dense functions and in the limit with the Krylov
    ones; S deflated by Eq. (3.1) equals the bilinear.  A planted mistake (the left functions
    taken without the conjugate shift) breaks the identity."""
    from oracle import deflation as odf
    dims, mu, l = (2, 2, 2, 2), 0.3, 6
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.4, 3)
    H = od.dense_H(lat, U, mu)
    x = syn.gaussian_source(dims, 5).ravel()
    y = syn.gaussian_source(dims, 6).ravel()
    G0 = osg.frechet_sylvester(H, np.outer(x, y.conj()))
    lam, R, L, _ = odf.eigenpairs(H, l)
    Gd = oad.G_deflated_dense(H, lam, R, L, x, y)
    assert np.abs(Gd - G0).max() < 1e-11 * np.abs(G0).max()
    # planted mistake: g_i with lambda_i instead of conj(lambda_i)
    c, d, F, xp, yp = oad.G_deflated_parts(lam, R, L, x, y)
    S = osg.sign_schur(H)
    bad = R @ (F * np.outer(c, d)) @ L + osg.frechet_sylvester(H, np.outer(xp, yp.conj()))
    for i in range(l):
        si = np.sign(lam[i].real)
        u = np.linalg.solve(lam[i] * np.eye(lat.n) - H.conj().T, si * yp - S.conj().T @ yp)
        v = np.linalg.solve(H - lam[i] * np.eye(lat.n), S @ xp - si * xp)
        u, v = u - L.conj().T @ (R.conj().T @ u), v - R @ (L @ v)
        bad += np.outer(R[:, i] * c[i], u.conj()) + np.outer(v * d[i], L[i])
    assert np.abs(bad - G0).max() > 1e-6 * np.abs(G0).max()
    # the Krylov blocks converge to it; S and the force follow
    A = lambda v: od.apply_H(lat, U, v, mu).ravel()        # noqa: E731
    Ah = lambda v: od.apply_Hdag(lat, U, v, mu).ravel()    # noqa: E731
    errs = []
    for k in (60, 120, 180):
        Gk, Sk = oad.G_deflated_tsl(A, Ah, lam, R, L, x, y, k)
        errs.append(np.abs(Gk - G0).max() / np.abs(G0).max())
    Sd, Fd, dmud = oad.grad_dense(lat, U, x, y, mu)
    assert errs[-1] < 1e-6 and errs[-1] < errs[0]
    assert abs(Sk - Sd) < 1e-8 * abs(Sd)
    Fk = oad.force_from_G(lat, U, Gk, mu)
    assert np.linalg.norm(Fk - Fd) < 1e-6 * np.linalg.norm(Fd)
    assert abs(oad.dmu_from_G(lat, U, Gk, mu) - dmud) < 1e-6 * abs(dmud)
