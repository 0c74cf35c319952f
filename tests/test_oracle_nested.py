"""Pins of the nested two-sided Lanczos projected sign (oracle.nested, Sec. 4): exact on an
invariant start vector, exact at full inner depth, convergent in the inner depth and faster than
the outer process truncated at the same depth, scale-independent in the limit; a sign mistake in
the folding map breaks it."""
import numpy as np
import pytest

import synthetic as syn
from oracle import nested as on
from oracle import sign as osg
from oracle import tsl as ot
from tests.helpers import oracle_ops, relerr


def _tridiag(rng, k, gap=0.3):
    """A non-normal tridiagonal with eigenvalues away from the imaginary axis."""
    a = (gap + np.abs(rng.standard_normal(k))) * np.where(rng.random(k) < 0.5, -1, 1) + 0.3j * rng.standard_normal(k)
    b = 0.3 * (rng.standard_normal(k - 1) + 1j * rng.standard_normal(k - 1))
    d = 0.3 * (rng.standard_normal(k - 1) + 1j * rng.standard_normal(k - 1))
    return np.diag(a) + np.diag(b, 1) + np.diag(d, -1)


def _exact(T):
    return osg.sign_schur(T)[:, 0]


def test_diagonal_start_is_invariant():
    """For diagonal T, e_1 is an eigenvector of M: the inner process stops at k_eff = 1 and the
    result is sign(Re t_11) e_1 exactly."""
    T = np.diag([-0.7 + 0.2j, 1.3, 0.4 - 1j, -2.0])
    s, r = on.nested_sign_e1(T, 4)
    assert r["k_eff"] == 1
    assert np.array_equal(s, np.array([-1, 0, 0, 0], complex))


def test_full_inner_depth_is_exact():
    rng = np.random.default_rng(1)
    T = _tridiag(rng, 40)
    s, r = on.nested_sign_e1(T, 40)
    assert relerr(s, _exact(T)) < 1e-10


def test_planted_sign_mistake_fails():
    """M = T/c - c T^{-1} flips the sign of the eigenvalues with |z| < c: wrong at any depth."""
    rng = np.random.default_rng(1)
    T = _tridiag(rng, 40)
    s, _ = on.nested_sign_e1(T, 40, sign=-1.0)
    assert relerr(s, _exact(T)) > 1e-2


def test_scale_only_moves_the_convergence():
    rng = np.random.default_rng(2)
    T = _tridiag(rng, 30)
    c = on.nested_scale(T)
    for f in (0.25, 4.0):
        s, _ = on.nested_sign_e1(T, 30, c=f * c)
        assert relerr(s, _exact(T)) < 1e-10


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_projected_matrix_of_the_wilson_kernel(mu):
    """T_64 of the oracle's process at 4^4: the nested error falls with the inner depth, and at
    every inner depth m it is below that of the outer process truncated at depth m (which is
    what an inner process on T_k itself, without the folding map, would give)."""
    dims, k = (4, 4, 4, 4), 64
    U = syn.gauge_field(dims, 0.4, 3)
    lat, A, Ah, E, Eh = oracle_ops(dims, U, mu)
    x = syn.gaussian_source(dims, 5).ravel()
    nx = np.linalg.norm(x)
    r = ot.tsl(A, Ah, x / nx, x / nx, k)
    T = r["T"]
    ex = _exact(T)
    errs = []
    for m in (8, 16, 24, 32):
        s, _ = on.nested_sign_e1(T, m)
        e = relerr(s, ex)
        trunc = np.zeros(k, complex)
        trunc[:m] = _exact(T[:m, :m])
        et = relerr(trunc, ex)
        print("mu %.1f m %d: nested %.3g, truncated outer %.3g" % (mu, m, e, et))
        assert e < et
        errs.append(e)
    assert errs[-1] < 1e-6 and all(b < a for a, b in zip(errs, errs[1:]))
