"""The nested two-sided Lanczos projected sign (LQ_PROJ_NESTED, Sec. 4) against the oracle
(oracle.nested): element by element at the same inner depth and scale on seeded tridiagonal
matrices of the Lanczos form (real positive sub-diagonal), exact at full inner depth, and inside
the sign solve against the oracle's same-depth process with the exact projected sign."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import nested as on
from oracle import sign as osg
from oracle import tsl as ot
from tests.helpers import FP64_SENS_FACTOR, oracle_ops, relerr

pytestmark = pytest.mark.gpu


def _tridiags(seed, nb, k):
    """nb non-normal tridiagonals of the Lanczos form with eigenvalues off the imaginary axis."""
    rng = np.random.default_rng(seed)
    al = (0.3 + np.abs(rng.standard_normal((nb, k)))) * np.where(rng.random((nb, k)) < 0.5, -1, 1) \
        + 0.3j * rng.standard_normal((nb, k))
    be = 0.3 * (rng.standard_normal((nb, k - 1)) + 1j * rng.standard_normal((nb, k - 1)))
    de = 0.3 * np.abs(rng.standard_normal((nb, k - 1))) + 0.05
    return al, be, de


def _dense(al, be, de):
    return np.diag(al) + np.diag(be, 1) + np.diag(de.astype(complex), -1)


@pytest.mark.parametrize("m", [8, 20, 40])
def test_nested_sign_parity(lqlib, m):
    from paper_1611_00195_gb300 import lq
    nb, k = 3, 60
    al, be, de = _tridiags(11, nb, k)
    T = [_dense(al[b], be[b], de[b]) for b in range(nb)]
    c = np.array([on.nested_scale(t) for t in T])
    ctx = lq.Context((2, 2, 2, 2))
    ctx.reserve(k, nb, False)
    s, chk = ctx.nested_sign(al, be, de, m, scale=c)
    rng = np.random.default_rng(5)
    for b in range(nb):
        ref, _ = on.nested_sign_e1(T[b], m, c=c[b])
        Tp = T[b] * (1 + 1e-16 * rng.standard_normal(T[b].shape))
        sens = relerr(on.nested_sign_e1(Tp, m, c=c[b])[0], ref)
        err = relerr(s[b], ref)
        ex = relerr(s[b], osg.sign_schur(T[b])[:, 0])
        print("nested m=%d matrix %d: parity %.3g (oracle sensitivity %.3g); vs exact %.3g, involution residual %.3g"
              % (m, b, err, sens, ex, chk[b]))
        assert err < max(1e-12, FP64_SENS_FACTOR * sens)
        # the involution residual tracks the error against the exact sign
        assert chk[b] > 0.1 * ex or ex < 1e-12


def test_nested_sign_full_depth_is_exact(lqlib):
    from paper_1611_00195_gb300 import lq
    nb, k = 2, 48
    al, be, de = _tridiags(12, nb, k)
    ctx = lq.Context((2, 2, 2, 2))
    ctx.reserve(k, nb, False)
    s, chk = ctx.nested_sign(al, be, de, k)       # the library's own scale estimate
    for b in range(nb):
        T = _dense(al[b], be[b], de[b])
        e = relerr(s[b], osg.sign_schur(T)[:, 0])
        print("nested full depth matrix %d: %.3g vs exact, involution residual %.3g" % (b, e, chk[b]))
        assert e < 1e-10 and chk[b] < 1e-10


@pytest.mark.parametrize("deriv", [False, True])
def test_nested_projected_sign_in_the_solve(lqlib, deriv):
    """sgn(H) x and d/dmu at 4^4, k = 64 with the projected sign by the nested process at full
    inner depth (= k, where it is exact): the same-depth parity bound of the Schur-based oracle."""
    from paper_1611_00195_gb300 import lq
    dims, k, mu, nsrc = (4, 4, 4, 4), 64, 0.3, 2
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5, nsrc=nsrc)
    c = lq.Context(dims, mu=mu, precision=lq.LQ_FP64)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, nsrc, True)
    xt = torch.from_numpy(x).cuda()
    if deriv:
        ys, yd, rep = c.sign_derivative_apply(xt, k, projected=lq.LQ_PROJ_NESTED, nested_m=k)
        got = [yd.cpu().numpy(), ys.cpu().numpy()]
    else:
        ys, rep = c.sign_apply(xt, k, projected=lq.LQ_PROJ_NESTED, nested_m=k)
        got = [ys.cpu().numpy()]
    lat, A, Ah, E, Eh = oracle_ops(dims, U, mu)
    rng = np.random.default_rng(99)

    def run(v):
        if deriv:
            return list(ot.tsl_sign_derivative(A, Ah, E, Eh, v, k)[:2])
        return [ot.tsl_sign(A, Ah, v, k)[0]]
    for s in range(nsrc):
        assert rep[s]["projected"] == lq.LQ_PROJ_NESTED and rep[s]["status"] == 0, rep[s]
        assert rep[s]["proj_check"] < 1e-10
        ref = run(x[s].ravel())
        xp = x[s].ravel() * (1 + 1e-16 * rng.standard_normal(x[s].size))
        sens = max(relerr(p, q) for p, q in zip(run(xp), ref))
        errs = [relerr(g[s], r) for g, r in zip(got, ref)]
        print("nested projected sign in the solve, deriv %d source %d: %s (sensitivity %.3g), check %.3g"
              % (deriv, s, ["%.3g" % e for e in errs], sens, rep[s]["proj_check"]))
        assert max(errs) < max(1e-11, FP64_SENS_FACTOR * sens) + 10 * rep[s]["proj_check"]
