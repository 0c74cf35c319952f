"""GPU parity of the projected Newton sign and of the full two-sided Lanczos path (sign and
derivative, Sec. 2, Eqs. (2.5)-(2.6)) against the CPU oracle at the same Krylov depth."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import sign as osg
from oracle import tsl as ot
from tests.helpers import oracle_ops, relerr

pytestmark = pytest.mark.gpu


def _rand_matrix(rng, k, gap=1.0):
    # eigenvalues kept off the imaginary axis: A = Q diag(+-(gap + |z|)) Q^-1 + small noise
    lam = (gap + np.abs(rng.standard_normal(k))) * np.where(rng.random(k) < 0.5, -1, 1) + 0.3j * rng.standard_normal(k)
    Q = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)) + 3 * np.eye(k)
    return Q @ np.diag(lam) @ np.linalg.inv(Q)


@pytest.mark.parametrize("k", [1, 2, 7, 40, 130])
def test_newton_sign_dense(lqlib, k):
    from paper_1611_00195_gb300 import lq
    rng = np.random.default_rng(k)
    nb = 3
    X = np.stack([_rand_matrix(rng, k) for _ in range(nb)])
    c = lq.Context((2, 2, 2, 2))
    c.reserve(max(k, 2), nb, False)
    S, iters = c.newton_sign(torch.from_numpy(X).cuda())
    S = S.cpu().numpy()
    for b in range(nb):
        ref = osg.sign_schur(X[b])
        assert relerr(S[b], ref) < 1e-11, (b, iters)
        assert iters[b] < 30


def _sensitivity(run, x):
    """Relative change of the oracle's own result when its input is perturbed by 1e-16
    (relative, random): the rounding amplification of the non-symmetric Lanczos process at
    this depth.  Two correct FP64 implementations cannot agree better than about this."""
    rng = np.random.default_rng(99)
    xp = x * (1 + 1e-16 * rng.standard_normal(x.shape))
    a, b = run(x), run(xp)
    return max(relerr(bb, aa) for aa, bb in zip(a, b))


def _parity_tol(sens):
    return max(1e-11, 30.0 * sens)


CASES = [((4, 4, 4, 4), 64, 1), ((3, 2, 2, 2), 40, 3), ((6, 3, 5, 2), 50, 2)]


@pytest.mark.parametrize("dims,k,nsrc", CASES)
def test_sign_apply_fp64_parity(lqlib, dims, k, nsrc):
    from paper_1611_00195_gb300 import lq
    mu = 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5, nsrc=nsrc)
    c = lq.Context(dims, mu=mu, precision=lq.LQ_FP64)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, nsrc, False)
    y, rep = c.sign_apply(torch.from_numpy(x).cuda(), k)
    y = y.cpu().numpy()
    lat, A, Ah, E, Eh = oracle_ops(dims, U, mu)
    for s in range(nsrc):
        ref, r = ot.tsl_sign(A, Ah, x[s], k)
        assert rep[s]["status"] == 0 and rep[s]["k_eff"] == k
        # the recurrence itself: early coefficients agree to rounding
        al, be, de = c.tsl_coefficients(s, k)
        m = min(k, 12)
        assert np.abs(al[:m] - r["alpha"][:m]).max() < 1e-12 * np.abs(r["alpha"][:m]).max()
        assert np.abs(de[:m - 1] - r["delta"][:m - 1]).max() < 1e-12 * np.abs(r["delta"][:m - 1]).max()
        assert np.abs(be[:m - 1] - r["beta"][:m - 1]).max() < 1e-12 * np.abs(r["beta"][:m - 1]).max()
        sens = _sensitivity(lambda v: [ot.tsl_sign(A, Ah, v, k)[0]], x[s].ravel())
        err = relerr(y[s], ref)
        print("sign parity k=%d: rel err %.3g, oracle self-sensitivity %.3g" % (k, err, sens))
        assert err < _parity_tol(sens)


@pytest.mark.parametrize("dims,k,nsrc", CASES)
@pytest.mark.parametrize("kind", [0, 1])
def test_sign_derivative_fp64_parity(lqlib, dims, k, nsrc, kind):
    from paper_1611_00195_gb300 import lq
    mu = 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5, nsrc=nsrc)
    field = syn.su3_direction(dims, 77) if kind == 1 else None
    c = lq.Context(dims, mu=mu, precision=lq.LQ_FP64)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, nsrc, True)
    ys, yd, rep = c.sign_derivative_apply(torch.from_numpy(x).cuda(), k, kind=kind,
                                          field=None if field is None else torch.from_numpy(field).cuda())
    ys, yd = ys.cpu().numpy(), yd.cpu().numpy()
    lat, A, Ah, E, Eh = oracle_ops(dims, U, mu, kind, field)
    for s in range(nsrc):
        rd, rs, r = ot.tsl_sign_derivative(A, Ah, E, Eh, x[s], k)
        assert rep[s]["status"] == 0 and rep[s]["k_eff"] == k
        al, be, de = c.tsl_coefficients(s, k)
        m = min(k, 12)
        assert np.abs(al[:m] - r["alpha"][:m]).max() < 1e-12 * np.abs(r["alpha"][:m]).max()
        assert np.abs(de[:m - 1] - r["delta"][:m - 1]).max() < 1e-12 * np.abs(r["delta"][:m - 1]).max()
        sens = _sensitivity(lambda v: ot.tsl_sign_derivative(A, Ah, E, Eh, v, k)[:2], x[s].ravel())
        es, ed = relerr(ys[s], rs), relerr(yd[s], rd)
        print("derivative parity k=%d: sign %.3g deriv %.3g, oracle self-sensitivity %.3g" % (k, es, ed, sens))
        assert es < _parity_tol(sens)
        assert ed < _parity_tol(sens)


def test_mixed_converges_to_exact(lqlib):
    """Mixed path (FP32 stencil and vectors; FP64 dots, coefficients and Newton) against the
    exact dense sign and Frechet derivative of the oracle, at a depth where the FP64 method
    has converged below 1e-8 (sign) / 1e-6 (derivative).  FP32 vector storage delays the
    convergence; a CPU emulation of it (vectors rounded to complex64 each step) reaches
    3.3e-7 / 3.7e-6 on this case at k = 500, which bounds what the mixed path can reach."""
    from oracle import dirac as od
    from paper_1611_00195_gb300 import lq
    dims, k, mu = (4, 4, 2, 2), 500, 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5, nsrc=1)
    c = lq.Context(dims, mu=mu, precision=lq.LQ_MIXED)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, 1, True)
    ys, yd, rep = c.sign_derivative_apply(torch.from_numpy(x).cuda(), k)
    lat = od.Lattice(dims)
    H = od.dense_H(lat, U, mu)
    ex = osg.sign_schur(H) @ x[0].ravel()
    exd = osg.frechet_sylvester(H, od.dense_dH_dmu(lat, U, mu)) @ x[0].ravel()
    es, ed = relerr(ys[0].cpu().numpy(), ex), relerr(yd[0].cpu().numpy(), exd)
    print("mixed vs exact at k=%d: sign %.3g deriv %.3g" % (k, es, ed))
    assert rep[0]["status"] == 0
    assert es < 1e-6 and ed < 1e-5
