"""GPU parity of the deflation of Sec. 3 against the CPU oracle: the standard deflation of
Eq. (3.1) for the sign, the eigenvector derivatives (end of Sec. 3) with the shifted solves done
by two-sided Lanczos approximations of the resolvent, and the generalised deflation of
Eqs. (3.2)-(3.4) for the derivative.  The eigenpairs come from the oracle's dense eig."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import deflation as odf
from oracle import dirac as od
from oracle import sign as osg
from oracle import tsl as ot
from tests.helpers import oracle_ops, relerr

pytestmark = pytest.mark.gpu

MU = 0.3


def _setup(lq, dims, l, k, nsrc=2, prec=0, seed=3):
    U = syn.gauge_field(dims, 0.4, seed)
    lat = od.Lattice(dims)
    A = od.dense_H(lat, U, MU)
    lam, R, L, full = odf.eigenpairs(A, l)
    x = syn.gaussian_source(dims, 5, nsrc=nsrc)
    c = lq.Context(dims, mu=MU, precision=prec)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, nsrc, True)
    Rk = np.ascontiguousarray(R.T.reshape(l, lat.V, 4, 3))
    Lk = np.ascontiguousarray(L.conj().reshape(l, lat.V, 4, 3))
    c.upload_deflation(lam, torch.from_numpy(Rk).cuda(), torch.from_numpy(Lk).cuda())
    return c, U, lat, A, lam, R, L, x


@pytest.mark.parametrize("dims,l,k", [((4, 4, 2, 2), 8, 120), ((4, 2, 2, 2), 6, 60)])
def test_sign_deflated_parity(lqlib, dims, l, k):
    from paper_1611_00195_gb300 import lq
    c, U, lat, A, lam, R, L, x = _setup(lq, dims, l, k)
    y, rep = c.sign_apply(torch.from_numpy(x).cuda(), k, deflate=1)
    y0, _ = c.sign_apply(torch.from_numpy(x).cuda(), k, deflate=0)
    y, y0 = y.cpu().numpy(), y0.cpu().numpy()
    _, Ao, Aho, _, _ = oracle_ops(dims, U, MU)
    S = osg.sign_schur(A)
    for s in range(x.shape[0]):
        xs = x[s].ravel()
        ref = odf.sign_deflated(lambda v: ot.tsl_sign(Ao, Aho, v, k)[0], lam, R, L, xs)
        err = relerr(y[s], ref)
        ex, ex0 = relerr(y[s], S @ xs), relerr(y0[s], S @ xs)
        print("deflated sign k=%d l=%d: parity %.3g; error vs exact %.3g (undeflated %.3g)" % (k, l, err, ex, ex0))
        assert err < 1e-9
        assert ex < 0.5 * ex0


def test_eigen_derivatives_parity(lqlib):
    from paper_1611_00195_gb300 import lq
    dims, l, k = (4, 2, 2, 2), 6, 300
    c, U, lat, A, lam, R, L, x = _setup(lq, dims, l, k)
    dlam, dR, dLk = c.deflation_derivatives(k, kind=lq.LQ_DIR_MU)
    lat_, Ao, Aho, Eo, Eho = oracle_ops(dims, U, MU)
    rl, rR, rL = odf.eigen_derivatives_tsl(Ao, Aho, Eo, Eho, lam, R, L, k)
    E = od.dense_dH_dmu(lat, U, MU)
    ex = odf.eigen_derivatives_projected(A, E, lam, R, L)
    gR = dR.reshape(l, -1).T
    gL = dLk.reshape(l, -1).conj()
    print("eigen-derivatives k=%d: dR parity %.3g, dL parity %.3g; vs exact %.3g / %.3g"
          % (k, relerr(gR, rR), relerr(gL, rL), relerr(gR, ex[1]), relerr(gL, ex[2])))
    assert np.abs(dlam - rl).max() < 1e-12 * np.abs(rl).max()
    assert relerr(gR, rR) < 1e-6 and relerr(gL, rL) < 1e-6


def test_derivative_generalised_deflation(lqlib):
    from paper_1611_00195_gb300 import lq
    dims, l, k = (4, 2, 2, 2), 6, 300
    c, U, lat, A, lam, R, L, x = _setup(lq, dims, l, k)
    xs_d = torch.from_numpy(x).cuda()
    ys, yd, rep = c.sign_derivative_apply(xs_d, k, deflate=1)
    ys0, yd0, _ = c.sign_derivative_apply(xs_d, k, deflate=0)
    ys, yd, ys0, yd0 = (t.cpu().numpy() for t in (ys, yd, ys0, yd0))
    lat_, Ao, Aho, Eo, Eho = oracle_ops(dims, U, MU)
    rl, rR, rL = odf.eigen_derivatives_tsl(Ao, Aho, Eo, Eho, lam, R, L, k)
    E = od.dense_dH_dmu(lat, U, MU)
    SB = odf.sign_block_exact(A, E)
    n = lat.n
    for s in range(x.shape[0]):
        psi = np.concatenate([np.zeros(n), x[s].ravel()])

        def blk(v):
            t, b, _ = ot.tsl_sign_block(Ao, Aho, Eo, Eho, v[:n], v[n:], k)
            return np.concatenate([t, b])
        ref = odf.sign_block_deflated(blk, lam, R, L, rR, rL, psi)
        ex = SB @ psi
        pd, ps = relerr(yd[s], ref[:n]), relerr(ys[s], ref[n:])
        ed, ed0 = relerr(yd[s], ex[:n]), relerr(yd0[s], ex[:n])
        print("deflated derivative k=%d l=%d: parity deriv %.3g sign %.3g; deriv error vs exact %.3g (undeflated %.3g)"
              % (k, l, pd, ps, ed, ed0))
        assert pd < 1e-6 and ps < 1e-6
        assert ed < ed0
