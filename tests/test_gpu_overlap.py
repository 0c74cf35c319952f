"""The overlap operator of Eq. (1.1), D_ov = 1 + gamma5 sgn(H(mu)), and its derivative through
lq_overlap_apply: same-depth parity with the oracle's two-sided Lanczos, convergence to the
oracle's dense D_ov, and the Ginsparg-Wilson relation on the GPU's own results."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import dirac as od
from oracle import overlap as oo
from oracle import tsl as ot
from tests.helpers import FP64_SENS_FACTOR, oracle_ops, relerr

pytestmark = pytest.mark.gpu
MU = 0.3


def _ctx(lq, dims, k, nsrc, prec=0):
    c = lq.Context(dims, mu=MU, precision=prec)
    c.upload_gauge(torch.from_numpy(syn.gauge_field(dims, 0.4, 3)).cuda())
    c.reserve(k, nsrc, True)
    return c


@pytest.mark.parametrize("kind", [0, 1])
def test_overlap_same_depth_parity(lqlib, kind):
    from paper_1611_00195_gb300 import lq
    dims, k, nsrc = (4, 4, 2, 6), 40, 2
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5, nsrc=nsrc)
    field = syn.su3_direction(dims, 77) if kind == 1 else None
    c = _ctx(lq, dims, k, nsrc)
    y, dy, rep = c.overlap_apply(torch.from_numpy(x).cuda(), k, kind=kind,
                                 field=None if field is None else torch.from_numpy(field).cuda())
    y0, _, _ = c.overlap_apply(torch.from_numpy(x).cuda(), k, derivative=False)
    y, dy, y0 = y.cpu().numpy(), dy.cpu().numpy(), y0.cpu().numpy()
    lat, A, Ah, E, Eh = oracle_ops(dims, U, MU, kind, field)
    g5 = oo.gamma5_full(lat)
    rng = np.random.default_rng(3)
    for s in range(nsrc):
        assert rep[s]["status"] == 0
        xv = x[s].ravel()

        def run(v):
            rd, rs, _ = ot.tsl_sign_derivative(A, Ah, E, Eh, v, k)
            return v + g5 @ rs, g5 @ rd
        ry, rdy = run(xv)
        sens = 0.0
        for _ in range(3):
            py, pdy = run(xv * (1 + 1e-16 * rng.standard_normal(xv.shape)))
            sens = max(sens, relerr(py, ry), relerr(pdy, rdy))
        tol = max(1e-11, FP64_SENS_FACTOR * sens)
        ey, edy = relerr(y[s], ry), relerr(dy[s], rdy)
        # the sign-only call runs the plain process (A, not B): against the oracle's plain TSL
        r0 = xv + g5 @ ot.tsl_sign(A, Ah, xv, k)[0]
        sens0 = 0.0
        for _ in range(3):
            xp = xv * (1 + 1e-16 * rng.standard_normal(xv.shape))
            sens0 = max(sens0, relerr(xp + g5 @ ot.tsl_sign(A, Ah, xp, k)[0], r0))
        e0 = relerr(y0[s], r0)
        print("overlap k=%d dir %d: D x %.3g, dD x %.3g (sensitivity %.3g); sign-only D x %.3g (sensitivity %.3g)"
              % (k, kind, ey, edy, sens, e0, sens0))
        assert ey < tol and edy < tol
        assert e0 < max(1e-11, FP64_SENS_FACTOR * sens0)


@pytest.mark.parametrize("prec,tol", [(0, 1e-6), (1, 1e-5)])
def test_overlap_converges_and_ginsparg_wilson(lqlib, prec, tol):
    """At k = 190 on 2^4 (n = 192) the GPU D_ov x and d D_ov x agree with the dense oracle, and
    the results satisfy gamma5 D x + D gamma5 x = D gamma5 D x (every D applied on the GPU)."""
    from paper_1611_00195_gb300 import lq
    dims, k = (2, 2, 2, 2), 190
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5, nsrc=1)
    c = _ctx(lq, dims, k, 1, prec)
    lat = od.Lattice(dims)
    Ed = od.dense_dH_dmu(lat, U, MU)
    yex, dyex = oo.overlap_apply(lat, U, MU, x[0], Ed)
    y, dy, rep = c.overlap_apply(torch.from_numpy(x).cuda(), k)
    ey, edy = relerr(y[0].cpu().numpy(), yex), relerr(dy[0].cpu().numpy(), dyex)
    g5 = np.diag(np.tile([1, 1, 1, 1, 1, 1, -1, -1, -1, -1, -1, -1], lat.V)).astype(complex)

    def D(v):
        out, _, _ = c.overlap_apply(torch.from_numpy(v.reshape(1, lat.V, 4, 3)).cuda(), k, derivative=False)
        return out[0].cpu().numpy().ravel()
    xv = x[0].ravel()
    Dx = D(xv)
    gw = relerr(g5 @ Dx + D(g5 @ xv), D(g5 @ Dx))
    print("overlap prec %d k=%d vs dense: D x %.3g, dD x %.3g; Ginsparg-Wilson residual %.3g" % (prec, k, ey, edy, gw))
    assert rep[0]["status"] == 0
    assert ey < tol and edy < 100 * tol and gw < 10 * tol
