"""Parity at the benchmark's full size (14x14^3, eps 0.4, gauge seed 2016, 16 Gaussian sources of
seed 1000, mu = 0.3, d/dmu), in the launch configuration bench.py times:
  * the operator H(mu) and its adjoint on all 16 sources in FP64, FP32 and float-float, two
    sampled sources against the oracle's stencil (an O(V) computation at any size);
  * the mixed block TSL with the bench's defaults (16 sources, the two halves as graph branches,
    the autotuned stencil schedule) at depth 24: sources 0 and 15 against the oracle's process at
    the same depth, within FP32_SENS_FACTOR of its response to FP32-size noise on every operator
    application (the oracle runs in a spawned process pool);
  * at a converged depth (k = 2400, float-float), the derivative of Eq. (2.6) against Richardson-
    extrapolated central differences of sgn(H(mu)) x in mu, a route that shares nothing with the
    block operator."""
import multiprocessing as mp

import numpy as np
import pytest
import torch

import synthetic as syn
from tests.helpers import FP32_SENS_FACTOR, relerr

pytestmark = pytest.mark.gpu
DIMS, EPS, GSEED, SSEED, MU, NSRC = (14, 14, 14, 14), 0.4, 2016, 1000, 0.3, 16


def _oracle_run(job):
    """Oracle block TSL (d/dmu) for source s of the benchmark batch at depth k; pert: None or
    (seed) for 6e-8 relative noise on every operator application.  Plain data in and out."""
    import numpy as np
    import synthetic as syn
    from oracle import tsl as ot
    from tests.helpers import oracle_ops
    s, k, pseed = job
    U = syn.gauge_field(DIMS, EPS, GSEED)
    x = syn.gaussian_source(DIMS, SSEED, nsrc=NSRC)[s].ravel()
    lat, A, Ah, E, Eh = oracle_ops(DIMS, U, MU)
    if pseed is not None:
        rng = np.random.default_rng(pseed)

        def wrap(op):
            def f(v):
                y = op(v)
                return y * (1 + 6e-8 * (rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape)) / np.sqrt(2))
            return f
        A, Ah, E, Eh = wrap(A), wrap(Ah), wrap(E), wrap(Eh)
    rd, rs, _ = ot.tsl_sign_derivative(A, Ah, E, Eh, x, k)
    return rd, rs


@pytest.fixture(scope="module")
def bench_inputs():
    U = syn.gauge_field(DIMS, EPS, GSEED)
    x = syn.gaussian_source(DIMS, SSEED, nsrc=NSRC)
    return U, x


def test_full_size_operator(lqlib, bench_inputs):
    from oracle import dirac as od
    from paper_1611_00195_gb300 import lq
    U, x = bench_inputs
    lat = od.Lattice(DIMS, m_w=-2.0)
    xt = torch.from_numpy(x).cuda()
    for prec, bound in ((lq.LQ_FP64, 1e-14), (lq.LQ_MIXED, 2e-6), (lq.LQ_FLOAT_FLOAT, 1e-12)):
        c = lq.Context(DIMS, m_w=-2.0, mu=MU, precision=prec)
        c.upload_gauge(torch.from_numpy(U).cuda())
        c.reserve(2, NSRC, True)
        for dag in (False, True):
            y = c.apply_H(xt, dagger=dag).cpu().numpy()
            for s in (0, NSRC - 1):
                ref = (od.apply_Hdag if dag else od.apply_H)(lat, U, x[s], MU)
                e = relerr(y[s], ref)
                print("14^4 precision %d H%s source %d: %.3g" % (prec, "^dag" if dag else "", s, e))
                assert e < bound
        del c


def test_full_size_block_tsl_in_the_bench_configuration(lqlib, bench_inputs):
    from paper_1611_00195_gb300 import lq
    U, x = bench_inputs
    k = 24
    jobs = [(s, k, p) for s in (0, NSRC - 1) for p in (None, 17)]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = dict(zip(jobs, pool.map(_oracle_run, jobs)))
    c = lq.Context(DIMS, m_w=-2.0, mu=MU, precision=lq.LQ_MIXED)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, NSRC, True)
    ys, yd, rep = c.sign_derivative_apply(torch.from_numpy(x).cuda(), k)   # the bench's defaults
    ys, yd = ys.cpu().numpy(), yd.cpu().numpy()
    for s in (0, NSRC - 1):
        assert rep[s]["status"] == 0 and rep[s]["k_eff"] == k
        rd, rs = res[(s, k, None)]
        pd, ps = res[(s, k, 17)]
        sens = max(relerr(pd, rd), relerr(ps, rs))
        errs = [relerr(ys[s], rs), relerr(yd[s], rd)]
        print("14^4 bench configuration k=%d source %d (schedule %d): sign %.3g deriv %.3g (FP32-size sensitivity %.3g, "
              "ratio %.2f)" % (k, s, rep[s]["hop_variant"], errs[0], errs[1], sens, max(errs) / sens))
        assert max(errs) < max(1e-6, FP32_SENS_FACTOR * sens)


def test_full_size_derivative_against_finite_differences(lqlib, bench_inputs):
    from paper_1611_00195_gb300 import lq
    U, x = bench_inputs
    k, s = 2400, 0
    x1 = torch.from_numpy(np.ascontiguousarray(x[s:s + 1])).cuda()
    Ut = torch.from_numpy(U).cuda()
    c = lq.Context(DIMS, m_w=-2.0, mu=MU, precision=lq.LQ_FLOAT_FLOAT)
    c.upload_gauge(Ut)
    c.reserve(k, 1, True)
    _, yd, rep = c.sign_derivative_apply(x1, k)
    yd = yd[0].cpu().numpy()
    eps = float(c.error_estimate(x1, k, kind=lq.LQ_DIR_MU)[0])
    del c

    def sign_at(mu):
        cm = lq.Context(DIMS, m_w=-2.0, mu=mu, precision=lq.LQ_FLOAT_FLOAT)
        cm.upload_gauge(Ut)
        cm.reserve(k, 1, False)
        y, r = cm.sign_apply(x1, k)
        assert r[0]["status"] == 0
        out = y[0].cpu().numpy()
        del cm
        return out

    h = 2e-3
    d = {hh: (sign_at(MU + hh) - sign_at(MU - hh)) / (2 * hh) for hh in (h, h / 2)}
    rich = (4 * d[h / 2] - d[h]) / 3                      # O(h^4)
    e_h, e_h2, e_r = relerr(d[h], yd), relerr(d[h / 2], yd), relerr(rich, yd)
    print("14^4 k=%d float-float derivative vs central differences: h %.3g, h/2 %.3g (ratio %.2f, O(h^2) gives 4), "
          "Richardson %.3g; eps_A of the derivative %.3g" % (k, e_h, e_h2, e_h / e_h2, e_r, eps))
    assert rep[0]["status"] == 0 and eps < 1e-8
    assert e_r < 1e-6
