"""Two-pass TSL (lq_opts.two_pass): the first pass keeps a ring of 32 basis vectors and yields
T_k, the second reruns the same process and recombines windows of 16 vectors.  The process is
deterministic, so T_k must be bitwise the one of a one-pass run and the result must agree to
the rounding of the recombination order."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import tsl as ot
from tests.helpers import FP64_SENS_FACTOR, oracle_ops, relerr

pytestmark = pytest.mark.gpu

DIMS, MU = (4, 4, 2, 6), 0.3


def _ctx(lq, prec, k, nsrc, two_pass):
    c = lq.Context(DIMS, mu=MU, precision=prec)
    c.upload_gauge(torch.from_numpy(syn.gauge_field(DIMS, 0.4, 3)).cuda())
    c.reserve(k, nsrc, True, two_pass=two_pass)
    return c


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 1e-7)])
@pytest.mark.parametrize("deriv", [False, True])
def test_two_pass_matches_one_pass(lqlib, prec, tol, deriv):
    from paper_1611_00195_gb300 import lq
    k, nsrc = 100, 3          # the ring wraps three times; the last window holds 4 vectors
    x = torch.from_numpy(syn.gaussian_source(DIMS, 5, nsrc=nsrc)).cuda()
    c1 = _ctx(lq, prec, k, nsrc, False)
    c2 = _ctx(lq, prec, k, nsrc, True)
    if deriv:
        a1 = c1.sign_derivative_apply(x, k, hop_variant=0)
        a2 = c2.sign_derivative_apply(x, k, hop_variant=0, two_pass=1)
        outs = [(a1[0], a2[0]), (a1[1], a2[1])]
        rep2 = a2[2]
    else:
        y1, _ = c1.sign_apply(x, k)
        y2, rep2 = c2.sign_apply(x, k, two_pass=1)
        outs = [(y1, y2)]
    for s in range(nsrc):
        assert rep2[s]["status"] == 0 and rep2[s]["k_eff"] == k
        t1, t2 = c1.tsl_coefficients(s, k), c2.tsl_coefficients(s, k)
        for p, q in zip(t1, t2):
            assert np.array_equal(p, q)            # the same process, bit for bit
        for p, q in outs:
            e = relerr(q[s].cpu().numpy(), p[s].cpu().numpy())
            print("two-pass vs one-pass (prec %d, deriv %d) source %d: %.3g" % (prec, deriv, s, e))
            assert e < tol


def test_two_pass_on_full_basis_and_short_runs(lqlib):
    """two_pass = 1 on a full-basis workspace gives the same result; a ring workspace runs
    depths within the ring in one pass and refuses deeper one-pass runs."""
    from paper_1611_00195_gb300 import lq
    x = torch.from_numpy(syn.gaussian_source(DIMS, 5, nsrc=2)).cuda()
    c1 = _ctx(lq, 0, 60, 2, False)
    y1, _ = c1.sign_apply(x, 60)
    y2, _ = c1.sign_apply(x, 60, two_pass=1)
    assert relerr(y2.cpu().numpy(), y1.cpu().numpy()) < 1e-13
    c2 = _ctx(lq, 0, 60, 2, True)
    y3, _ = c2.sign_apply(x, 20)                   # within the ring: one pass
    y4, _ = c1.sign_apply(x, 20)
    assert relerr(y3.cpu().numpy(), y4.cpu().numpy()) < 1e-14
    with pytest.raises(lq.LQError):
        c2.sign_apply(x, 60)                       # deeper than the ring without two_pass
    lq.Context(DIMS, mu=MU).reserve(60, 2, False, adjoint=True, two_pass=True)   # the two-pass adjoint workspace


@pytest.mark.parametrize("deriv", [False, True])
def test_two_pass_fp64_matches_the_oracle(lqlib, deriv):
    """The two-pass run (FP64, k = 100: the ring of 32 wraps three times) against the oracle's
    one-pass process at the same depth, within FP64_SENS_FACTOR of the oracle's own rounding
    sensitivity, like the one-pass parity tests."""
    from paper_1611_00195_gb300 import lq
    k, nsrc = 100, 2
    U = syn.gauge_field(DIMS, 0.4, 3)
    x = syn.gaussian_source(DIMS, 5, nsrc=nsrc)
    c = _ctx(lq, 0, k, nsrc, True)
    if deriv:
        ys, yd, rep = c.sign_derivative_apply(torch.from_numpy(x).cuda(), k, two_pass=1)
        got = [yd.cpu().numpy(), ys.cpu().numpy()]
    else:
        ys, rep = c.sign_apply(torch.from_numpy(x).cuda(), k, two_pass=1)
        got = [ys.cpu().numpy()]
    lat, A, Ah, E, Eh = oracle_ops(DIMS, U, MU)
    rng = np.random.default_rng(99)

    def run(v):
        if deriv:
            return list(ot.tsl_sign_derivative(A, Ah, E, Eh, v, k)[:2])
        return [ot.tsl_sign(A, Ah, v, k)[0]]
    for s in range(nsrc):
        assert rep[s]["status"] == 0 and rep[s]["k_eff"] == k
        ref = run(x[s].ravel())
        xp = x[s].ravel() * (1 + 1e-16 * rng.standard_normal(x[s].size))
        sens = max(relerr(p, q) for p, q in zip(run(xp), ref))
        errs = [relerr(g[s], r) for g, r in zip(got, ref)]
        print("two-pass FP64 vs oracle k=%d deriv %d source %d: %s (sensitivity %.3g, ratio %.2f)"
              % (k, deriv, s, ["%.3g" % e for e in errs], sens, max(errs) / sens))
        assert max(errs) < max(1e-11, FP64_SENS_FACTOR * sens)
