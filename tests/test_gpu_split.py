"""lq_opts.split: a derivative solve in FP32 with an even number of sources >= 8 runs the Krylov
loops of its two source halves as concurrent branches.  The halves are independent problems, so
the result is the unsplit one up to FP32 rounding (each half has its own reduction grids): both
are checked against the FP64 oracle at the same depth with the FP32-size bound of the schedule
tests, graph replay is bitwise equal to plain launches, and the split does not apply where it
must not (FP64, odd batches, kernel timing)."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import tsl as ot
from tests.helpers import FP32_SENS_FACTOR, oracle_ops, relerr

pytestmark = pytest.mark.gpu
DIMS, K, MU, NSRC = (4, 4, 2, 6), 40, 0.3, 8


def _ctx(lq, prec):
    c = lq.Context(DIMS, mu=MU, precision=prec)
    c.upload_gauge(torch.from_numpy(syn.gauge_field(DIMS, 0.4, 3)).cuda())
    c.reserve(K, NSRC, True)
    return c


def test_split_matches_oracle_and_unsplit(lqlib):
    from paper_1611_00195_gb300 import lq
    c = _ctx(lq, lq.LQ_MIXED)
    x = syn.gaussian_source(DIMS, 5, nsrc=NSRC)
    xt = torch.from_numpy(x).cuda()
    ys, yd, rep = c.sign_derivative_apply(xt, K)              # split (default)
    ys0, yd0, rep0 = c.sign_derivative_apply(xt, K, split=0)
    ys, yd, ys0, yd0 = (t.cpu().numpy() for t in (ys, yd, ys0, yd0))
    U = syn.gauge_field(DIMS, 0.4, 3)
    lat, A, Ah, E, Eh = oracle_ops(DIMS, U, MU)
    rng = np.random.default_rng(11)

    def pert(op):
        return lambda v: (lambda y: y * (1 + 6e-8 * (rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape))
                                         / np.sqrt(2)))(op(v))
    for s in range(NSRC):
        assert rep[s]["status"] == 0 and rep[s]["k_eff"] == K
        rd, rs, _ = ot.tsl_sign_derivative(A, Ah, E, Eh, x[s], K)
        rdp, rsp, _ = ot.tsl_sign_derivative(pert(A), pert(Ah), pert(E), pert(Eh), x[s], K)
        tol = max(1e-6, FP32_SENS_FACTOR * max(relerr(rdp, rd), relerr(rsp, rs)))
        errs = [relerr(ys[s], rs), relerr(yd[s], rd), relerr(ys0[s], rs), relerr(yd0[s], rd)]
        print("source %d: split sign %.3g deriv %.3g, unsplit sign %.3g deriv %.3g (bound %.3g)" % ((s,) + tuple(errs) + (tol,)))
        assert max(errs) < tol
        assert max(relerr(ys[s], ys0[s]), relerr(yd[s], yd0[s])) < tol


@pytest.mark.parametrize("prec", [0, 1])
def test_split_graph_is_bitwise_and_inert_where_it_does_not_apply(lqlib, prec):
    from paper_1611_00195_gb300 import lq
    c = _ctx(lq, prec)
    x = torch.from_numpy(syn.gaussian_source(DIMS, 5, nsrc=NSRC)).cuda()
    a = c.sign_derivative_apply(x, K, graph=-1)
    b = c.sign_derivative_apply(x, K, graph=-1)     # replay
    p = c.sign_derivative_apply(x, K, graph=0)
    for r in (b, p):
        assert torch.equal(a[0], r[0]) and torch.equal(a[1], r[1])
    if prec == lq.LQ_FP64:
        # FP64 never splits: split = 0 gives the same bits
        u = c.sign_derivative_apply(x, K, split=0)
        assert torch.equal(a[0], u[0]) and torch.equal(a[1], u[1])
    # an odd batch (7 sources) never splits either
    x7 = x[:7].contiguous()
    s7 = c.sign_derivative_apply(x7, K)
    u7 = c.sign_derivative_apply(x7, K, split=0)
    assert torch.equal(s7[0], u7[0]) and torch.equal(s7[1], u7[1])
    # kernel timing runs the unsplit loop
    u = c.sign_derivative_apply(x, K, split=0)
    c.profile_enable(True)
    t = c.sign_derivative_apply(x, K)
    c.profile_enable(False)
    assert torch.equal(t[0], u[0]) and torch.equal(t[1], u[1])
