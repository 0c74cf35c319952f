"""BF16 link storage (LQ_MIXED_BF16): FP32 vectors and arithmetic with the links stored in BF16.
The context works with the rounded gauge field (FP64 -> FP32 -> BF16, nearest even), so its
reference is the oracle on the same rounded links (tests.helpers.round_bf16, an input
transformation): the stencil to FP32 rounding and the derivative solve within the FP32 parity
bound at the same depth.  The difference to the unrounded field -- a different operator,
changed by the BF16 rounding of the links (relative 2^-9) -- is printed."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import dirac as od
from oracle import tsl as ot
from tests.helpers import FP32_SENS_FACTOR, oracle_ops, relerr, round_bf16

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dagger", [False, True])
def test_bf16_stencil(lqlib, dagger):
    from paper_1611_00195_gb300 import lq
    dims, mu = (4, 4, 2, 6), 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    Ur = round_bf16(U)
    x = syn.gaussian_source(dims, 5, nsrc=2)
    c = lq.Context(dims, mu=mu, precision=lq.LQ_MIXED_BF16)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(4, 2, True)
    y = c.apply_H(torch.from_numpy(x).cuda(), dagger=dagger).cpu().numpy()
    lat = od.Lattice(dims)
    op = od.apply_Hdag if dagger else od.apply_H
    for s in range(2):
        ref = op(lat, Ur, x[s], mu).ravel()
        e = relerr(y[s].ravel(), ref)
        e0 = relerr(y[s].ravel(), op(lat, U, x[s], mu).ravel())
        print("bf16 stencil (dagger %d) source %d: vs rounded links %.3g, vs unrounded %.3g" % (dagger, s, e, e0))
        assert e < 2e-6
        assert 1e-5 < e0 < 1e-2       # the BF16 rounding of the links is visible


@pytest.mark.parametrize("kind", [0, 1])
def test_bf16_derivative_solve(lqlib, kind):
    from paper_1611_00195_gb300 import lq
    dims, k, mu = (4, 4, 2, 6), 40, 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    Ur = round_bf16(U)
    x = syn.gaussian_source(dims, 5, nsrc=2)
    field = syn.su3_direction(dims, 77) if kind == 1 else None
    c = lq.Context(dims, mu=mu, precision=lq.LQ_MIXED_BF16)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, 2, True)
    fd = None if field is None else torch.from_numpy(field).cuda()
    ys, yd, rep = c.sign_derivative_apply(torch.from_numpy(x).cuda(), k, kind=kind, field=fd)
    ys, yd = ys.cpu().numpy(), yd.cpu().numpy()
    lat, A, Ah, E, Eh = oracle_ops(dims, Ur, mu, kind, field)
    _, A0, Ah0, E0, Eh0 = oracle_ops(dims, U, mu, kind, field)
    rng = np.random.default_rng(11)

    def pert(op):
        return lambda v: (lambda y: y * (1 + 6e-8 * (rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape))
                                         / np.sqrt(2)))(op(v))
    for s in range(2):
        assert rep[s]["status"] == 0 and rep[s]["hop_variant"] not in (6, 7, 8)
        rd, rs, _ = ot.tsl_sign_derivative(A, Ah, E, Eh, x[s], k)
        sens = 0.0
        for _ in range(2):
            rdp, rsp, _ = ot.tsl_sign_derivative(pert(A), pert(Ah), pert(E), pert(Eh), x[s], k)
            sens = max(sens, relerr(rdp, rd), relerr(rsp, rs))
        es, ed = relerr(ys[s], rs), relerr(yd[s], rd)
        d0, s0, _ = ot.tsl_sign_derivative(A0, Ah0, E0, Eh0, x[s], k)
        print("bf16 derivative solve kind %d source %d: vs rounded-link oracle sign %.3g deriv %.3g (FP32-size "
              "sensitivity %.3g, ratio %.2f); vs unrounded links sign %.3g deriv %.3g"
              % (kind, s, es, ed, sens, max(es, ed) / sens, relerr(ys[s], s0), relerr(yd[s], d0)))
        assert max(es, ed) < max(1e-6, FP32_SENS_FACTOR * sens)
