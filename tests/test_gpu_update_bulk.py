"""The FP32 Lanczos update with its inputs staged by bulk asynchronous copies (lq_opts.
update_variant -1 / 1, the default) against the register-streaming kernel (0) and the FP64 oracle:
both variants within the FP32-size bound of the oracle at the same depth, on a lattice whose
vector length leaves a ragged last tile of 256 chunks and on one where every block of the grid
refills its four stages several times (16 sources at 8^4)."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import tsl as ot
from tests.helpers import FP32_SENS_FACTOR, oracle_ops, relerr

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,nsrc,k,check", [((5, 3, 3, 4), 3, 40, 3), ((8, 8, 8, 8), 16, 24, 2)])
def test_bulk_update_matches_oracle_and_register_kernel(lqlib, dims, nsrc, k, check):
    from paper_1611_00195_gb300 import lq
    mu = 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5, nsrc=nsrc)
    c = lq.Context(dims, mu=mu, precision=lq.LQ_MIXED)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, nsrc, True)
    xt = torch.from_numpy(x).cuda()
    out = {}
    for uv in (-1, 0):
        ys, yd, rep = c.sign_derivative_apply(xt, k, update_variant=uv, split=0)
        assert all(r["status"] == 0 and r["k_eff"] == k for r in rep)
        out[uv] = (ys.cpu().numpy(), yd.cpu().numpy(), [c.tsl_coefficients(s, k) for s in range(nsrc)])
    lat, A, Ah, E, Eh = oracle_ops(dims, U, mu)
    rng = np.random.default_rng(11)

    def pert(op):
        return lambda v: (lambda y: y * (1 + 6e-8 * (rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape))
                                         / np.sqrt(2)))(op(v))
    for s in range(check):
        rd, rs, _ = ot.tsl_sign_derivative(A, Ah, E, Eh, x[s], k)
        rdp, rsp, _ = ot.tsl_sign_derivative(pert(A), pert(Ah), pert(E), pert(Eh), x[s], k)
        tol = max(1e-6, FP32_SENS_FACTOR * max(relerr(rdp, rd), relerr(rsp, rs)))
        errs = [relerr(out[uv][i][s], ref) for uv in (-1, 0) for i, ref in ((0, rs), (1, rd))]
        print("%s source %d: bulk sign %.3g deriv %.3g, register sign %.3g deriv %.3g (bound %.3g)"
              % ((dims, s) + tuple(errs) + (tol,)))
        assert max(errs) < tol
    for s in range(nsrc):
        # the first step's alpha comes from the same stencil; the vectors of the two updates are
        # bitwise the same and their scalars differ by the summation order of the dots only
        a1, a0 = out[-1][2][s][0], out[0][2][s][0]
        assert a1[0] == a0[0]
        d1, d0 = out[-1][2][s][2], out[0][2][s][2]
        assert abs(d1[0] - d0[0]) <= 1e-12 * abs(d0[0])
        assert max(relerr(out[-1][0][s], out[0][0][s]), relerr(out[-1][1][s], out[0][1][s])) < 1e-4


def test_bulk_update_in_the_adjoint_and_split_runs(lqlib):
    """The left basis copy of the adjoint (w_store) and the split run (the bulk kernel asked for
    explicitly) give the register kernel's results up to the order of the dot sums."""
    from paper_1611_00195_gb300 import lq
    dims, nsrc, k, mu = (4, 4, 2, 6), 8, 40, 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    x = torch.from_numpy(syn.gaussian_source(dims, 5, nsrc=nsrc)).cuda()
    c = lq.Context(dims, mu=mu, precision=lq.LQ_MIXED)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, nsrc, True)
    a = c.sign_derivative_apply(x, k, update_variant=1)     # split, bulk update
    b = c.sign_derivative_apply(x, k)                       # split, register update (the default)
    for p, q in zip(a[:2], b[:2]):
        assert relerr(p.cpu().numpy(), q.cpu().numpy()) < 1e-4
    ca = lq.Context(dims, mu=mu, precision=lq.LQ_MIXED)
    ca.upload_gauge(torch.from_numpy(U).cuda())
    ca.reserve(k, 2, block=False, adjoint=True)
    xs = torch.from_numpy(syn.gaussian_source(dims, 5, nsrc=1)[0]).cuda()
    ys = torch.from_numpy(syn.gaussian_source(dims, 9, nsrc=1)[0]).cuda()
    S1, F1, m1 = ca.bilinear_grad(xs, ys, k)
    S0, F0, m0 = ca.bilinear_grad(xs, ys, k, update_variant=0)
    print("adjoint: S %.12g / %.12g, dS/dmu %.12g / %.12g, force %.3g" % (S1, S0, m1, m0, relerr(F1.cpu().numpy(), F0.cpu().numpy())))
    assert abs(S1 - S0) <= 1e-5 * abs(S0) and abs(m1 - m0) <= 1e-4 * abs(m0)
    assert relerr(F1.cpu().numpy(), F0.cpu().numpy()) < 1e-4
