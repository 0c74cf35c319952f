"""The precision workload: 8^4 lattice (n = 49152), eps = 0.4, m_w = -2, one Gaussian source,
k = 200, mu in {0.0, 0.1, 0.2}.  The plain FP64 GPU path and the mixed path (FP32 stencil and
vectors; FP64 coefficients, compensated dots, projected sign) against the FP64 oracle at the same
depth (Sec. 2, Eq. (2.6), d/dmu), with the relative error per mu printed, and the mixed path
against the FP64 GPU path next to the 1e-6 target, which this undeflated workload does not meet
for mu > 0 at k = 200: there the process is not converged and amplifies FP32 rounding like any
other perturbation.  The bounds are the same-depth parity bounds: FP64 within FP64_SENS_FACTOR
of the oracle's response to 1e-16 input noise, mixed within FP32_DEEP_SENS_FACTOR of its response to
6e-8 noise on every operator application (the largest over three noise samples).  The oracle
runs in a spawned process pool (fifteen runs of about half a minute each)."""
import multiprocessing as mp
import os

import numpy as np
import pytest
import torch

import synthetic as syn
from tests.helpers import FP32_DEEP_SENS_FACTOR, FP64_SENS_FACTOR, oracle_block_tsl_run, relerr

pytestmark = pytest.mark.gpu
DIMS, EPS, K, GSEED, SSEED = (8, 8, 8, 8), 0.4, 200, 3, 5
MUS = (0.0, 0.1, 0.2)


@pytest.fixture(scope="module")
def oracle_results():
    jobs = [(DIMS, EPS, GSEED, SSEED, mu, K, p, ps) for mu in MUS
            for p, ps in ((None, 17), ("input", 17), ("step", 17), ("step", 18), ("step", 19))]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        res = pool.map(oracle_block_tsl_run, jobs)
    return {(mu, p, ps): r for (_, _, _, _, mu, _, p, ps), r in zip(jobs, res)}


@pytest.mark.parametrize("mu", MUS)
def test_precision_workload(lqlib, oracle_results, mu):
    from paper_1611_00195_gb300 import lq
    U = torch.from_numpy(syn.gauge_field(DIMS, EPS, GSEED)).cuda()
    x = torch.from_numpy(syn.gaussian_source(DIMS, SSEED, nsrc=1)).cuda()
    rd, rs = oracle_results[(mu, None, 17)]
    pd, ps = oracle_results[(mu, "input", 17)]
    sens64 = max(relerr(pd, rd), relerr(ps, rs))
    sens32 = max(max(relerr(qd, rd), relerr(qs, rs))
                 for qd, qs in (oracle_results[(mu, "step", q)] for q in (17, 18, 19)))
    out = {}
    for prec in (lq.LQ_FP64, lq.LQ_MIXED):
        c = lq.Context(DIMS, mu=mu, precision=prec)
        c.upload_gauge(U)
        c.reserve(K, 1, True)
        ys, yd, rep = c.sign_derivative_apply(x, K)
        assert rep[0]["status"] == 0 and rep[0]["k_eff"] == K
        out[prec] = (relerr(ys[0].cpu().numpy(), rs), relerr(yd[0].cpu().numpy(), rd),
                     ys[0].cpu().numpy(), yd[0].cpu().numpy())
    (e64s, e64d, y64s, y64d), (e32s, e32d, y32s, y32d) = out[lq.LQ_FP64], out[lq.LQ_MIXED]
    ms, md = relerr(y32s, y64s), relerr(y32d, y64d)
    print("8^4 k=%d mu=%.1f vs oracle: FP64 sign %.3g deriv %.3g (sensitivity %.3g, ratio %.2f); mixed sign %.3g "
          "deriv %.3g (FP32-size sensitivity %.3g, ratio %.2f); mixed vs FP64 GPU: sign %.3g deriv %.3g "
          "(target 1e-6: %s)" % (K, mu, e64s, e64d, sens64, max(e64s, e64d) / sens64, e32s, e32d, sens32,
                                 max(e32s, e32d) / sens32, ms, md, "met" if max(ms, md) <= 1e-6 else "not met"))
    assert max(e64s, e64d) < max(1e-11, FP64_SENS_FACTOR * sens64)
    assert max(e32s, e32d) < max(1e-6, FP32_DEEP_SENS_FACTOR * sens32)
