"""Per-source failure statuses of the CUDA path, each caused from the host side by a
crafted input (nothing here faults, traps or hangs the device):

* an invariant Krylov subspace (free-field plane wave): the process stops with k_eff < k and
  LQ_ERR_BREAKDOWN, and the result from T_{k_eff} equals the free-field closed form;
* a NaN in the host input: LQ_ERR_NONFINITE for that source only;
* a projected matrix with eigenvalues on the imaginary axis, where sgn is undefined (the branch
  cut of Sec. 3): the Newton iteration cannot converge and reports LQ_ERR_NEWTON.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import dirac as od
from oracle import free_field as ff
from oracle import sign as osg
from tests.helpers import relerr
from tests.test_oracle_tsl import _plane_wave

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 2, 2)


def _free_ctx(lq, prec, mu, k, nsrc, block):
    lat = od.Lattice(DIMS)
    U = np.tile(np.eye(3, dtype=complex), (4, lat.V, 1, 1))
    c = lq.Context(DIMS, mu=mu, precision=prec)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, nsrc, block)
    return lat, c


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_plane_wave_stops_with_breakdown(lqlib, prec):
    from paper_1611_00195_gb300 import lq
    p = lq.LQ_FP64 if prec == "fp64" else lq.LQ_MIXED
    tol_s, tol_d = (1e-12, 1e-11) if prec == "fp64" else (2e-6, 2e-5)
    mu, k = 0.3, 8
    lat, c = _free_ctx(lq, p, mu, k, 2, True)
    x = _plane_wave(lat, 4).reshape(lat.V, 4, 3)
    g = np.random.default_rng(9).standard_normal((lat.V, 4, 3)) * (1 + 0j)
    X = torch.from_numpy(np.stack([x, g])).cuda()
    # sign: the plane wave stops at k_eff = 2 (H(p)^2 is a scalar), the Gaussian source runs on
    y, rep = c.sign_apply(X, k)
    torch.cuda.synchronize()
    assert rep[0]["status"] == lq.LQ_ERR_BREAKDOWN and rep[0]["k_eff"] == 2, rep[0]
    assert rep[1]["status"] == lq.LQ_OK and rep[1]["k_eff"] == k, rep[1]
    assert relerr(y[0].cpu().numpy().ravel(), ff.free_sign(lat, x.ravel(), mu).ravel()) < tol_s
    # derivative along mu: two 2x2 Jordan blocks, k_eff = 4 (Eq. (3.2))
    ys, yd, rep = c.sign_derivative_apply(X, k)
    torch.cuda.synchronize()
    assert rep[0]["status"] == lq.LQ_ERR_BREAKDOWN and rep[0]["k_eff"] == 4, rep[0]
    assert rep[1]["status"] == lq.LQ_OK and rep[1]["k_eff"] == k, rep[1]
    assert relerr(ys[0].cpu().numpy().ravel(), ff.free_sign(lat, x.ravel(), mu).ravel()) < tol_s
    assert relerr(yd[0].cpu().numpy().ravel(), ff.free_sign_dmu(lat, x.ravel(), mu).ravel()) < tol_d


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nonfinite_source_is_reported_alone(lqlib, prec):
    import synthetic as syn
    from paper_1611_00195_gb300 import lq
    p = lq.LQ_FP64 if prec == "fp64" else lq.LQ_MIXED
    mu, k = 0.3, 16
    U = syn.gauge_field(DIMS, 0.4, 3)
    c = lq.Context(DIMS, mu=mu, precision=p)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, 2, True)
    x = syn.gaussian_source(DIMS, 5, nsrc=2)
    xb = x.copy()
    xb[0, 7, 2, 1] = np.nan                   # one NaN in the first source, host side
    ys_ref, yd_ref, rep_ref = c.sign_derivative_apply(torch.from_numpy(x).cuda(), k)
    ys, yd, rep = c.sign_derivative_apply(torch.from_numpy(xb).cuda(), k)
    torch.cuda.synchronize()
    assert rep[0]["status"] == lq.LQ_ERR_NONFINITE, rep[0]
    assert rep[1]["status"] == lq.LQ_OK and rep[1]["k_eff"] == k, rep[1]
    # the other source is untouched: the same arithmetic as without the NaN
    assert torch.equal(ys[1], ys_ref[1]) and torch.equal(yd[1], yd_ref[1])
    assert rep_ref[0]["status"] == lq.LQ_OK
    # and the plain sign path
    y, rep = c.sign_apply(torch.from_numpy(xb).cuda(), k)
    torch.cuda.synchronize()
    assert rep[0]["status"] == lq.LQ_ERR_NONFINITE and rep[1]["status"] == lq.LQ_OK
    assert torch.isfinite(y[1]).all()


def test_newton_on_the_imaginary_axis_reports_failure(lqlib):
    """sgn is undefined for an eigenvalue with Re lambda = 0.  The real 2x2 block
    [[0, b], [-b, 0]] has eigenvalues +-ib and the Newton map keeps it exactly in that form
    (its inverse is [[0, -1/b], [1/b, 0]]), so the iteration never converges; the second
    matrix of the batch is regular and must still come out right."""
    from paper_1611_00195_gb300 import lq
    k = 4
    bad = np.array([[0, 0.7, 0, 0], [-0.7, 0, 0, 0], [0, 0, 1.3, 0.2], [0, 0, 0, -0.9]], dtype=complex)
    rng = np.random.default_rng(4)
    Q = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)) + 3 * np.eye(k)
    good = Q @ np.diag([1.1, -0.6 + 0.2j, 2.0, -1.4j + 0.5]) @ np.linalg.inv(Q)
    X = torch.from_numpy(np.stack([bad, good])).cuda()
    S = torch.zeros_like(X)
    it = (ctypes.c_int * 2)()
    c = lq.Context((2, 2, 2, 2))
    c.reserve(k, 2, False)
    L = lq.lib()
    code = L.lq_newton_sign(c._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(S.data_ptr()), k, 2, 50, 1e-13, it,
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert code == lq.LQ_ERR_NEWTON
    assert it[0] == 50
    assert relerr(S[1].cpu().numpy(), osg.sign_schur(good)) < 1e-12
    with pytest.raises(lq.LQError):
        c.newton_sign(X)
    # the allocation-free entry point reports the same status
    S2 = torch.zeros_like(X)
    code = L.lq_newton_sign_noalloc(ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(S2.data_ptr()), k, 2, 50, 1e-13, it,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == lq.LQ_ERR_NEWTON
