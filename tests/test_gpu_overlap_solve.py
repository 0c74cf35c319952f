"""The overlap solver and the conserved axial current (the paper's conclusion): z = D(m)^{-1} b
with D(m) = (1 - m/2) D_ov + m by BiCGStab on the library's Lanczos overlap operator, and the
per-noise estimates eta^dag D(m)^{-1} dD(m) gamma5 eta, against the dense oracle.  A solve cannot
be more accurate than the operator it iterates on, so each tolerance is the oracle's condition
number of D(m) times the measured error of the GPU's own D(m) application, times 30."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import dirac as od
from oracle import overlap as oo
from tests.helpers import relerr

pytestmark = pytest.mark.gpu
DIMS, MU = (2, 2, 2, 2), 0.3


def _setup(lq, prec, k):
    U = syn.gauge_field(DIMS, 0.4, 3)
    c = lq.Context(DIMS, mu=MU, precision=prec)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, 3, True, solve=True)
    return c, U, od.Lattice(DIMS)


def _apply_error(lq, c, lat, U, k, mass, E=None, theta=None):
    """Relative error of the GPU's D(m) x (and of its dD_ov x along theta) against the dense oracle."""
    x = syn.gaussian_source(DIMS, 77, nsrc=1)
    xt = torch.from_numpy(x).cuda()
    if theta is None:
        y = c.overlap_apply(xt, k, derivative=False)[0]
    else:
        y, dy, _ = c.overlap_apply(xt, k, kind=lq.LQ_DIR_U1, field=torch.from_numpy(theta).cuda())
    ym = (1 - mass / 2) * y[0].cpu().numpy().ravel() + mass * x[0].ravel()
    e = relerr(ym, oo.massive_overlap_dense(lat, U, MU, mass) @ x[0].ravel())
    if theta is not None:
        e = max(e, relerr(dy[0].cpu().numpy(), oo.overlap_derivative_dense(lat, U, MU, E) @ x[0].ravel()))
    return e


@pytest.mark.parametrize("prec,k,tol", [(0, 180, 1e-10), (1, 180, 1e-6)])
@pytest.mark.parametrize("mass", [0.0, 0.2])
def test_overlap_solve_against_dense(lqlib, prec, k, tol, mass):
    from paper_1611_00195_gb300 import lq
    c, U, lat = _setup(lq, prec, k)
    Dm = oo.massive_overlap_dense(lat, U, MU, mass)
    cond = np.linalg.cond(Dm)
    eD = _apply_error(lq, c, lat, U, k, mass)
    b = syn.gaussian_source(DIMS, 5, nsrc=3)
    z, rep = c.overlap_solve(torch.from_numpy(b).cuda(), k, mass=mass, tol=tol, max_iter=200)
    z = z.cpu().numpy()
    bound = max(1e-10, 30 * cond * max(eD, tol))
    for s in range(3):
        ex = np.linalg.solve(Dm, b[s].ravel())
        e = relerr(z[s], ex)
        print("prec %d m %.1f source %d: %d iterations, residual %.3g, error %.3g (cond %.3g, apply error %.3g, bound %.3g)"
              % (prec, mass, s, rep[s]["iterations"], rep[s]["residual"], e, cond, eD, bound))
        assert rep[s]["status"] == 0
        assert e < bound


@pytest.mark.parametrize("mass", [0.0, 0.2])
def test_axial_current_estimates_against_dense(lqlib, mass):
    from paper_1611_00195_gb300 import lq
    k, tol = 180, 1e-10
    c, U, lat = _setup(lq, lq.LQ_FP64, k)
    theta = syn.u1_direction(DIMS, 9)
    E = od.dense_dH_dir(lat, U, od.link_derivative(U, theta=theta), MU)
    eta = syn.z2_source(DIMS, 123, nsrc=3)
    ref = oo.axial_current_estimates(lat, U, MU, E, eta, mass)
    j, rep = c.axial_current(torch.from_numpy(eta).cuda(), k, kind=lq.LQ_DIR_U1, field=torch.from_numpy(theta).cuda(),
                             mass=mass, tol=tol, max_iter=200)
    Dm = oo.massive_overlap_dense(lat, U, MU, mass)
    dD = (1 - mass / 2) * oo.overlap_derivative_dense(lat, U, MU, E)
    scale = np.linalg.norm(eta[0]) ** 2 * np.linalg.norm(np.linalg.solve(Dm, dD), 2)
    e = _apply_error(lq, c, lat, U, k, mass, E, theta)
    bound = 30 * np.linalg.cond(Dm) * max(e, tol) * scale
    print("axial current m %.1f: GPU %s, oracle %s, |diff| %.3g (bound %.3g)" % (mass, j, ref, np.abs(j - ref).max(), bound))
    assert all(r["status"] == 0 for r in rep)
    assert np.abs(j - ref).max() < bound


def test_solver_errors(lqlib):
    from paper_1611_00195_gb300 import lq
    c, U, lat = _setup(lq, lq.LQ_FP64, 40)
    b = torch.from_numpy(syn.gaussian_source(DIMS, 5, nsrc=2)).cuda()
    z, rep = c.overlap_solve(b, 40, tol=1e-14, max_iter=1)
    assert all(r["status"] == -10 for r in rep)                      # LQ_ERR_NOT_CONVERGED
    c2 = lq.Context(DIMS, mu=MU, precision=0)
    c2.upload_gauge(torch.from_numpy(U).cuda())
    c2.reserve(40, 2, True)
    with pytest.raises(lq.LQError) as err:
        c2.overlap_solve(b, 40)
    assert err.value.code == -8
