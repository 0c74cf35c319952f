"""GPU parity of the stencil kernels (Eq. (1.1), block operator of Eq. (2.5)) against the
CPU oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import dirac as od
from tests.helpers import oracle_ops, relerr

pytestmark = pytest.mark.gpu

DIMS = [(4, 4, 4, 4), (6, 3, 5, 2), (3, 2, 2, 2), (2, 1, 3, 1)]


def make_ctx(lq, dims, mu, prec, U, kmax=4, nsrc=3, block=True):
    c = lq.Context(dims, m_w=-2.0, mu=mu, precision=prec)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(kmax, nsrc, block)
    return c


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_H(lqlib, dims, prec, dagger):
    from paper_1611_00195_gb300 import lq
    mu = 0.3
    U = syn.gauge_field(dims, 0.4, 11)
    x = syn.gaussian_source(dims, 12, nsrc=3)
    c = make_ctx(lq, dims, mu, prec, U)
    y = c.apply_H(torch.from_numpy(x).cuda(), dagger=dagger).cpu().numpy()
    lat = od.Lattice(dims)
    f = od.apply_Hdag if dagger else od.apply_H
    tol = 1e-14 if prec == 0 else 2e-6
    for s in range(3):
        assert relerr(y[s], f(lat, U, x[s], mu)) < tol


def test_apply_H_host_buffers(lqlib):
    """Host (numpy) buffers go through the library's own staging copies."""
    from paper_1611_00195_gb300 import lq
    dims, mu = (4, 2, 3, 2), -0.2
    U = syn.gauge_field(dims, 0.4, 1)
    x = syn.gaussian_source(dims, 2, nsrc=2)
    c = lq.Context(dims, mu=mu)
    c.upload_gauge(U)
    c.reserve(2, 2, False)
    y = c.apply_H(x)
    assert isinstance(y, np.ndarray)
    lat = od.Lattice(dims)
    for s in range(2):
        assert relerr(y[s], od.apply_H(lat, U, x[s], mu)) < 1e-14


@pytest.mark.parametrize("dims", DIMS[:3])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_block(lqlib, dims, prec, kind, dagger):
    from paper_1611_00195_gb300 import lq
    mu = 0.3
    U = syn.gauge_field(dims, 0.4, 21)
    field = None
    if kind == 1:
        field = syn.su3_direction(dims, 77)
    elif kind == 2:
        field = syn.u1_direction(dims, 78)
    xt = syn.gaussian_source(dims, 31, nsrc=2)
    xb = syn.gaussian_source(dims, 32, nsrc=2)
    c = make_ctx(lq, dims, mu, prec, U, nsrc=2)
    c.set_direction(kind, None if field is None else torch.from_numpy(field).cuda())
    yt, yb = c.apply_block(torch.from_numpy(xt).cuda(), torch.from_numpy(xb).cuda(), dagger=dagger)
    yt, yb = yt.cpu().numpy(), yb.cpu().numpy()
    lat, A, Ah, E, Eh = oracle_ops(dims, U, mu, kind, field)
    tol = 1e-14 if prec == 0 else 2e-6
    for s in range(2):
        t, b = xt[s].ravel(), xb[s].ravel()
        if not dagger:
            rt, rb = A(t) + E(b), A(b)
        else:
            rt, rb = Ah(t), Eh(t) + Ah(b)
        assert relerr(np.concatenate([yt[s].ravel(), yb[s].ravel()]), np.concatenate([rt, rb])) < tol
