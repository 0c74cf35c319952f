"""GPU parity of the adjoint (fermionic force): S = Re <y| sgn(H(mu)) |x>, dS/dw^a_nu(s) for every
link and generator, and dS/dmu, against the oracle's Krylov route at the same depth, the dense
trace-identity route at a converged depth, central finite differences of the GPU's own S along
random link directions, and the torch.autograd.Function wrapper."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

import synthetic as syn
from oracle import adjoint as oad
from oracle import dirac as od

pytestmark = pytest.mark.gpu

MU = 0.3


def _ctx(lq, dims, U, k, prec=0):
    c = lq.Context(dims, mu=MU, precision=prec)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, 2, block=False, adjoint=True)
    return c


@pytest.mark.parametrize("dims,k", [((4, 2, 2, 2), 80), ((3, 2, 2, 2), 60), ((4, 4, 4, 4), 64)])
def test_force_parity_same_depth(lqlib, dims, k):
    from paper_1611_00195_gb300 import lq
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5)
    y = syn.gaussian_source(dims, 6)
    c = _ctx(lq, dims, U, k)
    S, F, dmu = c.bilinear_grad(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), k)
    F = F.cpu().numpy()
    So, Fo, dmuo = oad.grad_tsl(lat, U, x, y, MU, k)
    # rounding sensitivity of the oracle itself to 1e-16 perturbations of either input (the
    # left basis of the y process can be badly conditioned)
    rng = np.random.default_rng(1)
    sens = 0.0
    for xp, yp in ((x * (1 + 1e-16 * rng.standard_normal(x.shape)), y), (x, y * (1 + 1e-16 * rng.standard_normal(y.shape)))):
        Sp, Fp, dmup = oad.grad_tsl(lat, U, xp, yp, MU, k)
        sens = max(sens, np.linalg.norm(Fp - Fo) / np.linalg.norm(Fo))
    eF = np.linalg.norm(F - Fo) / np.linalg.norm(Fo)
    print("force parity %s k=%d: S %.3g F %.3g dmu %.3g (oracle self-sensitivity %.3g)"
          % (dims, k, abs(S - So) / abs(So), eF, abs(dmu - dmuo) / abs(dmuo), sens))
    tol = max(1e-10, 30 * sens)
    assert eF < tol
    assert abs(S - So) < tol * abs(So) and abs(dmu - dmuo) < tol * max(abs(dmuo), 1e-3)


def test_force_against_dense_and_finite_differences(lqlib):
    """At a converged depth on 2^4 the Krylov force matches the dense trace-identity route, and
    central differences (step 1e-4) of the GPU's own S along random link directions match the
    force contracted with those directions."""
    from paper_1611_00195_gb300 import lq
    dims, k = (2, 2, 2, 2), 150
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.3, 3)
    x = syn.gaussian_source(dims, 5)
    y = syn.gaussian_source(dims, 6)
    c = _ctx(lq, dims, U, k)
    S, F, dmu = c.bilinear_grad(x, y, k)
    Sd, Fd, dmud = oad.grad_dense(lat, U, x, y, MU)
    eF = np.linalg.norm(F - Fd) / np.linalg.norm(Fd)
    print("force vs dense k=%d: S %.3g F %.3g dmu %.3g" % (k, abs(S - Sd) / abs(Sd), eF, abs(dmu - dmud) / abs(dmud)))
    assert eF < 1e-6 and abs(S - Sd) < 1e-8 * abs(Sd)
    h = 1e-4
    for seed in range(16):
        om = syn.su3_direction(dims, 100 + seed)
        Om = od.su3_tangent(om)
        Ups = []
        for t in (h, -h):
            Ut = np.einsum("dsij,dsjk->dsik", np.array([[sla.expm(1j * t * Om[d, s]) for s in range(lat.V)] for d in range(4)]), U)
            c.upload_gauge(Ut)
            Ups.append(c.bilinear_grad(x, y, k)[0])
        c.upload_gauge(U)
        fd = (Ups[0] - Ups[1]) / (2 * h)
        assert abs(fd - np.sum(om * F)) < 1e-6 * max(1.0, np.abs(F).max())


def test_autograd_function(lqlib):
    from paper_1611_00195_gb300 import lq
    dims, k = (4, 2, 2, 2), 80
    U = syn.gauge_field(dims, 0.4, 3)
    x = torch.from_numpy(syn.gaussian_source(dims, 5)).cuda()
    y = torch.from_numpy(syn.gaussian_source(dims, 6)).cuda()
    c = _ctx(lq, dims, U, k)
    V = int(np.prod(dims))
    omega = torch.zeros((4, V, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    mu = torch.tensor(MU, dtype=torch.float64, requires_grad=True)
    S = lq.SignBilinearForce.apply(omega, mu, c, x, y, k)
    (2.0 * S).backward()
    S2, F, dmu = c.bilinear_grad(x, y, k)
    assert abs(S.item() - S2) < 1e-14 * abs(S2)
    assert torch.allclose(omega.grad, 2.0 * F)
    assert abs(mu.grad.item() - 2.0 * dmu) < 1e-14 * abs(dmu)


def test_force_mixed_precision(lqlib):
    from paper_1611_00195_gb300 import lq
    dims, k = (4, 2, 2, 2), 80
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5)
    y = syn.gaussian_source(dims, 6)
    c64 = _ctx(lq, dims, U, k, 0)
    c32 = _ctx(lq, dims, U, k, 1)
    S64, F64, d64 = c64.bilinear_grad(x, y, k)
    S32, F32, d32 = c32.bilinear_grad(x, y, k)
    e = np.linalg.norm(F32 - F64) / np.linalg.norm(F64)
    print("force mixed vs fp64 k=%d: %.3g" % (k, e))
    assert e < 1e-3
