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
from tests.helpers import ADJ_SENS_FACTOR

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
    tol = max(1e-10, ADJ_SENS_FACTOR * sens)
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


def _exp_direction(U, omega, t):
    """Links exp(i t Omega_nu(x)) U_nu(x) for the su(3) field omega [4][V][8] (batched
    eigendecomposition of the Hermitian Omega; test infrastructure only)."""
    w, Q = np.linalg.eigh(od.su3_tangent(omega))
    E = np.einsum("dsij,dsj,dskj->dsik", Q, np.exp(1j * t * w), Q.conj())
    return np.einsum("dsij,dsjk->dsik", E, U)


def test_force_workload_12x12c3(lqlib):
    """The differentiation workload at full size: 12x12^3 (n = 248832), eps = 0.4, mu = 0.3,
    Gaussian x and y.  (a) At the workload's depth k = 300, the torch.autograd.Function (mixed
    and FP64) gives the force for all 4 V links x 8 generators and dS/dmu within 10 eps_A of
    the converged force (eps_A of Sec. 4 for x and y at that depth).  (b) At a depth where the
    process has converged (k = 1800, eps_A <= 1e-10), central differences with step 1e-4 of
    S = Re <y|sgn(H)|x> (each S one FP64 solve on the GPU) along 16 random su(3) link
    directions and in mu agree with the force.  Below convergence the finite differences
    measure the change of the Krylov truncation error with the links, not the derivative."""
    from paper_1611_00195_gb300 import lq
    dims, h = (12, 12, 12, 12), 1e-4
    V = int(np.prod(dims))
    U = syn.gauge_field(dims, 0.4, 3)
    x = torch.from_numpy(syn.gaussian_source(dims, 5)).cuda()
    y = torch.from_numpy(syn.gaussian_source(dims, 6)).cuda()
    kc = 1800
    c = _ctx(lq, dims, U, kc)
    S, F, dmu = c.bilinear_grad(x, y, kc)
    F = F.cpu().numpy()
    x1 = x.reshape(1, V, 4, 3)
    eps_c = max(c.error_estimate(x1, kc)[0], c.error_estimate(y.reshape(1, V, 4, 3), kc)[0])
    assert eps_c <= 1e-10, eps_c

    def S_of():
        z, rep = c.sign_apply(x1, kc)
        assert rep[0]["status"] == 0
        return float(torch.real(torch.vdot(y.reshape(-1), z.reshape(-1))))
    worst = 0.0
    for seed in range(16):
        om = syn.su3_direction(dims, 100 + seed)
        Sp = []
        for t in (h, -h):
            c.upload_gauge(torch.from_numpy(_exp_direction(U, om, t)).cuda())
            Sp.append(S_of())
        d = float(np.sum(om * F))
        fd = (Sp[0] - Sp[1]) / (2 * h)
        worst = max(worst, abs(fd - d) / abs(d))
        assert abs(fd - d) <= 1e-4 * abs(d) + 1e-12, (seed, fd, d)
    c.upload_gauge(torch.from_numpy(U).cuda())
    Sm = []
    for m in (MU + h, MU - h):
        c.set_mu(m)
        Sm.append(S_of())
    c.set_mu(MU)
    fdm = (Sm[0] - Sm[1]) / (2 * h)
    print("12^4 k=%d (eps_A %.2g): force vs central differences on 16 directions, worst rel %.3g; dS/dmu %.3g"
          % (kc, eps_c, worst, abs(fdm - dmu) / abs(dmu)))
    assert abs(fdm - dmu) <= 1e-6 * abs(dmu)
    del c

    k = 300
    for prec in (1, 0):
        cw = _ctx(lq, dims, U, k, prec)
        omega = torch.zeros((4, V, 8), dtype=torch.float64, device="cuda", requires_grad=True)
        mu = torch.tensor(MU, dtype=torch.float64, requires_grad=True)
        Sw = lq.SignBilinearForce.apply(omega, mu, cw, x, y, k)
        Sw.backward()
        eps_k = max(cw.error_estimate(x1, k)[0], cw.error_estimate(y.reshape(1, V, 4, 3), k)[0])
        eF = float(np.linalg.norm(omega.grad.cpu().numpy() - F) / np.linalg.norm(F))
        emu = abs(mu.grad.item() - dmu) / abs(dmu)
        eS = abs(Sw.item() - S) / abs(S)
        print("12^4 k=%d prec %d via autograd: S %.3g force %.3g dS/dmu %.3g against the converged values (eps_A %.3g)"
              % (k, prec, eS, eF, emu, eps_k))
        assert max(eS, eF, emu) <= 10 * eps_k
        del cw


def _upload_eigenpairs(c, lat, U, l):
    from oracle import deflation as odf
    H = od.dense_H(lat, U, MU)
    lam, R, L, _ = odf.eigenpairs(H, l)
    c.upload_deflation(lam, torch.from_numpy(np.ascontiguousarray(R.T.reshape(l, lat.V, 4, 3))).cuda(),
                       torch.from_numpy(np.ascontiguousarray(L.conj().reshape(l, lat.V, 4, 3))).cuda())
    return lam, R, L


@pytest.mark.parametrize("dims,k,l", [((4, 2, 2, 2), 80, 6), ((2, 2, 2, 2), 60, 8)])
def test_deflated_force_parity_same_depth(lqlib, dims, k, l):
    """The deflated adjoint (opts.deflate = 1) against the oracle's deflated Krylov route at the
    same depth, with the oracle's eigenpairs installed: S, the force on every link and dS/dmu,
    within ADJ_SENS_FACTOR times the oracle's own rounding sensitivity."""
    from paper_1611_00195_gb300 import lq
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5)
    y = syn.gaussian_source(dims, 6)
    c = _ctx(lq, dims, U, k)
    lam, R, L = _upload_eigenpairs(c, lat, U, l)
    S, F, dmu = c.bilinear_grad(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), k, deflate=1)
    F = F.cpu().numpy()
    A = lambda v: od.apply_H(lat, U, v, MU).ravel()        # noqa: E731
    Ah = lambda v: od.apply_Hdag(lat, U, v, MU).ravel()    # noqa: E731

    def oracle(xx, yy):
        G, So = oad.G_deflated_tsl(A, Ah, lam, R, L, xx.ravel(), yy.ravel(), k)
        return So, oad.force_from_G(lat, U, G, MU), oad.dmu_from_G(lat, U, G, MU)
    So, Fo, dmuo = oracle(x, y)
    rng = np.random.default_rng(1)
    sens = 0.0
    for xp, yp in ((x * (1 + 1e-16 * rng.standard_normal(x.shape)), y), (x, y * (1 + 1e-16 * rng.standard_normal(y.shape)))):
        Sp, Fp, dmup = oracle(xp, yp)
        sens = max(sens, np.linalg.norm(Fp - Fo) / np.linalg.norm(Fo))
    eF = np.linalg.norm(F - Fo) / np.linalg.norm(Fo)
    print("deflated force parity %s k=%d l=%d: S %.3g F %.3g dmu %.3g (oracle self-sensitivity %.3g)"
          % (dims, k, l, abs(S - So) / abs(So), eF, abs(dmu - dmuo) / abs(dmuo), sens))
    tol = max(1e-10, ADJ_SENS_FACTOR * sens)
    assert eF < tol
    assert abs(S - So) < tol * abs(So) and abs(dmu - dmuo) < tol * max(abs(dmuo), 1e-3)


@pytest.mark.parametrize("prec", [0, 1])
def test_deflated_force_converges(lqlib, prec):
    """At a converged depth on 2^4 the deflated force equals the dense one (and the undeflated
    GPU force); in mixed precision it matches the FP64 deflated force to FP32 accuracy."""
    from paper_1611_00195_gb300 import lq
    dims, k, l = (2, 2, 2, 2), 150, 8
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.3, 3)
    x = syn.gaussian_source(dims, 5)
    y = syn.gaussian_source(dims, 6)
    c = _ctx(lq, dims, U, k, prec)
    _upload_eigenpairs(c, lat, U, l)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    S, F, dmu = c.bilinear_grad(xt, yt, k, deflate=1)
    S0, F0, dmu0 = c.bilinear_grad(xt, yt, k)
    F, F0 = F.cpu().numpy(), F0.cpu().numpy()
    Sd, Fd, dmud = oad.grad_dense(lat, U, x, y, MU)
    eF, eF0 = np.linalg.norm(F - Fd) / np.linalg.norm(Fd), np.linalg.norm(F0 - Fd) / np.linalg.norm(Fd)
    print("prec %d k=%d: deflated force vs dense %.3g (undeflated %.3g); S %.3g dmu %.3g"
          % (prec, k, eF, eF0, abs(S - Sd) / abs(Sd), abs(dmu - dmud) / abs(dmud)))
    tol = 1e-6 if prec == 0 else 1e-3
    assert eF < tol and abs(S - Sd) < tol * abs(Sd) and abs(dmu - dmud) < tol * abs(dmud)


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-6)])
def test_two_pass_adjoint(lqlib, prec, tol):
    """The adjoint with O(n) memory (lq_opts.two_pass on a workspace reserved with
    LQ_RESERVE_ADJOINT | LQ_RESERVE_TWO_PASS): rings of 32 right and left basis vectors per
    source; the second pass accumulates the 2N pair vectors of the force window by window.  The
    processes are the same, so S, the force and dS/dmu equal the one-pass run up to the order of
    the recombination sums (k = 100 wraps the rings three times; 4x4x2x6).  The FP64 two-pass
    force is also checked against the oracle's Krylov route at the same depth."""
    from paper_1611_00195_gb300 import lq
    dims, k = (4, 4, 2, 6), 100
    lat = od.Lattice(dims)
    U = syn.gauge_field(dims, 0.4, 3)
    x = torch.from_numpy(syn.gaussian_source(dims, 5)).cuda()
    y = torch.from_numpy(syn.gaussian_source(dims, 6)).cuda()
    c1 = _ctx(lq, dims, U, k, prec)
    c2 = lq.Context(dims, mu=MU, precision=prec)
    c2.upload_gauge(torch.from_numpy(U).cuda())
    c2.reserve(k, 2, block=False, adjoint=True, two_pass=True)
    S1, F1, m1 = c1.bilinear_grad(x, y, k)
    S2, F2, m2 = c2.bilinear_grad(x, y, k, two_pass=1)
    F1, F2 = F1.cpu().numpy(), F2.cpu().numpy()
    eF = np.linalg.norm(F2 - F1) / np.linalg.norm(F1)
    print("two-pass adjoint prec %d: S %.3g F %.3g dmu %.3g against one pass"
          % (prec, abs(S2 - S1) / abs(S1), eF, abs(m2 - m1) / abs(m1)))
    assert eF < tol and abs(S2 - S1) < tol * abs(S1) and abs(m2 - m1) < tol * abs(m1)
    with pytest.raises(lq.LQError):
        c2.bilinear_grad(x, y, k)                     # deeper than the ring without two_pass
    if prec == 0:
        So, Fo, mo = oad.grad_tsl(lat, U, x.cpu().numpy(), y.cpu().numpy(), MU, k)
        rng = np.random.default_rng(1)
        xp = x.cpu().numpy() * (1 + 1e-16 * rng.standard_normal(x.shape))
        Sp, Fp, mp = oad.grad_tsl(lat, U, xp, y.cpu().numpy(), MU, k)
        sens = np.linalg.norm(Fp - Fo) / np.linalg.norm(Fo)
        e = np.linalg.norm(F2 - Fo) / np.linalg.norm(Fo)
        print("two-pass adjoint FP64 vs oracle: F %.3g (sensitivity %.3g)" % (e, sens))
        assert e < max(1e-10, ADJ_SENS_FACTOR * sens)
