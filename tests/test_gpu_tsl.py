"""GPU parity of the projected Newton sign and of the full two-sided Lanczos path (sign and
derivative, Sec. 2, Eqs. (2.5)-(2.6)) against the CPU oracle at the same Krylov depth."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import sign as osg
from oracle import tsl as ot
from tests.helpers import FP32_SENS_FACTOR, FP64_SENS_FACTOR, oracle_ops, relerr

pytestmark = pytest.mark.gpu


def _rand_matrix(rng, k, gap=1.0):
    # eigenvalues kept off the imaginary axis: A = Q diag(+-(gap + |z|)) Q^-1 + small noise
    lam = (gap + np.abs(rng.standard_normal(k))) * np.where(rng.random(k) < 0.5, -1, 1) + 0.3j * rng.standard_normal(k)
    Q = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)) + 3 * np.eye(k)
    return Q @ np.diag(lam) @ np.linalg.inv(Q)


@pytest.mark.parametrize("k", [1, 2, 7, 40, 130])
def test_newton_sign_dense(lqlib, k):
    from paper_1611_00195_gb300 import lq
    rng = np.random.default_rng(k)
    nb = 3
    X = np.stack([_rand_matrix(rng, k) for _ in range(nb)])
    c = lq.Context((2, 2, 2, 2))
    c.reserve(max(k, 2), nb, False)
    S, iters = c.newton_sign(torch.from_numpy(X).cuda())
    S = S.cpu().numpy()
    for b in range(nb):
        ref = osg.sign_schur(X[b])
        assert relerr(S[b], ref) < 1e-11, (b, iters)
        assert iters[b] < 30


def _sensitivity(run, x):
    """Relative change of the oracle's own result when its input is perturbed by 1e-16
    (relative, random): the rounding amplification of the non-symmetric Lanczos process at
    this depth.  Two correct FP64 implementations cannot agree better than about this."""
    rng = np.random.default_rng(99)
    xp = x * (1 + 1e-16 * rng.standard_normal(x.shape))
    a, b = run(x), run(xp)
    return max(relerr(bb, aa) for aa, bb in zip(a, b))


def _parity_tol(sens):
    return max(1e-11, FP64_SENS_FACTOR * sens)


CASES = [((4, 4, 4, 4), 64, 1), ((3, 2, 2, 2), 40, 3), ((6, 3, 5, 2), 50, 2)]


@pytest.mark.parametrize("dims,k,nsrc", CASES)
def test_sign_apply_fp64_parity(lqlib, dims, k, nsrc):
    from paper_1611_00195_gb300 import lq
    mu = 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5, nsrc=nsrc)
    c = lq.Context(dims, mu=mu, precision=lq.LQ_FP64)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, nsrc, False)
    y, rep = c.sign_apply(torch.from_numpy(x).cuda(), k)
    y = y.cpu().numpy()
    lat, A, Ah, E, Eh = oracle_ops(dims, U, mu)
    for s in range(nsrc):
        ref, r = ot.tsl_sign(A, Ah, x[s], k)
        assert rep[s]["status"] == 0 and rep[s]["k_eff"] == k
        # the recurrence itself: early coefficients agree to rounding
        al, be, de = c.tsl_coefficients(s, k)
        m = min(k, 12)
        assert np.abs(al[:m] - r["alpha"][:m]).max() < 1e-12 * np.abs(r["alpha"][:m]).max()
        assert np.abs(de[:m - 1] - r["delta"][:m - 1]).max() < 1e-12 * np.abs(r["delta"][:m - 1]).max()
        assert np.abs(be[:m - 1] - r["beta"][:m - 1]).max() < 1e-12 * np.abs(r["beta"][:m - 1]).max()
        sens = _sensitivity(lambda v: [ot.tsl_sign(A, Ah, v, k)[0]], x[s].ravel())
        err = relerr(y[s], ref)
        print("sign parity k=%d: rel err %.3g, oracle self-sensitivity %.3g (ratio %.2f)" % (k, err, sens, err / sens))
        assert err < _parity_tol(sens)


@pytest.mark.parametrize("dims,k,nsrc", CASES)
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_sign_derivative_fp64_parity(lqlib, dims, k, nsrc, kind, variant):
    from paper_1611_00195_gb300 import lq
    mu = 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5, nsrc=nsrc)
    field = syn.su3_direction(dims, 77) if kind == 1 else None
    c = lq.Context(dims, mu=mu, precision=lq.LQ_FP64)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, nsrc, True)
    ys, yd, rep = c.sign_derivative_apply(torch.from_numpy(x).cuda(), k, kind=kind,
                                          field=None if field is None else torch.from_numpy(field).cuda(),
                                          hop_variant=variant)
    ys, yd = ys.cpu().numpy(), yd.cpu().numpy()
    lat, A, Ah, E, Eh = oracle_ops(dims, U, mu, kind, field)
    for s in range(nsrc):
        rd, rs, r = ot.tsl_sign_derivative(A, Ah, E, Eh, x[s], k)
        assert rep[s]["status"] == 0 and rep[s]["k_eff"] == k
        al, be, de = c.tsl_coefficients(s, k)
        m = min(k, 12)
        assert np.abs(al[:m] - r["alpha"][:m]).max() < 1e-12 * np.abs(r["alpha"][:m]).max()
        assert np.abs(de[:m - 1] - r["delta"][:m - 1]).max() < 1e-12 * np.abs(r["delta"][:m - 1]).max()
        sens = _sensitivity(lambda v: ot.tsl_sign_derivative(A, Ah, E, Eh, v, k)[:2], x[s].ravel())
        es, ed = relerr(ys[s], rs), relerr(yd[s], rd)
        print("derivative parity k=%d: sign %.3g deriv %.3g, oracle self-sensitivity %.3g (ratio %.2f)"
              % (k, es, ed, sens, max(es, ed) / sens))
        assert es < _parity_tol(sens)
        assert ed < _parity_tol(sens)


@pytest.mark.parametrize("variant", list(range(10)))
@pytest.mark.parametrize("kind", [0, 1])
def test_sign_derivative_mixed_schedules(lqlib, variant, kind):
    """Every FP32 stencil schedule of the block TSL step (lq_opts.hop_variant) against the FP64
    oracle at the same depth.  FP32 arithmetic and storage perturb every step by about 6e-8
    (relative), so the bound scales with the oracle's own response to a 6e-8 relative random
    perturbation of every operator application (the FP32 analogue of the FP64 bound above).
    All schedules must also agree with each other to FP32 rounding.  The lattice (V = 192) leaves
    a ragged last block for the 128-site schedules and tiles exactly for schedule 6."""
    from paper_1611_00195_gb300 import lq
    dims, k, mu = (4, 4, 2, 6), 40, 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5, nsrc=2)
    field = syn.su3_direction(dims, 77) if kind == 1 else None
    c = lq.Context(dims, mu=mu, precision=lq.LQ_MIXED)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, 2, True)
    fd = None if field is None else torch.from_numpy(field).cuda()
    ys, yd, rep = c.sign_derivative_apply(torch.from_numpy(x).cuda(), k, kind=kind, field=fd, hop_variant=variant)
    ys, yd = ys.cpu().numpy(), yd.cpu().numpy()
    lat, A, Ah, E, Eh = oracle_ops(dims, U, mu, kind, field)
    rng = np.random.default_rng(11)

    def pert(op):
        return lambda v: (lambda y: y * (1 + 6e-8 * (rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape))
                                         / np.sqrt(2)))(op(v))
    for s in range(2):
        assert rep[s]["status"] == 0 and rep[s]["hop_variant"] == variant
        rd, rs, _ = ot.tsl_sign_derivative(A, Ah, E, Eh, x[s], k)
        sens = 0.0
        for _ in range(2):
            rdp, rsp, _ = ot.tsl_sign_derivative(pert(A), pert(Ah), pert(E), pert(Eh), x[s], k)
            sens = max(sens, relerr(rdp, rd), relerr(rsp, rs))
        es, ed = relerr(ys[s], rs), relerr(yd[s], rd)
        print("schedule %d direction %d mixed vs oracle k=%d: sign %.3g deriv %.3g (oracle FP32-size sensitivity %.3g, "
              "ratio %.2f)" % (variant, kind, k, es, ed, sens, max(es, ed) / sens))
        assert es < max(1e-6, FP32_SENS_FACTOR * sens) and ed < max(1e-6, FP32_SENS_FACTOR * sens)
    if variant > 0:
        y0s, y0d, _ = c.sign_derivative_apply(torch.from_numpy(x).cuda(), k, kind=kind, field=fd, hop_variant=0)
        # two FP32 schedules differ by rounding only: the same per-step bound as against the oracle
        tol = max(1e-6, FP32_SENS_FACTOR * sens)
        assert relerr(ys, y0s.cpu().numpy()) < tol and relerr(yd, y0d.cpu().numpy()) < tol


def test_mixed_converges_to_exact(lqlib):
    """Mixed path (FP32 stencil and vectors; FP64 dots, coefficients and Newton) against the
    exact dense sign and Frechet derivative of the oracle, at a depth where the FP64 method
    has converged below 1e-8 (sign) / 1e-6 (derivative).  FP32 vector storage delays the
    convergence; a CPU emulation of it (vectors rounded to complex64 each step) reaches
    3.3e-7 / 3.7e-6 on this case at k = 500, which bounds what the mixed path can reach."""
    from oracle import dirac as od
    from paper_1611_00195_gb300 import lq
    dims, k, mu = (4, 4, 2, 2), 500, 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5, nsrc=1)
    c = lq.Context(dims, mu=mu, precision=lq.LQ_MIXED)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, 1, True)
    ys, yd, rep = c.sign_derivative_apply(torch.from_numpy(x).cuda(), k)
    lat = od.Lattice(dims)
    H = od.dense_H(lat, U, mu)
    ex = osg.sign_schur(H) @ x[0].ravel()
    exd = osg.frechet_sylvester(H, od.dense_dH_dmu(lat, U, mu)) @ x[0].ravel()
    es, ed = relerr(ys[0].cpu().numpy(), ex), relerr(yd[0].cpu().numpy(), exd)
    print("mixed vs exact at k=%d: sign %.3g deriv %.3g" % (k, es, ed))
    assert rep[0]["status"] == 0
    assert es < 1e-6 and ed < 1e-5


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims,k", [((4, 4, 4, 4), 64), ((6, 3, 5, 2), 120), ((3, 2, 2, 2), 1), ((3, 2, 2, 2), 2)])
def test_projected_quadrature_matches_newton(lqlib, prec, dims, k):
    """The same Lanczos run finished by the Newton iteration and by the quadrature of
    sgn(T) = (2/pi) T int (t^2 + T^2)^{-1} dt must give the same sgn(T_k) e_1 (to rounding),
    and the automatic choice must accept the quadrature through its involution check."""
    from paper_1611_00195_gb300 import lq
    mu = 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    x = torch.from_numpy(syn.gaussian_source(dims, 5, nsrc=2)).cuda()
    c = lq.Context(dims, mu=mu, precision=prec)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, 2, True)
    out = {}
    for proj in (lq.LQ_PROJ_NEWTON, lq.LQ_PROJ_QUAD, lq.LQ_PROJ_AUTO):
        ys, yd, rep = c.sign_derivative_apply(x, k, projected=proj)
        out[proj] = (ys.cpu().numpy(), yd.cpu().numpy(), rep)
    for s in range(2):
        rq = out[lq.LQ_PROJ_QUAD][2][s]
        errs = []
        for i in (0, 1):
            a, b = out[lq.LQ_PROJ_QUAD][i][s], out[lq.LQ_PROJ_NEWTON][i][s]
            errs.append(0.0 if np.linalg.norm(b) == 0 else relerr(a, b))
        print("quadrature k=%d: check %.3g, vs Newton sign %.3g deriv %.3g, auto used %d"
              % (k, rq["proj_check"], errs[1], errs[0], out[lq.LQ_PROJ_AUTO][2][s]["projected"]))
        assert out[lq.LQ_PROJ_NEWTON][2][s]["projected"] == lq.LQ_PROJ_NEWTON
        assert rq["projected"] == lq.LQ_PROJ_QUAD
        assert rq["proj_check"] < 1e-11
        assert out[lq.LQ_PROJ_AUTO][2][s]["projected"] == lq.LQ_PROJ_QUAD
        assert max(errs) < 1e-11
        for i in (0, 1):
            assert np.array_equal(out[lq.LQ_PROJ_AUTO][i][s], out[lq.LQ_PROJ_QUAD][i][s])


def test_projected_auto_falls_back_to_newton(lqlib):
    """With an involution tolerance no quadrature can meet, the automatic choice must climb
    the node ladder, then finish with the Newton iteration and say so."""
    from paper_1611_00195_gb300 import lq
    dims, k, mu = (4, 4, 4, 4), 64, 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    x = torch.from_numpy(syn.gaussian_source(dims, 5, nsrc=1)).cuda()
    c = lq.Context(dims, mu=mu)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, 1, False)
    yn, rn = c.sign_apply(x, k, projected=lq.LQ_PROJ_NEWTON)
    ya, ra = c.sign_apply(x, k, projected=lq.LQ_PROJ_AUTO, quad_nodes=2, proj_tol=1e-300)
    assert ra[0]["projected"] == lq.LQ_PROJ_NEWTON and ra[0]["status"] == 0
    assert relerr(ya.cpu().numpy(), yn.cpu().numpy()) < 1e-15


def test_projected_auto_node_ladder(lqlib):
    """A quadrature started far too coarse (2 nodes) must be retried with the large node count
    until its involution residual passes, per source, without the Newton fallback, and then
    agree with the Newton iteration."""
    from paper_1611_00195_gb300 import lq
    dims, k, mu = (4, 4, 4, 4), 64, 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    x = torch.from_numpy(syn.gaussian_source(dims, 5, nsrc=2)).cuda()
    c = lq.Context(dims, mu=mu)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, 2, False)
    yn, rn = c.sign_apply(x, k, projected=lq.LQ_PROJ_NEWTON)
    ya, ra = c.sign_apply(x, k, projected=lq.LQ_PROJ_AUTO, quad_nodes=2, proj_tol=1e-11)
    for s in range(2):
        print("ladder: source %d check %.3g" % (s, ra[s]["proj_check"]))
        assert ra[s]["projected"] == lq.LQ_PROJ_QUAD and ra[s]["status"] == 0
        assert ra[s]["proj_check"] <= 1e-11
        assert relerr(ya[s].cpu().numpy(), yn[s].cpu().numpy()) < 1e-10


@pytest.mark.parametrize("dims,k", [((3, 2, 2, 2), 40), ((4, 4, 4, 4), 64)])
@pytest.mark.parametrize("deriv", [False, True])
def test_error_estimate_parity(lqlib, dims, k, deriv):
    """eps_A of Sec. 4 (sign, and the derivative version with B and (0, x)) against the
    oracle's own estimate at the same depth."""
    from paper_1611_00195_gb300 import lq
    mu = 0.3
    U = syn.gauge_field(dims, 0.4, 3)
    x = syn.gaussian_source(dims, 5, nsrc=2)
    c = lq.Context(dims, mu=mu)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, 2, True)
    eps = c.error_estimate(torch.from_numpy(x).cuda(), k, kind=lq.LQ_DIR_MU if deriv else None)
    lat, A, Ah, E, Eh = oracle_ops(dims, U, mu)
    for s in range(2):
        if deriv:
            ref = ot.error_estimate_derivative(A, Ah, E, Eh, x[s], k)
        else:
            ref = ot.error_estimate(A, Ah, x[s], k)
        print("eps_A %s k=%d: gpu %.6e oracle %.6e" % ("deriv" if deriv else "sign", k, eps[s], ref))
        assert abs(eps[s] - ref) <= 1e-6 * ref


@pytest.mark.parametrize("dims", [(4, 4, 2, 6), (6, 4, 4, 4), (5, 3, 3, 4)])
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_packed_schedules_are_bitwise_schedule_3(lqlib, dims, kind):
    """Schedules 7 and 8 (packed FP32 pair arithmetic, the hop factor -1/2 taken out of the sum,
    and for 8 the prefetched neighbours) perform the same roundings in the same order as schedule 3: every result, report and Lanczos coefficient must be bitwise identical, for the three
    derivative kinds (d/dmu, su(3) and U(1) link directions), on lattices whose site count leaves
    a ragged last block of the 128-site grid (V = 192, 384, 180)."""
    from paper_1611_00195_gb300 import lq
    k, mu, nsrc = 30, 0.3, 3
    U = syn.gauge_field(dims, 0.4, 3)
    x = torch.from_numpy(syn.gaussian_source(dims, 5, nsrc=nsrc)).cuda()
    field = None
    if kind == 1:
        field = torch.from_numpy(syn.su3_direction(dims, 77)).cuda()
    elif kind == 2:
        field = torch.from_numpy(syn.u1_direction(dims, 78)).cuda()
    c = lq.Context(dims, mu=mu, precision=lq.LQ_MIXED)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, nsrc, True)
    out = {}
    for v in (3, 7, 8):
        ys, yd, rep = c.sign_derivative_apply(x, k, kind=kind, field=field, hop_variant=v)
        coef = [c.tsl_coefficients(s, k) for s in range(nsrc)]
        out[v] = (ys.cpu().numpy(), yd.cpu().numpy(), rep, coef)
        assert all(r["hop_variant"] == v and r["status"] == 0 for r in rep)
    for v in (7, 8):
        assert np.array_equal(out[v][0], out[3][0]) and np.array_equal(out[v][1], out[3][1])
        for s in range(nsrc):
            for a, b in zip(out[v][3][s], out[3][3][s]):
                assert np.array_equal(a, b)
