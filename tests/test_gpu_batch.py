"""Ragged batches through lq_batch_apply: several lattices of uneven size, parameters, sources
and Krylov depth in one CUDA graph launch.  Each member must equal, bit for bit, the
single-problem call on the same context (same kernels, schedule and reduction order), and the
FP64 members agree with the oracle's two-sided Lanczos process (Sec. 2) at the same depth."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import tsl as ot
from tests.helpers import FP64_SENS_FACTOR, oracle_ops, relerr

pytestmark = pytest.mark.gpu


def _member(lq, dims, eps, mu, k, nsrc, prec, seed, kind, z2=False):
    U = syn.gauge_field(dims, eps, seed)
    c = lq.Context(dims, mu=mu, precision=prec)
    c.upload_gauge(torch.from_numpy(U).cuda())
    c.reserve(k, nsrc, kind is not None)
    gen = syn.z2_source if z2 else syn.gaussian_source
    x = torch.from_numpy(gen(dims, seed + 100, nsrc=nsrc)).cuda()
    field = None
    if kind == 1:
        field = syn.su3_direction(dims, seed + 200)
    elif kind == 2:
        field = syn.u1_direction(dims, seed + 300)
    return {"ctx": c, "x": x, "k": k, "kind": kind,
            "field": None if field is None else torch.from_numpy(field).cuda()}, U, field


def _single(m):
    c = m["ctx"]
    if m["kind"] is None:
        y, rep = c.sign_apply(m["x"], m["k"])
        return y, None, rep
    return c.sign_derivative_apply(m["x"], m["k"], kind=m["kind"], field=m["field"])


def _assert_same(a, b):
    ys, yd, ra = a
    zs, zd, rb = b
    assert torch.equal(ys, zs)
    assert (yd is None) == (zd is None)
    if yd is not None:
        assert torch.equal(yd, zd)
    for p, q in zip(ra, rb):
        assert (p["status"], p["k_eff"], p["hop_variant"], p["projected"]) == \
               (q["status"], q["k_eff"], q["hop_variant"], q["projected"])


# (dims, eps, mu, k, nsrc, kind): tiles, ragged last blocks, periodic-size mixes, three
# direction kinds and a sign-only member
SMALL = [((4, 4, 2, 6), 0.4, 0.3, 40, 2, 0), ((2, 2, 2, 4), 0.5, 0.1, 25, 1, None),
         ((6, 3, 5, 2), 0.3, 0.2, 50, 3, 1), ((4, 4, 4, 4), 0.4, 0.3, 64, 1, 2)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("graph", [-1, 0])
def test_batch_equals_single_calls(lqlib, prec, graph):
    from paper_1611_00195_gb300 import lq
    members = [_member(lq, d, e, mu, k, n, prec, 11 + i, kind)[0] for i, (d, e, mu, k, n, kind) in enumerate(SMALL)]
    singles = [_single(m) for m in members]           # tunes each context's schedule first
    for m in members:
        m["graph"] = graph
    for rep in range(2):                              # capture, then replay
        out = lq.batch_apply(members)
        for a, b in zip(out, singles):
            _assert_same(a, b)
            assert all(r["status"] == 0 for r in a[2])


def test_batch_fp64_parity_with_oracle(lqlib):
    from paper_1611_00195_gb300 import lq
    built = [_member(lq, d, e, mu, k, n, lq.LQ_FP64, 11 + i, kind) for i, (d, e, mu, k, n, kind) in enumerate(SMALL)]
    out = lq.batch_apply([b[0] for b in built])
    rng = np.random.default_rng(5)
    for (m, U, field), (d, e, mu, k, n, kind), (ys, yd, rep) in zip(built, SMALL, out):
        lat, A, Ah, E, Eh = oracle_ops(d, U, mu, kind or 0, field)
        x = m["x"].cpu().numpy()
        for s in range(n):
            assert rep[s]["status"] == 0 and rep[s]["k_eff"] == k

            def run(v):
                if kind is None:
                    return [ot.tsl_sign(A, Ah, v, k)[0]]
                return list(ot.tsl_sign_derivative(A, Ah, E, Eh, v, k)[:2])
            ref = run(x[s].ravel())
            xp = x[s].ravel() * (1 + 1e-16 * rng.standard_normal(x[s].size))
            sens = max(relerr(p, q) for p, q in zip(run(xp), ref))
            got = [ys[s].cpu().numpy()] if kind is None else [yd[s].cpu().numpy(), ys[s].cpu().numpy()]
            errs = [relerr(g, r) for g, r in zip(got, ref)]
            print("batch member %s k=%d src %d: rel err %s, sensitivity %.3g" % (d, k, s, errs, sens))
            assert max(errs) < max(1e-11, FP64_SENS_FACTOR * sens)


@pytest.mark.parametrize("prec", [0, 1])
def test_ragged_workload(lqlib, prec):
    """The ragged batch of the batching workload at full size (6^4, 8^4, 8x12^3, 10^4 with
    depths 100-300, Z2 sources, d/dmu): every member equals its single call bit for bit, all
    sources finish at full depth; in FP64 the 6^4 member also matches the oracle."""
    from paper_1611_00195_gb300 import lq
    nsrc = 2
    built = [_member(lq, d, e, syn.RAGGED_MU, k, nsrc, prec, seed, 0, z2=True) for d, e, k, seed in syn.RAGGED_BATCH]
    members = [b[0] for b in built]
    singles = [_single(m) for m in members]
    out = lq.batch_apply(members)
    for (d, e, k, seed), a, b in zip(syn.RAGGED_BATCH, out, singles):
        _assert_same(a, b)
        assert all(r["status"] == 0 and r["k_eff"] == k for r in a[2]), (d, a[2])
    if prec == lq.LQ_FP64:
        (m, U, _), (d, e, k, seed) = built[0], syn.RAGGED_BATCH[0]
        lat, A, Ah, E, Eh = oracle_ops(d, U, syn.RAGGED_MU)
        x = m["x"][0].cpu().numpy().ravel()
        rd, rs, _ = ot.tsl_sign_derivative(A, Ah, E, Eh, x, k)
        rng = np.random.default_rng(7)
        pd, ps, _ = ot.tsl_sign_derivative(A, Ah, E, Eh, x * (1 + 1e-16 * rng.standard_normal(x.size)), k)
        sens = max(relerr(pd, rd), relerr(ps, rs))
        es, ed = relerr(out[0][0][0].cpu().numpy(), rs), relerr(out[0][1][0].cpu().numpy(), rd)
        print("ragged 6^4 k=%d vs oracle: sign %.3g deriv %.3g (sensitivity %.3g)" % (k, es, ed, sens))
        assert max(es, ed) < max(1e-11, FP64_SENS_FACTOR * sens)


def test_batch_argument_errors(lqlib):
    from paper_1611_00195_gb300 import lq
    m, _, _ = _member(lq, (2, 2, 2, 4), 0.4, 0.3, 10, 1, lq.LQ_FP64, 3, 0)
    with pytest.raises(lq.LQError) as e:
        lq.batch_apply([m, dict(m)])                  # one context twice
    assert e.value.code == -1
    with pytest.raises(lq.LQError) as e:
        lq.batch_apply([dict(m, two_pass=1)])
    assert e.value.code == -1
    with pytest.raises(lq.LQError) as e:
        lq.batch_apply([dict(m, deflate=1)])
    assert e.value.code == -1
    out = lq.batch_apply([m])                         # the context is still usable
    assert out[0][2][0]["status"] == 0
