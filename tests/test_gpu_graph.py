"""The Krylov loop replayed from a CUDA graph (lq_opts.graph): the same kernels with the same
arguments, so results are bitwise those of plain launches, on the first call (capture), on
repeated calls (replay), after a change of mu (a new configuration) and after the workspace is
reserved again (graphs dropped)."""
import time

import numpy as np
import pytest
import torch

import synthetic as syn

pytestmark = pytest.mark.gpu
DIMS = (4, 4, 2, 6)


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_is_bitwise(lqlib, prec):
    from paper_1611_00195_gb300 import lq
    k, nsrc = 60, 2
    c = lq.Context(DIMS, mu=0.3, precision=prec)
    c.upload_gauge(torch.from_numpy(syn.gauge_field(DIMS, 0.4, 3)).cuda())
    c.reserve(k, nsrc, True)
    x = torch.from_numpy(syn.gaussian_source(DIMS, 5, nsrc=nsrc)).cuda()

    def run(graph):
        ys, yd, _ = c.sign_derivative_apply(x, k, graph=graph)
        y, _ = c.sign_apply(x, k, graph=graph)
        return [t.cpu().numpy() for t in (ys, yd, y)]
    ref = run(0)
    for _ in range(2):                                    # capture, then replay
        for a, b in zip(run(-1), ref):
            assert np.array_equal(a, b)
    c.set_mu(0.2)                                         # a new configuration key
    ref2 = run(0)
    for a, b in zip(run(-1), ref2):
        assert np.array_equal(a, b)
    assert not np.array_equal(ref2[0], ref[0])
    c.reserve(k, nsrc, True)                              # graphs dropped with the workspace
    for a, b in zip(run(-1), ref2):
        assert np.array_equal(a, b)


def test_graph_saves_launch_overhead_on_small_lattice(lqlib):
    """On 4^4 the kernels are a few microseconds long and launch gaps dominate: the replayed
    loop must not be slower than plain launches (timings printed)."""
    from paper_1611_00195_gb300 import lq
    dims, k, nsrc = (4, 4, 4, 4), 200, 4
    c = lq.Context(dims, mu=0.3, precision=1)
    c.upload_gauge(torch.from_numpy(syn.gauge_field(dims, 0.4, 3)).cuda())
    c.reserve(k, nsrc, True)
    x = torch.from_numpy(syn.gaussian_source(dims, 5, nsrc=nsrc)).cuda()
    t = {}
    for graph in (0, -1, 0, -1):
        c.sign_derivative_apply(x, k, graph=graph)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            c.sign_derivative_apply(x, k, graph=graph)
        torch.cuda.synchronize()
        t[graph] = (time.perf_counter() - t0) / 3
    print("4^4, k=%d, %d sources: %.2f ms per solve batch with plain launches, %.2f ms from the graph"
          % (k, nsrc, 1e3 * t[0], 1e3 * t[-1]))
    assert t[-1] < 1.2 * t[0]
