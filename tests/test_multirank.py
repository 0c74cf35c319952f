"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, no data-path collective).
Checks the rendezvous, the barrier, max-over-ranks timing, the whole-job rate, that replicas
solve different sources, and that only rank 0 runs the CPU reference arm."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import numpy as np
    import torch.distributed as dist
    import bench
    import synthetic as syn
    got_ws, got_rank, _ = bench.dist_setup()
    assert dist.get_backend() == "gloo"
    bench.barrier(got_ws)
    ms = 10.0 * (rank + 1)                       # rank 1 is the slow one
    ms_max = bench.allmax(got_ws, ms)
    x = syn.gaussian_source((2, 2, 2, 2), bench.rank_sources(rank), nsrc=3)

    class A:
        steps, k = 1, 8
    t0 = __import__("time").perf_counter()
    if rank != 0:
        bench.run_reference(A, got_ws, rank)       # must return at once without work
    elapsed = __import__("time").perf_counter() - t0
    out[rank] = (got_ws, got_rank, ms_max, bench.whole_job_rate(3, 2, got_ws, ms_max), np.asarray(x), elapsed)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 2 and (r0[1], r1[1]) == (0, 1)
    assert r0[2] == r1[2] == 20.0                 # both ranks see the slowest rank's time
    assert r0[3] == pytest.approx(3 * 2 * 2 / 0.020)   # whole-job solves/s over both replicas
    assert not (r0[4] == r1[4]).all()             # different sources per replica
    assert r1[5] < 1.0                            # rank 1 skips the reference arm
