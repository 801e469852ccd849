"""Multi-rank host logic of bench.py on CPU: two gloo ranks (world_size 2).

Each rank runs an independent mock (its own seed); the whole-job figure is
the sum of units over ranks divided by the slowest rank's time.  Only rank 0
runs the CPU reference arm.
"""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, loc = bench.dist_setup()
    assert dist.get_backend() == "gloo"
    ms, total, value = bench.aggregate(10.0 + 5.0 * r, 100.0 * (r + 1), w)
    bench.barrier(w)

    class A:
        warmup, steps, gpus = 0, 1, w
    printed = None
    if r != 0:
        import io
        import contextlib
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.run_reference(A, r, w)  # must return at once without output
        printed = buf.getvalue()
    q.put((r, w, ms, total, value, bench.rank_seed(r), printed))
    dist.destroy_process_group()


def test_two_rank_aggregate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, ms, total, value, seed, printed in res:
        assert w == 2
        assert ms == 15.0                 # max over ranks
        assert total == 300.0             # sum over ranks
        assert np.isclose(value, 300.0 / 0.015)
    assert res[0][5] != res[1][5]         # independent mocks
    assert res[1][6] == ""                # rank 1 runs no reference work


def test_rank_mocks_differ():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2507_00129_gb300 import synth
    a = synth.spec_for(1, seed=bench.rank_seed(0))
    b = synth.spec_for(1, seed=bench.rank_seed(1))
    a.n_forests = b.n_forests = 50
    ca, cb = synth.generate(a), synth.generate(b)
    assert not np.array_equal(ca.ra, cb.ra)
    assert ca.n_forests == cb.n_forests
