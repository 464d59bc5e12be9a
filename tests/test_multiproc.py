"""Multi-process host logic of the benchmark on CPU (gloo, world size 2, 127.0.0.1): the
rank set-up, the barrier, max-over-ranks timing and the whole-job sum, and the reference
arm that only rank 0 runs.  Every GPU run in this project has one GPU, so N > 1 is run as
independent replicas (view batches) with no data-path collective."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), BENCH_BACKEND="gloo")
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    w, r, _ = bench.dist_setup()
    bench.barrier(w)
    t_max = bench.max_over_ranks(10.0 + r, w)
    total = bench.sum_over_ranks(1.0 + r, w)
    # the reference arm prints only on rank 0; other ranks return without work
    import io
    import contextlib
    buf = io.StringIO()
    if r != 0:
        with contextlib.redirect_stdout(buf):
            bench.run_reference(None, w, r)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, w, t_max, total, buf.getvalue()))


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, w, t_max, total, printed in out:
        assert w == 2
        assert t_max == 11.0          # max over ranks
        assert total == 3.0           # whole-job sum
        if r == 1:
            assert printed == ""
