"""The N > 1 host path of bench.py on CPU: two ranks over gloo (127.0.0.1),
each an independent replica, joined only by the timing barrier and the
max-over-ranks of the timed region; rank 0 alone prints.  No GPU."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2",
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import bench
    ws, r, local = bench.dist_info()
    dist = bench.dist_init(ws)
    try:
        bench.barrier(dist)
        # each rank's own timed-region length: the job's time is the slowest rank's
        t = bench.max_over_ranks(dist, 1.5 + r)
        out.put((r, ws, local, t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_max_over_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(out.get(timeout=5) for _ in range(2))
    assert [x[0] for x in res] == [0, 1]
    assert all(x[1] == 2 and x[2] == x[0] for x in res)
    assert all(x[3] == 2.5 for x in res)


def test_reference_arm_runs_on_rank_zero_only():
    import bench

    class A:
        warmup, steps, gpus = 0, 1, 2

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A, 1, 2)
    assert buf.getvalue() == ""


def test_single_process_needs_no_process_group():
    import bench
    assert bench.dist_init(1) is None
    bench.barrier(None)
    assert bench.max_over_ranks(None, 3.25) == 3.25
