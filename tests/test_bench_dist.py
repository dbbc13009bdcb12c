"""The multi-rank plumbing of bench.py on CPU (gloo, world size 2): the job time
is the slowest rank's, the work is summed over ranks, and the reference arm runs
on rank 0 only (the other ranks exit 0 without work).  The images are
independent units, so no collective touches the data path."""
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    r, local, w = bench.dist_env()
    dist = bench.init_dist(w)
    mx = bench.max_over_ranks(dist, [0.25, 0.75][rank])
    total = bench.sum_over_ranks(dist, float(1000 * (rank + 1)))
    bench.barrier(dist)
    out = io.StringIO()
    rc_ref = None
    if rank != 0:
        with redirect_stdout(out):
            rc_ref = bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    dist.destroy_process_group()
    q.put((r, local, w, mx, total, rc_ref, out.getvalue()))


def test_rank_aggregation_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, local, w, mx, total, rc_ref, printed) in enumerate(got):
        assert (r, local, w) == (rank, rank, 2)
        assert mx == 0.75           # slowest rank
        assert total == 3000.0      # work of both ranks
    # the reference arm on rank 1: no work, no output, exit status 0
    assert got[1][5] == 0 and got[1][6] == ""


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.init_dist(1) is None
    assert bench.max_over_ranks(None, 2.5) == 2.5
    assert bench.sum_over_ranks(None, 7.0) == 7.0
