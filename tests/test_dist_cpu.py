"""The multi-GPU plumbing of bench.py on CPU: two gloo ranks agree on the
slowest rank's step time (the max over ranks), meet at the barrier, and the
whole-job throughput counts every rank's evaluations (weak scaling, no
data-path exchange)."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

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

    class A:
        impl = "reference"

    r, w, local, pg = bench.dist_setup(A(), backend="gloo")
    t = bench.dist_max(pg, 10.0 + 3.0 * r, "cpu")  # rank 1 is the slow one
    bench.barrier(pg)
    q.put((r, w, local, t, bench.weak_throughput(1000, w, t)))
    pg.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[3] == 13.0 for o in out)          # max over ranks
    assert all(abs(o[4] - 2000 / 0.013) < 1e-6 for o in out)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        impl = "curob"

    os.environ.pop("WORLD_SIZE", None)
    r, w, local, pg = bench.dist_setup(A())
    assert (w, pg) == (1, None)
    assert bench.dist_max(pg, 5.0, "cpu") == 5.0
    assert bench.weak_throughput(37 * 16384, 1, 31.8) == pytest.approx(37 * 16384 / 0.0318)
