"""Multi-process (N > 1) host logic of bench.py on CPU: two gloo ranks.

On several GPUs every rank simulates its own replica (the path has no data
exchange); the JSON line's value is the units of all ranks over the slowest
rank's time, and only rank 0 runs the reference arm.  These checks run that
host logic as two processes with the gloo backend, no GPU involved.
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q) -> None:
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    try:
        import bench
        d = bench.Dist("gloo")
        d.barrier()
        # rank r: (r + 1) * 1000 units in 0.5 + r seconds
        value, t_max = bench.job_throughput(d, 1000.0 * (rank + 1), 0.5 + rank)
        total = d.reduce(float(rank + 1), "sum")
        slowest = d.reduce(float(rank), "max")
        ref_skipped = None
        if rank != 0:
            # the reference arm runs on rank 0 only; other ranks return at once
            bench.run_reference(None, d)
            ref_skipped = True
        d.barrier()
        d.close()
        q.put((rank, value, t_max, total, slowest, ref_skipped, None))
    except Exception as e:  # reported to the parent
        q.put((rank, None, None, None, None, None, repr(e)))


def test_two_gloo_ranks_aggregate_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(2):
            rank, *rest = q.get(timeout=120)
            out[rank] = rest
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    assert set(out) == {0, 1}
    for rank, (value, t_max, total, slowest, ref_skipped, err) in out.items():
        assert err is None, err
        assert t_max == pytest.approx(1.5)
        assert value == pytest.approx(3000.0 / 1.5)
        assert total == pytest.approx(3.0)
        assert slowest == pytest.approx(1.0)
    assert out[1][4] is True
    assert all(p.exitcode == 0 for p in procs)
