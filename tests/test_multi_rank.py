"""The multi-GPU form is replicas only: each rank runs its own sequence with
no data-path collective, and the benchmark takes the slowest rank's time.
This checks that aggregation with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        ms = 10.0 + 5.0 * rank  # rank 1 is the slowest replica
        dist.barrier()
        m = bench.aggregate_max_ms(ms, ws)
        q.put((rank, m, bench.whole_job_value(m, ws, 300, 20), bench.dist_env()))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v, env in res:
        assert m == 15.0
        assert abs(v - 2 * 300 * 20 / 0.015) < 1e-6
        assert env == (2, rank, 0)
