"""The N > 1 replica path of bench.py on CPU: two gloo ranks, barrier, max-over-ranks timing and the
whole-job throughput (each rank runs its own replica; no data-path collective)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as td
    import bench
    td.init_process_group("gloo", rank=rank, world_size=ws)
    bench.barrier(ws)
    ms = 100.0 * (rank + 1)              # rank 1 is the slow one
    mx = bench.max_over_ranks(ws, ms, "cpu")
    out.put((rank, mx, bench.job_throughput(ws, 10, mx)))
    bench.barrier(ws)
    td.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [200.0, 200.0]
    assert res[0][2] == pytest.approx(2 * 10 / 0.2)
