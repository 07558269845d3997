"""The N > 1 path of bench.py on the CPU: two ranks over gloo run the
replica logic (barrier, max-over-ranks step time, whole-job value)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    rep = bench.Replicas("gloo")
    rep.barrier()
    ms = 10.0 * (rank + 1)               # the slower rank decides
    m = rep.max(ms)
    v = rep.value(30.0, m)
    rep.barrier()
    rep.close()
    out.put((rank, rep.world, m, v))


def test_two_rank_replicas_over_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, m, v in res:
        assert w == 2
        assert m == 20.0                  # max over ranks
        assert abs(v - 2 * 30.0 / 0.020) < 1e-9   # all ranks' units / slowest time


def test_single_process_replicas():
    sys.path.insert(0, ROOT)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    import bench
    rep = bench.Replicas("gloo")
    assert rep.world == 1 and rep.dist is None
    assert rep.max(3.5) == 3.5
    assert rep.value(100, 50.0) == 2000.0
    rep.close()
