"""The multi-GPU path of bench.py on CPU: two gloo ranks.

With N GPUs the renderer runs N replicas: each rank renders its own
iteration range (no collective on the data path), the timed region is
bracketed by barriers, and the whole-job time is the slowest rank's. These
are the host-side pieces; they run here on two CPU processes.
"""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", init_method="env://")
    try:
        env = bench.dist_env()
        local_ms = [30.0, 45.0, 12.5][rank]
        dist.barrier()
        total = bench.job_ms(local_ms, dist, "cpu")
        value = bench.job_value(1000, ws, total)
        q.put((rank, env, bench.rank_iter_base(rank), total, value))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_replicas_take_the_slowest_rank_and_disjoint_iterations(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    slowest = max([30.0, 45.0, 12.5][:ws])
    for rank, env, base, total, value in res:
        assert env == (ws, rank, rank)
        assert total == slowest
        assert abs(value - 1000 * ws / (slowest * 1e-3) / 1e6) < 1e-12
    # each rank's iteration range (here up to 2^20 iterations) is disjoint from the others'
    bases = sorted(r[2] for r in res)
    assert len(set(bases)) == ws
    assert all(b2 - b1 >= (1 << 20) for b1, b2 in zip(bases, bases[1:]))


def test_single_rank_needs_no_collective():
    import bench
    assert bench.job_ms(17.0) == 17.0
    assert bench.rank_iter_base(0) == 0
