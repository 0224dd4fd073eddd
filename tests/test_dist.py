"""Multi-rank host logic on CPU: two gloo ranks (no GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_1810_06250_gb300.dist import throughput, max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [3.0, 5.0][rank]                   # rank 1 is the slow one
        v, tmax = throughput(units_per_rank=1_000_000_000, steps=10, t_ms_local=local, world=world)
        dist.barrier()
        q.put((rank, v, tmax, max_over_ranks(-float(rank))))
    finally:
        dist.destroy_process_group()


def test_throughput_uses_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, v, tmax, m in out:
        assert tmax == 5.0                           # max over ranks
        assert abs(v - 2 * 1e9 * 10 / 5e-3 / 1e9) < 1e-6   # all ranks' units / slowest time
        assert m == 0.0                              # max of (0, -1)


def test_los_ranges_partition_the_cube():
    from paper_1810_06250_gb300.dist import los_range
    for nlos in (0, 1, 7, 262144, 1000003):
        for world in (1, 2, 3, 8):
            spans = [los_range(nlos, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == nlos
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        los_range(10, 2, 2)


def test_single_process_needs_no_group():
    from paper_1810_06250_gb300.dist import throughput
    v, t = throughput(100, 2, 4.0, 1)
    assert t == 4.0 and abs(v - 100 * 2 / 4e-3 / 1e9) < 1e-15
