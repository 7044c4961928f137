"""Multi-GPU mode is replicas only: two gloo ranks on the CPU check the cell
partition (disjoint, complete) and the benchmark's timing reduction (max of
times, sum of bits)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_1905_01141_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cells = replicas.cell_block(41, world, rank)
    seconds = 0.5 + rank          # the slower rank decides the time
    bits = 1000 * (rank + 1)
    t, b = replicas.reduce_time_bits(seconds, bits)
    out.put((rank, cells, t, b, replicas.rank_seed(1, rank)))
    dist.destroy_process_group()


def test_two_gloo_replicas():
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cells = res[0][1] + res[1][1]
    assert sorted(cells) == list(range(41)) and not set(res[0][1]) & set(res[1][1])
    assert all(r[2] == 1.5 and r[3] == 3000.0 for r in res)
    assert res[0][4] != res[1][4]
