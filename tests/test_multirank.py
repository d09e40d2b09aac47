"""World-size-2 gloo run of the replica host logic (barrier, max over ranks,
whole-job rate) on CPU processes."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_1702_02256_gb300 import replicas
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, lr = replicas.world()
    assert (ws, r, lr) == (world, rank, rank)
    dist.barrier()
    per_rank_seconds = [0.5, 2.0][rank]
    m = replicas.max_over_ranks(per_rank_seconds, dist)
    rate = replicas.job_rate(100.0, ws, m)
    out.put((rank, m, rate, replicas.rank_seed(5, rank)))
    dist.destroy_process_group()


def test_two_rank_max_and_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[1] for x in res] == [2.0, 2.0]          # both see the slowest rank
    assert [x[2] for x in res] == [100.0, 100.0]      # 2 ranks x 100 units / 2 s
    assert res[0][3] != res[1][3]                     # distinct banks per rank
