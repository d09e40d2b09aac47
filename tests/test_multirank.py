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


@pytest.mark.gpu
def test_replicas_behind_the_abi_match_one_bank():
    """spiir_replicas on the device list [0, 0, 0] (three template ranges on
    one GPU: independent banks, nothing waits on another) gives the SNR of
    one bank of all templates, multi-rate and two streams, over two host
    pushes: to the last bits (the packer's slot order depends on which units
    share a warp) and against the oracle; every range is non-empty and they
    tile the bank."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import numpy as np
    from paper_1702_02256_gb300 import inputs, spiir
    bank = inputs.multi_rate_bank(40, 4, seed=21, delay_max=500)
    x = inputs.strain(2, 2 * 2048, seed=22)
    one = spiir.Bank(bank, n_streams=2, block_len=2048)
    rep = spiir.Replicas(bank, [0, 0, 0], n_streams=2, block_len=2048)
    r = rep.ranges()
    assert [t0 for _, t0, _ in r] == [0, r[0][2], r[0][2] + r[1][2]] and sum(n for _, _, n in r) == 40
    assert all(n > 0 for _, _, n in r)
    from oracle import oracle
    from tests._util import TOL_PLAIN, rel_rms
    got = []
    for k in range(2):
        xk = np.ascontiguousarray(x[:, k * 2048:(k + 1) * 2048])
        zr = rep.push_host(xk).astype(np.complex128)
        assert rel_rms(zr, one.push_host(xk).astype(np.complex128)).max() <= 1e-6
        got.append(zr)
    rep.close()
    one.close()
    got = np.concatenate(got, axis=-1)
    for s in range(2):
        assert rel_rms(got[s], oracle.spiir_multirate(bank, x[s])).max() <= TOL_PLAIN
