"""Failure detection without a GPU fault.

Host side: bad arguments are refused before any launch. Device side: a push in
which one work item never publishes its progress makes the dependent item's
bounded wait give up (about 2 s); the status word reports SPIIR_ETIMEOUT, the
kernel finishes, and the bank keeps working afterwards."""
import numpy as np
import pytest

from paper_1702_02256_gb300 import inputs
from tests._util import TOL_PLAIN, rel_rms


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.gpu
def test_bounded_wait_reports_timeout_and_bank_recovers(torch_cuda, oracle_mod):
    import torch
    from paper_1702_02256_gb300 import spiir
    bank = inputs.single_rate_bank(1, 6, 50, seed=3)
    x = inputs.strain(1, 8192, seed=5)
    xd = torch.from_numpy(x).cuda()
    b = spiir.Bank(bank, n_streams=1, block_len=4096, max_push_blocks=2)
    assert b.test_stall(xd) == spiir.OK           # launched without error
    assert b.sync_status_code() == spiir.ETIMEOUT  # the wait gave up, no hang
    assert b.sync_status_code() == spiir.OK        # reported once, then cleared
    b.reset()
    b.push(xd)
    z = b.read(8192, stream_id=0).cpu().numpy()
    b.sync_status()
    b.close()
    ref = oracle_mod.spiir_single(bank, x[0])
    assert rel_rms(z, ref).max() <= TOL_PLAIN


@pytest.mark.gpu
def test_bad_pushes_are_refused_before_launch(torch_cuda):
    import torch
    from paper_1702_02256_gb300 import spiir
    bank = inputs.single_rate_bank(2, 4, 10, seed=1)
    b = spiir.Bank(bank, n_streams=2, block_len=1024, max_push_blocks=2)
    x = torch.zeros((2, 1000), device="cuda")
    with pytest.raises(spiir.SpiirError) as e:
        b.push(x)                                   # not a multiple of block_len
    assert e.value.status == spiir.EINVAL
    with pytest.raises(spiir.SpiirError) as e:
        b.push(torch.zeros((2, 3 * 1024), device="cuda"))   # above max_push_blocks
    assert e.value.status == spiir.EINVAL
    with pytest.raises(spiir.SpiirError) as e:
        b.read(1024)                                # nothing pushed yet
    assert e.value.status == spiir.ESTATE
    b.push(torch.zeros((2, 1024), device="cuda"))
    b.sync_status()
    b.close()
