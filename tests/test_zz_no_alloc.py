"""spiir_filter_noalloc: the entry point for callers that cannot allocate
device memory (a real-time thread of a host framework that forbids
cudaMalloc, or a process whose device memory is divided up in advance). It
runs the bank path's own plan and kernels out of one fixed scratch array, so
its SNR must equal the ordinary create/push/read entry points bit for bit,
call after call, even though every call reuses that array; and both must
match the FP64 oracle.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1702_02256_gb300 import inputs
from tests._util import TOL_PLAIN, gpu_snr, rel_rms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _cases():
    single = inputs.single_rate_bank(9, [0, 1, 5, 40, 64, 100, 333, 520, 7], 600, seed=31)
    multi = inputs.multi_rate_bank(6, 3, seed=32, delay_max=120)
    return [("single", single, 4096), ("multi", multi, 2048)]


@pytest.mark.parametrize("name,bank,n", _cases(), ids=["single", "multi"])
def test_noalloc_matches_bank_entry_points(torch_cuda, oracle_mod, name, bank, n):
    import torch
    from paper_1702_02256_gb300 import spiir
    x = inputs.strain(1, n, seed=5)
    ref = gpu_snr(bank, x, block_len=n)[0]          # create + push + read
    if bank.n_levels > 1:
        exact = oracle_mod.spiir_multirate(bank, x[0])
    else:
        exact = oracle_mod.spiir_single(bank, x[0])
    xd = torch.from_numpy(x[0]).cuda()
    for call in range(2):                            # two calls in a row share the scratch
        z = spiir.filter_noalloc(bank, xd)
        torch.cuda.synchronize()
        got = z.cpu().numpy().astype(np.complex128)
        assert np.array_equal(got, ref), call
        err = rel_rms(got, exact)
        assert err.max() <= TOL_PLAIN, (call, err)


def test_noalloc_ignores_block_fields(torch_cuda):
    """block_len and max_push_blocks of the description play no part: a C
    caller may leave them zero."""
    import torch
    from paper_1702_02256_gb300 import spiir
    bank = inputs.single_rate_bank(5, [3, 64, 0, 200, 17], 300, seed=8)
    x = torch.from_numpy(inputs.strain(1, 4096, seed=6)[0]).cuda()
    want = spiir.filter_noalloc(bank, x)
    d, _keep = spiir.make_desc(bank, n_streams=1, block_len=0, max_push_blocks=0)
    got = torch.empty_like(want)
    spiir.check(spiir.lib().spiir_filter_noalloc(ctypes.byref(d), x.data_ptr(), 4096,
                                                 got.data_ptr(), spiir._stream_handle()))
    torch.cuda.synchronize()
    assert torch.equal(got, want)


def test_noalloc_rejects_banks_above_its_scratch(torch_cuda):
    import torch
    from paper_1702_02256_gb300 import spiir
    big = inputs.single_rate_bank(3000, 512, 1023, seed=0)   # about 43 MB of packed slots
    xd = torch.zeros(4096, dtype=torch.float32, device="cuda")
    with pytest.raises(spiir.SpiirError) as e:
        spiir.filter_noalloc(big, xd)
    assert e.value.status == spiir.EINVAL
    assert "scratch" in str(e.value)
