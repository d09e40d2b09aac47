"""spiir_filter_noalloc: the entry point for callers that cannot allocate
device memory (for instance while a CUDA graph is being captured, or on a
real-time thread of a host framework that forbids cudaMalloc). It must give
the same SNR as the ordinary create/push/read entry points, call after call,
even though every call reuses one fixed scratch array on the device.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
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
def test_noalloc_matches_bank_entry_points(torch_cuda, name, bank, n):
    import torch
    from paper_1702_02256_gb300 import spiir
    x = inputs.strain(1, n, seed=5)
    ref = gpu_snr(bank, x, block_len=n)[0]          # create + push + read
    xd = torch.from_numpy(x[0]).cuda()
    for call in range(2):                            # two calls in a row share the scratch
        z = spiir.filter_noalloc(bank, xd)
        torch.cuda.synchronize()
        got = z.cpu().numpy().astype(np.complex128)
        err = rel_rms(got, ref)
        assert err.max() <= TOL_PLAIN, (call, err)
        nz = np.abs(ref).max(axis=1) == 0
        assert np.all(got[nz] == 0)


def test_noalloc_rejects_banks_above_its_scratch(torch_cuda):
    import torch
    from paper_1702_02256_gb300 import spiir
    big = inputs.single_rate_bank(3000, 512, 1023, seed=0)   # about 43 MB of packed slots
    xd = torch.zeros(4096, dtype=torch.float32, device="cuda")
    with pytest.raises(spiir.SpiirError) as e:
        spiir.filter_noalloc(big, xd)
    assert e.value.status == spiir.EINVAL
    assert "scratch" in str(e.value)
