"""Checkpoint and resume (spiir_state_export / spiir_state_import) and the
|z| / normalisation read (spiir_read_snr_abs), on the GPU.

A stream resumed from an exported state must continue exactly as if it had
never stopped: the same kernels see the same state, so the SNR of the pushes
after the resume is compared bit for bit with an uninterrupted run. The
|z| read is checked against the complex read and against the FP64 oracle."""
import numpy as np
import pytest

from paper_1702_02256_gb300 import inputs
from tests._util import TOL_PLAIN, rel_rms

pytestmark = pytest.mark.gpu

BLOCK = 4096


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _bank(case):
    if case == "plain-multirate":
        return inputs.multi_rate_bank(5, 4, seed=8), dict(mode="plain")
    bank = inputs.single_rate_bank(7, [3, 40, 130, 1, 64, 300, 257], 900, seed=5)
    if case == "plain-single":
        return bank, dict(mode="plain")
    if case == "fp16-fp64-carry":
        return bank, dict(mode="fp16", chunk_len=256)
    if case == "bf16x2-fp64-carry":
        return bank, dict(mode="bf16x2", chunk_len=256)
    return bank, dict(mode="fp16", chunk_len=256, carry="df")


def _pushes(b, xd, first, last):
    out = []
    for i in range(first, last):
        b.push(xd[:, i * BLOCK:(i + 1) * BLOCK].contiguous(), stream_id=-1)
        out.append(b.read(BLOCK, stream_id=-1).cpu().numpy())
    return out


@pytest.mark.parametrize("case", ["plain-single", "plain-multirate", "fp16-fp64-carry", "fp16-df-carry",
                                  "bf16x2-fp64-carry"])
def test_resume_continues_bitwise(torch_cuda, case):
    import torch
    from paper_1702_02256_gb300 import spiir
    bank, kw = _bank(case)
    S = 2
    xd = torch.from_numpy(inputs.strain(S, 4 * BLOCK, seed=33)).cuda()
    a = spiir.Bank(bank, n_streams=S, block_len=BLOCK, **kw)
    whole = _pushes(a, xd, 0, 4)
    a.close()
    b = spiir.Bank(bank, n_streams=S, block_len=BLOCK, **kw)
    _pushes(b, xd, 0, 2)
    blob = b.export_state()
    b.close()
    c = spiir.Bank(bank, n_streams=S, block_len=BLOCK, **kw)
    c.import_state(blob)
    with pytest.raises(spiir.SpiirError) as e:   # the output ring is not state
        c.read(BLOCK)
    assert e.value.status == spiir.ESTATE
    resumed = _pushes(c, xd, 2, 4)
    c.close()
    for got, want in zip(resumed, whole[2:]):
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_resume_one_stream_into_another_bank(torch_cuda):
    """The blob of stream 1 of a two-stream bank resumes as stream 0 of a
    one-stream bank (the per-stream state does not depend on the stream
    count); the plain kernels treat streams independently, so bit for bit."""
    import torch
    from paper_1702_02256_gb300 import spiir
    bank, kw = _bank("plain-multirate")
    xd = torch.from_numpy(inputs.strain(2, 3 * BLOCK, seed=34)).cuda()
    a = spiir.Bank(bank, n_streams=2, block_len=BLOCK, **kw)
    whole = _pushes(a, xd, 0, 3)
    a.close()
    b = spiir.Bank(bank, n_streams=2, block_len=BLOCK, **kw)
    _pushes(b, xd, 0, 2)
    blob = b.export_state(stream_id=1)
    b.close()
    c = spiir.Bank(bank, n_streams=1, block_len=BLOCK, **kw)
    c.import_state(blob, stream_id=0)
    c.push(xd[1:2, 2 * BLOCK:3 * BLOCK].contiguous(), stream_id=-1)
    got = c.read(BLOCK, stream_id=-1).cpu().numpy()[0]
    c.close()
    assert np.array_equal(got.view(np.uint32), whole[2][1].view(np.uint32))


def test_import_refuses_foreign_or_short_blobs(torch_cuda):
    import torch
    from paper_1702_02256_gb300 import spiir
    bank, kw = _bank("plain-single")
    xd = torch.from_numpy(inputs.strain(1, BLOCK, seed=35)).cuda()
    b = spiir.Bank(bank, n_streams=1, block_len=BLOCK, **kw)
    b.push(xd)
    blob = b.export_state()
    other = inputs.single_rate_bank(7, [3, 40, 130, 1, 64, 300, 257], 900, seed=6)
    c = spiir.Bank(other, n_streams=1, block_len=BLOCK, **kw)
    for bad in (blob[:40], blob[:-8]):
        with pytest.raises(spiir.SpiirError) as e:
            b.import_state(bad)
        assert e.value.status == spiir.EINVAL
    with pytest.raises(spiir.SpiirError) as e:      # another bank's coefficients
        c.import_state(blob)
    assert e.value.status == spiir.EINVAL
    t = spiir.Bank(bank, n_streams=1, block_len=BLOCK, mode="fp16")
    with pytest.raises(spiir.SpiirError) as e:      # another form
        t.import_state(blob)
    assert e.value.status == spiir.EINVAL
    junk = blob.copy()
    junk[:8] = 0
    with pytest.raises(spiir.SpiirError):
        b.import_state(junk)
    b.import_state(blob)                             # its own blob is fine
    for x in (b, c, t):
        x.close()


@pytest.mark.parametrize("mode", ["plain", "fp16"])
def test_read_abs_over_norm(torch_cuda, oracle_mod, mode):
    """|z| / norm_t: equal (to rounding of the modulus) to the complex read
    and, for the plain form, within its tolerance of the oracle."""
    import torch
    from paper_1702_02256_gb300 import spiir
    bank = inputs.single_rate_bank(9, [5, 64, 200, 1, 33, 128, 90, 300, 17], 700, seed=9)
    x = inputs.strain(1, 2 * BLOCK, seed=36)
    norm = np.linspace(0.5, 4.0, bank.n_templates).astype(np.float32)
    b = spiir.Bank(bank, n_streams=1, block_len=BLOCK, max_push_blocks=2, mode=mode)
    xd = torch.from_numpy(x).cuda()
    b.push(xd)
    z = b.read(2 * BLOCK).cpu().numpy()
    got = b.read_abs(2 * BLOCK, norm=torch.from_numpy(norm).cuda()).cpu().numpy()
    plain_abs = b.read_abs(BLOCK, stream_id=0).cpu().numpy()
    b.close()
    want = np.abs(z.astype(np.complex128)) / norm[None, :, None]
    assert got.shape == want.shape
    assert np.allclose(got, want, rtol=5e-7, atol=0)
    assert np.allclose(plain_abs, np.abs(z[0, :, BLOCK:].astype(np.complex128)), rtol=5e-7, atol=0)
    if mode == "plain":
        ref = np.abs(oracle_mod.spiir_single(bank, x[0])) / norm[:, None]
        assert rel_rms(got[0], ref).max() <= TOL_PLAIN
