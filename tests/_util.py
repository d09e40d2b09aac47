"""Shared helpers for the test suite (comparison metrics, GPU runs)."""
import numpy as np

# Tolerances (stated per template as RMS error over RMS of the oracle SNR):
# the plain FP32 path must stay within 1e-5, the tensor-core forms within 1e-3.
TOL_PLAIN = 1e-5
TOL_TC = 1e-3


def rel_rms(z, ref):
    """Per-template ||z - ref||_rms / ||ref||_rms (templates with zero
    reference SNR use the absolute RMS)."""
    z = np.asarray(z)
    ref = np.asarray(ref)
    num = np.sqrt(np.mean(np.abs(z - ref) ** 2, axis=-1))
    den = np.sqrt(np.mean(np.abs(ref) ** 2, axis=-1))
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def gpu_snr(bank, x, block_len=4096, push_blocks=None, n_streams=1, **kw):
    """Run the CUDA path: push x [n_streams, n] in pushes of push_blocks blocks,
    return complex128 [n_streams, T, n]."""
    import torch
    from paper_1702_02256_gb300 import spiir
    x = np.atleast_2d(np.asarray(x, np.float32))
    n = x.shape[1]
    assert n % block_len == 0
    nb = n // block_len
    push_blocks = push_blocks or nb
    b = spiir.Bank(bank, n_streams=n_streams, block_len=block_len,
                   max_push_blocks=push_blocks, **kw)
    xd = torch.from_numpy(x).cuda()
    out = np.zeros((n_streams, bank.n_templates, n), np.complex128)
    step = push_blocks * block_len
    for s0 in range(0, n, step):
        m = min(step, n - s0)
        b.push(xd[:, s0:s0 + m].contiguous(), stream_id=-1)
        z = b.read(m, stream_id=-1)
        out[:, :, s0:s0 + m] = z.cpu().numpy()
    b.sync_status()
    b.close()
    return out
