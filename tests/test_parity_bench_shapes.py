"""GPU parity at the shapes bench.py times, against the FP64 oracle.

The benchmark's numbers rest on these launch configurations, so each one is
compared here with the oracle (Eqs. iireq0 and iireq1, summed in filter
order): the full-size bank is built and pushed exactly as the bench pushes
it, and a spread sample of templates (first, last and evenly spaced ones in
between) is checked per template and stream against the oracle's SNR over
the whole series.

* single-rate 1024 x 512 filters, delays 0-4095 (F = 4096, K = 4352 for the
  block form), 16 s as one 16-block push: plain FP32 at 1e-5, the fp16 and
  split-bf16 block forms at 1e-3;
* 8000 x 256 filters, delays 0-1023, two streams, 8 s in 1 s pushes (16 carry
  batches of 8 chunks per push and stream pair): plain at 1e-5, fp16 and
  split bf16 at 1e-3;
* the multi-rate 4000-template bank with the autotuner on (tune = 1): the
  variant it keeps is one of the compiled ones, gives the same SNR bit for
  bit as that variant forced, and matches the oracle at 1e-5.
"""
import numpy as np
import pytest

from paper_1702_02256_gb300 import inputs, replicas
from tests._util import TOL_PLAIN, TOL_TC, rel_rms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _sample(T, k):
    return np.unique(np.linspace(0, T - 1, k).round().astype(np.int64))


def _run_sampled(bank, x, sel, push_blocks, n_streams, **kw):
    """Push x [S, n] in pushes of push_blocks 1 s blocks through a full-size
    bank; return the SNR of the templates `sel` as complex128 [S, len(sel), n]."""
    import torch
    from paper_1702_02256_gb300 import spiir
    S, n = x.shape
    step = 4096 * push_blocks
    b = spiir.Bank(bank, n_streams=n_streams, block_len=4096, max_push_blocks=push_blocks, **kw)
    xd = torch.from_numpy(x).cuda()
    idx = torch.from_numpy(sel).cuda()
    out = np.zeros((S, len(sel), n), np.complex128)
    zbuf = torch.empty((S, bank.n_templates, step), dtype=torch.complex64, device="cuda")
    for s0 in range(0, n, step):
        b.push(xd[:, s0:s0 + step].contiguous(), stream_id=-1)
        b.read(step, stream_id=-1, out=zbuf)
        out[:, :, s0:s0 + step] = zbuf.index_select(1, idx).cpu().numpy()
    b.sync_status()
    info = b.info()
    b.close()
    return out, info


def _config1_bank():
    # bench.py's default workload (rank 0)
    return inputs.single_rate_bank(1024, 512, 4095, seed=replicas.rank_seed(0, 0))


@pytest.mark.parametrize("form,tol", [("plain", TOL_PLAIN), ("fp16", TOL_TC), ("bf16x2", TOL_TC)])
def test_config1_bench_shape_16_block_push(torch_cuda, oracle_mod, form, tol):
    bank = _config1_bank()
    x = inputs.strain(1, 16 * 4096, seed=1)
    sel = _sample(bank.n_templates, 32)
    kw = {} if form == "plain" else dict(mode=form, chunk_len=256)
    z, info = _run_sampled(bank, x, sel, 16, 1, **kw)
    if form != "plain":
        assert info["tc_fir_len"] == 4096       # delays up to 4095: K = 4352 lags
    ref = oracle_mod.spiir_single(bank, x[0], templates=sel)
    err = rel_rms(z[0], ref)
    assert err.max() <= tol, (form, float(err.max()))


@pytest.mark.parametrize("form,tol", [("plain", TOL_PLAIN), ("fp16", TOL_TC), ("bf16x2", TOL_TC)])
def test_config3_bench_shape_8s_in_1s_pushes(torch_cuda, oracle_mod, form, tol):
    bank = inputs.single_rate_bank(8000, 256, 1023, seed=replicas.rank_seed(0, 0))
    x = inputs.strain(2, 8 * 4096, seed=1)
    sel = _sample(bank.n_templates, 24)
    kw = {} if form == "plain" else dict(mode=form, chunk_len=256)
    z, info = _run_sampled(bank, x, sel, 1, 2, **kw)
    for s in range(2):
        ref = oracle_mod.spiir_single(bank, x[s], templates=sel)
        err = rel_rms(z[s], ref)
        assert err.max() <= tol, (form, s, float(err.max()))


def test_multirate_autotuned_bank(torch_cuda, oracle_mod):
    """tune = 1 times every compiled recursion variant at bank creation and
    keeps the fastest; the bank it builds is the forced variant's bank."""
    import torch
    from paper_1702_02256_gb300 import spiir
    bank = inputs.multi_rate_bank(4000, 7, seed=replicas.rank_seed(0, 0))
    x = inputs.strain(1, 4 * 4096, seed=1)
    sel = _sample(bank.n_templates, 24)
    z, info = _run_sampled(bank, x, sel, 1, 1, tune=1)
    v = info["kernel_variant"]
    n_var = 6
    assert 0 <= v < n_var
    assert info["segment_base"] in (2048, 4096, 8192) and info["ctas_per_sm"] >= 1
    assert info["tune_ms"] > 0
    # the tuned time-segment length and CTA count change the schedule, not
    # the arithmetic: the forced variant with default segments gives the same
    # SNR bit for bit
    z_forced, info_f = _run_sampled(bank, x, sel, 1, 1, tune=-(v + 1))
    assert info_f["kernel_variant"] == v and info_f["segment_base"] == 4096
    assert np.array_equal(z, z_forced)
    ref = oracle_mod.spiir_multirate(bank, x[0], templates=sel)
    err = rel_rms(z[0], ref)
    assert err.max() <= TOL_PLAIN, float(err.max())


def test_block_form_autotuned_chunk_length(torch_cuda, oracle_mod):
    """tune = 1 on the block form picks the chunk length (128 or 256) by
    timing; the bank it keeps matches the oracle."""
    bank = inputs.single_rate_bank(300, 256, 1023, seed=replicas.rank_seed(0, 0))
    x = inputs.strain(2, 3 * 4096, seed=1)
    sel = _sample(bank.n_templates, 16)
    z, info = _run_sampled(bank, x, sel, 1, 2, mode="fp16", tune=1)
    assert info["time_tile"] in (128, 256) and info["tune_ms"] > 0
    for s in range(2):
        ref = oracle_mod.spiir_single(bank, x[s], templates=sel)
        assert rel_rms(z[s], ref).max() <= TOL_TC
