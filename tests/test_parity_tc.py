"""GPU parity of the block-parallel tensor-core form against the FP64 oracle.

Tolerance for the FP16 panels: per-template RMS error / RMS SNR <= 1e-3. The
single-pass BF16 form rounds operands to 8 significant bits, so its error is
reported against a looser bound (see the test). The first chunk of a fresh
bank has zero carried state, so its error isolates the FIR contraction; the
later chunks add the state contractions and the FP64 carry."""
import numpy as np
import pytest

from paper_1702_02256_gb300 import inputs
from tests._util import TOL_TC, gpu_snr, rel_rms

pytestmark = pytest.mark.gpu

# Single-pass BF16 rounds both operands to 8 significant bits and misses the
# stated 1e-3 (about 2.4e-3 measured); it is held to this looser bound, and
# the test ids say so. Split BF16 (bf16x2: the FIR contraction as hi*hi +
# hi*lo + lo*hi bf16 passes) is held to 1e-3.
TOL_BF16 = 1e-2
BF16_IDS = ["fp16-1e-3", "bf16-single-pass-misses-1e-3-held-to-1e-2"]
MODES3 = [("fp16", TOL_TC), ("bf16", TOL_BF16), ("bf16x2", TOL_TC)]
MODES3_IDS = BF16_IDS + ["bf16x2-split-1e-3"]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _check(z, ref, tol, L):
    err = rel_rms(z, ref)
    first = rel_rms(z[..., :L], ref[..., :L]) if np.abs(ref[..., :L]).max() > 0 else np.zeros(1)
    assert err.max() <= tol, (f"max rel rms {err.max():.3e}; first chunk (FIR only) "
                              f"{np.max(first):.3e}")
    return float(err.max())


@pytest.mark.parametrize("mode,tol", MODES3, ids=MODES3_IDS)
def test_config3_scaled_two_streams(torch_cuda, oracle_mod, mode, tol):
    """Config-3 filters (256 per template, delays to 1023), 2 streams, 4 s pushed
    as 1 s blocks, chunk length 256."""
    w = inputs.workload(3, scale_templates=96, n_samples=4 * 4096)
    z = gpu_snr(w["bank"], w["x"], push_blocks=1, n_streams=2, mode=mode, chunk_len=256)
    for s in range(2):
        ref = oracle_mod.spiir_single(w["bank"], w["x"][s])
        _check(z[s], ref, tol, 256)


def test_split_bf16_fir_passes(torch_cuda, oracle_mod):
    """Split BF16 against single-pass BF16 on the same bank: in the first
    chunk of a fresh bank (no carried state, so the FIR contraction alone)
    the three passes leave an error near 16-bit significands, far below
    single-pass bf16; over the whole series (carry contractions single-pass)
    the error is at least 4x below single-pass bf16 and within 1e-3.
    Uneven templates (one without filters), chunk length 128, two streams."""
    counts = [0, 1, 3, 100, 128, 130, 300, 257]
    bank = inputs.single_rate_bank(len(counts), counts, 900, seed=19)
    x = inputs.strain(2, 3 * 2048, seed=13)
    kw = dict(block_len=2048, push_blocks=1, n_streams=2, chunk_len=128)
    z1 = gpu_snr(bank, x, mode="bf16", **kw)
    z2 = gpu_snr(bank, x, mode="bf16x2", **kw)
    assert np.all(z2[:, 0] == 0)
    for s in range(2):
        ref = oracle_mod.spiir_single(bank, x[s])[1:]
        e1 = rel_rms(z1[s, 1:], ref)
        e2 = rel_rms(z2[s, 1:], ref)
        live = np.abs(ref[:, :128]).max(axis=-1) > 0     # templates with output there
        f1 = rel_rms(z1[s, 1:, :128], ref[:, :128])[live]
        f2 = rel_rms(z2[s, 1:, :128], ref[:, :128])[live]
        assert live.sum() >= 3
        assert f2.max() <= 1e-4 and np.all(f2 <= f1 / 20), (f1, f2)
        assert e2.max() <= TOL_TC and e2.max() <= e1.max() / 4, (e1, e2)


def test_uneven_templates_chunk128(torch_cuda, oracle_mod):
    counts = [0, 1, 3, 100, 128, 130, 300]
    bank = inputs.single_rate_bank(len(counts), counts, 600, seed=17)
    x = inputs.strain(1, 3 * 2048, seed=12)
    z = gpu_snr(bank, x, block_len=2048, push_blocks=1, mode="fp16", chunk_len=128)[0]
    ref = oracle_mod.spiir_single(bank, x[0])
    assert np.all(z[0] == 0)
    _check(z[1:], ref[1:], TOL_TC, 128)


def test_several_batch_groups_per_push(torch_cuda, oracle_mod):
    """Two streams, pushes of 2 s: 32 chunks of 256 in 4 carry batches, so the
    filter state passes between batch groups inside one push; templates of 1,
    2 and 3 filter tiles (odd tile counts put consecutive jobs on one slot)."""
    counts = [60, 128, 200, 256, 300, 1, 383]
    bank = inputs.single_rate_bank(len(counts), counts, 700, seed=23)
    x = inputs.strain(2, 3 * 8192, seed=14)
    z = gpu_snr(bank, x, push_blocks=2, n_streams=2, mode="fp16", chunk_len=256)
    for s in range(2):
        ref = oracle_mod.spiir_single(bank, x[s])
        _check(z[s], ref, TOL_TC, 256)


def test_three_streams_pair_and_single(torch_cuda, oracle_mod):
    """Three detector streams: the carry runs them as a pair plus a single
    stream (two kernel instantiations); each stream against the oracle."""
    bank = inputs.single_rate_bank(9, [40, 128, 200, 5, 300, 64, 129, 256, 90], 500, seed=31)
    x = inputs.strain(3, 3 * 4096, seed=21)
    z = gpu_snr(bank, x, push_blocks=1, n_streams=3, mode="fp16", chunk_len=256)
    for s in range(3):
        ref = oracle_mod.spiir_single(bank, x[s])
        _check(z[s], ref, TOL_TC, 256)


@pytest.mark.parametrize("mode,tol", [("fp16", TOL_TC), ("bf16", TOL_BF16)], ids=BF16_IDS)
def test_double_float_carry_matches_fp64(torch_cuda, oracle_mod, mode, tol):
    """The double-float batch anchor (carry="df") against the default FP64
    anchor: the FP32 chunk states both hand to the contractions agree, so the
    SNR series agree far below the tolerance; and the double-float form
    against the oracle. Two streams, pushes of 3 blocks of 1024 (12 chunks:
    one full batch of 8 and a partial one, whose power a^(nb L) the kernel
    builds in the anchor's arithmetic)."""
    counts = [60, 128, 200, 256, 300, 1, 383]
    bank = inputs.single_rate_bank(len(counts), counts, 700, seed=23)
    x = inputs.strain(2, 4 * 3072, seed=14)
    kw = dict(block_len=1024, push_blocks=3, n_streams=2, mode=mode, chunk_len=256)
    z64 = gpu_snr(bank, x, **kw)
    zdf = gpu_snr(bank, x, carry="df", **kw)
    assert rel_rms(zdf, z64).max() <= 1e-6
    for s in range(2):
        _check(zdf[s], oracle_mod.spiir_single(bank, x[s]), tol, 256)


@pytest.mark.parametrize("carry", ["fp64", "df", "fp64chunk"])
def test_long_stream_does_not_drift(torch_cuda, oracle_mod, carry):
    """32 s of strain in 1 s pushes (512 chunks, 32 carry batches per
    stream) through filters with time constants up to 2000 samples: the
    state carried from batch to batch (FP64 or double-float) keeps the error
    within the tolerance to the end, and the last 4 s are no worse than
    1.5x seconds 4-8 (after the start-up transient of the first chunks,
    whose state term starts from zero)."""
    bank = inputs.single_rate_bank(12, [64, 200, 3, 128, 256, 40, 90, 300, 17, 129, 77, 1], 1023, seed=41)
    x = inputs.strain(1, 32 * 4096, seed=42)
    z = gpu_snr(bank, x, push_blocks=1, mode="fp16", chunk_len=256, carry=carry)[0]
    ref = oracle_mod.spiir_single(bank, x[0])
    _check(z, ref, TOL_TC, 256)
    w = 4 * 4096
    early = rel_rms(z[:, w:2 * w], ref[:, w:2 * w]).max()
    late = rel_rms(z[:, -w:], ref[:, -w:]).max()
    assert late <= 1.5 * early, (early, late)


def test_tc_matches_plain_path(torch_cuda):
    """Same bank through both forms: they agree to the TC tolerance."""
    bank = inputs.single_rate_bank(70, 64, 300, seed=3)
    x = inputs.strain(1, 2 * 4096, seed=4)
    zp = gpu_snr(bank, x, push_blocks=2)[0]
    zt = gpu_snr(bank, x, push_blocks=2, mode="fp16")[0]
    assert rel_rms(zt, zp).max() <= TOL_TC


def test_tc_reset_and_host_entry(torch_cuda):
    import torch
    from paper_1702_02256_gb300 import spiir
    bank = inputs.single_rate_bank(8, 40, 200, seed=6)
    x = inputs.strain(1, 4096, seed=2)
    b = spiir.Bank(bank, n_streams=1, block_len=4096, mode="fp16")
    xd = torch.from_numpy(x).cuda()
    b.push(xd)
    first = b.read(4096).cpu().numpy()
    b.push(xd)
    b.reset()
    zh = b.push_host(x)
    b.sync_status()
    b.close()
    assert np.array_equal(first, zh)


def test_fp64_every_chunk_matches_anchor_per_batch(torch_cuda, oracle_mod):
    """carry = 2 updates the filter state in FP64 at every chunk instead of
    anchoring it once per batch of chunks; the contractions see the state
    rounded to FP32 either way, so the two agree far below the tolerance, and
    both match the oracle. Two streams, partial batches (3 blocks of 1024)."""
    counts = [60, 128, 200, 256, 300, 1, 383]
    bank = inputs.single_rate_bank(len(counts), counts, 700, seed=23)
    x = inputs.strain(2, 4 * 3072, seed=14)
    kw = dict(block_len=1024, push_blocks=3, n_streams=2, mode="fp16", chunk_len=256)
    z64 = gpu_snr(bank, x, **kw)
    zch = gpu_snr(bank, x, carry="fp64chunk", **kw)
    assert rel_rms(zch, z64).max() <= 1e-5
    for s in range(2):
        _check(zch[s], oracle_mod.spiir_single(bank, x[s]), TOL_TC, 256)


def test_block_form_graph_replay_matches_direct_launches(torch_cuda):
    """Block-form pushes replay a captured CUDA graph (one per stream set,
    length, previous lengths and output offset); pushes with tracing on
    launch the kernels one by one. Both give the same SNR bit for bit, with
    three streams (a pair and a single) and pushes of 2, 1 and 2 blocks."""
    import torch
    from paper_1702_02256_gb300 import spiir
    bank = inputs.single_rate_bank(9, [40, 128, 200, 5, 300, 64, 129, 256, 90], 500, seed=33)
    x = torch.from_numpy(inputs.strain(3, 5 * 1024, seed=34)).cuda()
    out = []
    for timing in (False, True):
        b = spiir.Bank(bank, n_streams=3, block_len=1024, max_push_blocks=2, mode="fp16", chunk_len=256)
        b.enable_timing(timing)
        zs = []
        for a0, nb in ((0, 2), (2, 1), (3, 2)):
            b.push(x[:, a0 * 1024:(a0 + nb) * 1024].contiguous(), stream_id=-1)
            zs.append(b.read(nb * 1024, stream_id=-1).cpu().numpy())
        info = b.info()
        b.sync_status()
        b.close()
        assert info["graph_captured"] == (0 if timing else 1)
        out.append(np.concatenate(zs, axis=-1))
    assert np.array_equal(out[0], out[1])
