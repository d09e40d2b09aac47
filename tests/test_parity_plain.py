"""GPU parity of the FP32 path (single-rate and multi-rate) against the FP64
oracle, through the C ABI. Tolerance: per-template RMS error / RMS SNR <= 1e-5
(the plain FP32 path's bound). Integer and layout facts are checked exactly."""
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


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_config0_all_templates(torch_cuda, oracle_mod, variant):
    w = inputs.workload(0)
    z = gpu_snr(w["bank"], w["x"], tune=-(variant + 1))[0]
    ref = oracle_mod.spiir_single(w["bank"], w["x"][0])
    err = rel_rms(z, ref)
    assert err.max() <= TOL_PLAIN, err


def test_uneven_templates_ragged_tail(torch_cuda, oracle_mod):
    """Uneven filter counts (0 .. 1100, so some templates split into parts),
    and a block length that leaves a ragged last time tile."""
    counts = [0, 1, 2, 3, 5, 17, 31, 33, 64, 129, 300, 513, 1100]
    bank = inputs.single_rate_bank(len(counts), counts, 700, seed=21)
    x = inputs.strain(1, 3 * 4100, seed=3)
    for variant in (0, 1):
        z = gpu_snr(bank, x, block_len=4100, push_blocks=2, tune=-(variant + 1))[0]
        ref = oracle_mod.spiir_single(bank, x[0])
        assert np.all(z[0] == 0)            # template without filters
        err = rel_rms(z[1:], ref[1:])
        assert err.max() <= TOL_PLAIN, err


def test_block_split_invariance_and_reset(torch_cuda):
    """Pushing 4 blocks at once equals 4 pushes of one block, bit for bit, and
    state_reset gives a fresh bank."""
    import torch
    from paper_1702_02256_gb300 import spiir
    bank = inputs.single_rate_bank(6, 100, 900, seed=5)
    x = inputs.strain(1, 4 * 1024, seed=8)
    z4 = gpu_snr(bank, x, block_len=1024, push_blocks=4)
    z1 = gpu_snr(bank, x, block_len=1024, push_blocks=1)
    assert np.array_equal(z4, z1)
    b = spiir.Bank(bank, n_streams=1, block_len=1024, max_push_blocks=4)
    xd = torch.from_numpy(x).cuda()
    b.push(xd)
    first = b.read(4096).cpu().numpy()
    b.push(xd)
    b.reset()
    b.push(xd)
    again = b.read(4096).cpu().numpy()
    b.sync_status()
    assert np.array_equal(first, again)
    assert np.array_equal(first, z4)


def test_two_streams_match_separate_banks(torch_cuda, oracle_mod):
    bank = inputs.single_rate_bank(5, 40, 300, seed=9)
    x = inputs.strain(2, 2 * 2048, seed=4)
    z = gpu_snr(bank, x, block_len=2048, n_streams=2)
    for s in range(2):
        zs = gpu_snr(bank, x[s:s + 1], block_len=2048, n_streams=1)[0]
        assert np.array_equal(z[s], zs)
        ref = oracle_mod.spiir_single(bank, x[s])
        assert rel_rms(z[s], ref).max() <= TOL_PLAIN


def test_config1_scaled_all_templates(torch_cuda, oracle_mod):
    """Config-1 filters (512 per template, delays to 4095) on 48 templates x 4 s."""
    w = inputs.workload(1, scale_templates=48, n_samples=4 * 4096)
    z = gpu_snr(w["bank"], w["x"], push_blocks=4)[0]
    ref = oracle_mod.spiir_single(w["bank"], w["x"][0])
    err = rel_rms(z, ref)
    assert err.max() <= TOL_PLAIN, err.max()


def test_config1_full_size_sampled(torch_cuda, oracle_mod):
    """The benchmark's configuration: 1024 templates x 512 filters, 16 s in one
    push of 16 blocks; 24 seeded templates checked against the oracle."""
    w = inputs.workload(1)
    z = gpu_snr(w["bank"], w["x"], push_blocks=16)[0]
    sel = np.random.default_rng(0).choice(1024, 24, replace=False)
    ref = oracle_mod.spiir_single(w["bank"], w["x"][0], templates=sel)
    err = rel_rms(z[sel], ref)
    assert err.max() <= TOL_PLAIN, err.max()
    # every template produced a finite, non-trivial series
    assert np.all(np.isfinite(z))
    assert np.all(np.abs(z).max(axis=1) > 0)


@pytest.mark.parametrize("align", [True, False])
def test_multirate_scaled(torch_cuda, oracle_mod, align):
    w = inputs.workload(2, scale_templates=12, n_samples=4 * 4096)
    z = gpu_snr(w["bank"], w["x"], push_blocks=1, align=align)[0]
    ref = oracle_mod.spiir_multirate(w["bank"], w["x"][0], align=align)
    err = rel_rms(z, ref)
    assert err.max() <= TOL_PLAIN, err


def test_multirate_custom_taps_and_empty_levels(torch_cuda, oracle_mod):
    counts = np.array([[3, 0, 2, 0], [0, 0, 0, 5], [1, 2, 3, 4], [0, 0, 0, 0]])
    bank = inputs.multi_rate_bank(4, 4, seed=2, counts=counts, delay_max=200)
    hd = oracle_mod.kaiser_taps(16, 50.0)
    hu = oracle_mod.kaiser_taps(16, 40.0)
    x = inputs.strain(1, 3 * 1024, seed=6)
    z = gpu_snr(bank, x, block_len=1024, push_blocks=1, h_down=hd, h_up=hu)[0]
    ref = oracle_mod.spiir_multirate(bank, x[0], h_down=hd, h_up=hu)
    assert np.all(z[3] == 0)
    err = rel_rms(z[:3], ref[:3])
    assert err.max() <= TOL_PLAIN, err


def test_multirate_twelve_rates(torch_cuda, oracle_mod):
    """The deepest cascade (12 rates, 4096 Hz down to 2 Hz): the combine
    works in time chunks of 8192 samples, one per push here. Without the
    alignment delays: aligned, the base rate would wait 31 * (2^11 - 1)
    samples, more than a shared-memory strain window holds."""
    bank = inputs.multi_rate_bank(6, 12, seed=4, count_range=(2.0, 60.0), delay_max=300)
    x = inputs.strain(1, 3 * 8192, seed=9)
    z = gpu_snr(bank, x, block_len=8192, push_blocks=1, align=False)[0]
    ref = oracle_mod.spiir_multirate(bank, x[0], align=False)
    err = rel_rms(z, ref)
    assert err.max() <= TOL_PLAIN, err


def test_multirate_uneven_pushes_span_chunks(torch_cuda, oracle_mod):
    """Pushes of 3 and 2 blocks of 1024: the first push spans two combine
    time chunks (2048 + 1024 samples), so the upsampler history carries both
    inside a push and across pushes."""
    bank = inputs.multi_rate_bank(10, 5, seed=8, delay_max=400)
    x = inputs.strain(1, 5 * 1024, seed=10)
    z = gpu_snr(bank, x, block_len=1024, push_blocks=3)[0]
    ref = oracle_mod.spiir_multirate(bank, x[0])
    err = rel_rms(z, ref)
    assert err.max() <= TOL_PLAIN, err


@pytest.mark.parametrize("n_taps", [6, 64])
def test_multirate_interpolator_lengths(torch_cuda, oracle_mod, n_taps):
    """Interpolators of 3 and 32 taps per polyphase branch (the generic and the
    longest unrolled combine paths)."""
    bank = inputs.multi_rate_bank(8, 4, seed=5, delay_max=300)
    h = oracle_mod.kaiser_taps(n_taps, 60.0)
    x = inputs.strain(1, 3 * 1024, seed=11)
    z = gpu_snr(bank, x, block_len=1024, push_blocks=1, h_down=h, h_up=h)[0]
    ref = oracle_mod.spiir_multirate(bank, x[0], h_down=h, h_up=h)
    err = rel_rms(z, ref)
    assert err.max() <= TOL_PLAIN, err


def test_multirate_paper_resampler(torch_cuda, oracle_mod):
    """The paper's resampler pair (Sec. 2.2): a 384-tap 100 dB Kaiser decimator
    with a 32-tap 60 dB interpolator, aligned levels, 7 rates."""
    bank = inputs.multi_rate_bank(10, 7, seed=19, delay_max=500)
    hd = oracle_mod.kaiser_taps(384, 100.0)
    hu = oracle_mod.kaiser_taps(32, 60.0)
    x = inputs.strain(1, 3 * 4096, seed=23)
    z = gpu_snr(bank, x, push_blocks=1, h_down=hd, h_up=hu)[0]
    ref = oracle_mod.spiir_multirate(bank, x[0], h_down=hd, h_up=hu)
    err = rel_rms(z, ref)
    assert err.max() <= TOL_PLAIN, err


def test_multirate_full_size_sampled(torch_cuda, oracle_mod):
    """Config 2 at full size (4000 templates, 7 rates), 4 s pushed in 1 s
    blocks; 12 seeded templates against the oracle."""
    w = inputs.workload(2, n_samples=4 * 4096)
    z = gpu_snr(w["bank"], w["x"], push_blocks=1)[0]
    sel = np.random.default_rng(1).choice(4000, 12, replace=False)
    ref = oracle_mod.spiir_multirate(w["bank"], w["x"][0], templates=sel)
    err = rel_rms(z[sel], ref)
    assert err.max() <= TOL_PLAIN, err.max()


def test_host_entry_point_matches_device_path(torch_cuda):
    from paper_1702_02256_gb300 import spiir
    bank = inputs.single_rate_bank(4, 30, 100, seed=3)
    x = inputs.strain(1, 2048, seed=2)
    zd = gpu_snr(bank, x, block_len=2048)
    b = spiir.Bank(bank, n_streams=1, block_len=2048)
    zh = b.push_host(x)
    b.close()
    assert np.array_equal(zh.astype(np.complex128), zd)


def test_kernel_timing_counts_launches(torch_cuda):
    import torch
    from paper_1702_02256_gb300 import spiir
    bank = inputs.multi_rate_bank(8, 3, seed=1)
    b = spiir.Bank(bank, n_streams=1, block_len=1024)
    b.enable_timing(True)
    xd = torch.from_numpy(inputs.strain(1, 1024)).cuda()
    for _ in range(3):
        b.push(xd)
    kt = b.kernel_times()
    assert kt["recur"][1] == 3 and kt["combine"][1] == 3 and kt["decimate"][1] == 3
    assert kt["prologue"][1] == 2 * 3        # history move + new-sample copy
    assert all(ms >= 0 for ms, _ in kt.values())
    b.close()


@pytest.mark.parametrize("form", ["plain-multirate", "fp16"])
def test_pipelined_host_push(torch_cuda, oracle_mod, form):
    """A host push of several blocks runs as pieces whose SNR is copied back
    while the next piece computes. Two streams, a 7-block host push (pieces
    of 1, 2, 2, 2 blocks), then an ordinary device push and a 3-block host
    push: the stream continues as if pushed in one piece; every sample
    against the oracle (and, for the plain form, bit for bit against device
    pushes)."""
    import torch
    from paper_1702_02256_gb300 import spiir
    blk = 1024
    if form == "fp16":
        bank = inputs.single_rate_bank(6, [40, 128, 200, 5, 300, 64], 500, seed=51)
        kw = dict(mode="fp16", chunk_len=256)
        tol = 1e-3
    else:
        bank = inputs.multi_rate_bank(5, 3, seed=52, delay_max=200)
        kw = {}
        tol = TOL_PLAIN
    x = inputs.strain(2, 11 * blk, seed=53)
    b = spiir.Bank(bank, n_streams=2, block_len=blk, max_push_blocks=7, **kw)
    z1 = b.push_host(np.ascontiguousarray(x[:, :7 * blk]))
    xd = torch.from_numpy(np.ascontiguousarray(x[:, 7 * blk:8 * blk])).cuda()
    b.push(xd, stream_id=-1)
    z2 = b.read(blk, stream_id=-1).cpu().numpy()
    z3 = b.push_host(np.ascontiguousarray(x[:, 8 * blk:]))
    got = np.concatenate([z1, z2, z3], axis=-1).astype(np.complex128)
    zr = b.read(3 * blk, stream_id=-1).cpu().numpy()
    b.sync_status()
    b.close()
    assert np.array_equal(zr, z3)                       # the ring holds the whole last push
    if form != "fp16":
        ref_dev = gpu_snr(bank, x, block_len=blk, push_blocks=1, n_streams=2, **kw)
        assert np.array_equal(got, ref_dev)
    for s in range(2):
        if bank.n_levels > 1:
            ref = oracle_mod.spiir_multirate(bank, x[s])
        else:
            ref = oracle_mod.spiir_single(bank, x[s])
        assert rel_rms(got[s], ref).max() <= tol


@pytest.mark.parametrize("form,ring_pushes", [("plain-multirate", 2), ("fp16", 2), ("fp16", 1)])
def test_async_host_pushes(torch_cuda, oracle_mod, form, ring_pushes):
    """Asynchronous host pushes of one block: with a ring of two pushes they
    alternate ring halves (a push computes while the SNR of the one before it
    is copied out), with a ring of one each waits for that copy. Six of them,
    then a device push, a synchronous host push and two more asynchronous
    ones, on two streams: every push's SNR equals, bit for bit, the same
    pushes made synchronously on a bank of its own; a read returns the last
    push; every sample against the oracle."""
    import torch
    from paper_1702_02256_gb300 import spiir
    blk = 1024
    if form == "fp16":
        bank = inputs.single_rate_bank(6, [40, 128, 200, 5, 300, 64], 500, seed=61)
        kw = dict(mode="fp16", chunk_len=256)
        tol = 1e-3
    else:
        bank = inputs.multi_rate_bank(5, 3, seed=62, delay_max=200)
        kw = {}
        tol = TOL_PLAIN
    n_blk = 10
    x = inputs.strain(2, n_blk * blk, seed=63)
    xb = [np.ascontiguousarray(x[:, i * blk:(i + 1) * blk]) for i in range(n_blk)]
    r = spiir.Bank(bank, n_streams=2, block_len=blk, max_push_blocks=ring_pushes, **kw)
    ref = [r.push_host(xi) for xi in xb]
    r.close()
    b = spiir.Bank(bank, n_streams=2, block_len=blk, max_push_blocks=ring_pushes, **kw)
    xs = [torch.from_numpy(xi).pin_memory() for xi in xb]
    zs = [torch.empty((2, bank.n_templates, blk), dtype=torch.complex64).pin_memory() for _ in range(n_blk)]
    for i in range(6):
        b.push_host_async(xs[i], zs[i])
    b.push(xs[6].cuda(), stream_id=-1)          # waits on the device for the copies
    zd = b.read(blk, stream_id=-1).cpu().numpy()
    b.push_host(xb[7], z_out=zs[7])
    b.push_host_async(xs[8], zs[8])
    b.push_host_async(xs[9], zs[9])
    last = b.read(blk, stream_id=-1).cpu().numpy()
    b.host_sync()
    b.sync_status()
    b.close()
    got = [z.numpy() for z in zs]
    got[6] = zd
    for i in range(n_blk):
        assert np.array_equal(got[i], ref[i]), i
    assert np.array_equal(last, got[9])
    full = np.concatenate(got, axis=-1).astype(np.complex128)
    for s in range(2):
        if bank.n_levels > 1:
            want = oracle_mod.spiir_multirate(bank, x[s])
        else:
            want = oracle_mod.spiir_single(bank, x[s])
        assert rel_rms(full[s], want).max() <= tol
