"""Pins for the FP64 oracle: each check compares it with something other than
itself (closed forms, scipy routines the method reduces to, brute force,
invariants and the paper's own tables), so that a dropped term, a wrong sign,
an off-by-one delay or a transposed operand fails at least one of them."""
import json
import math
import os

import numpy as np
import pytest
import scipy.signal as ss
import scipy.special as sp

from paper_1702_02256_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _complex(bank):
    a = bank.a_re.astype(np.float64) + 1j * bank.a_im.astype(np.float64)
    b = bank.b_re.astype(np.float64) + 1j * bank.b_im.astype(np.float64)
    return a, b


def _rel(x, ref):
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))


# --------------------------------------------------------------------------
# Kaiser taps and their building blocks (Sec. 2.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("x", [0.0, 0.5, 1.0, 3.7, 5.65326, 10.056, 20.0])
def test_bessel_i0_matches_scipy(oracle_mod, x):
    assert oracle_mod.bessel_i0(x) == pytest.approx(float(sp.i0(x)), rel=1e-14)


@pytest.mark.parametrize("atten", [10.0, 21.0, 30.0, 50.0, 60.0, 100.0])
def test_kaiser_beta_matches_scipy(oracle_mod, atten):
    assert oracle_mod.kaiser_beta(atten) == pytest.approx(ss.kaiser_beta(atten), rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("n_taps,atten", [(32, 60.0), (16, 60.0), (64, 80.0), (384, 100.0)])
def test_kaiser_taps_match_firwin(oracle_mod, n_taps, atten):
    h = oracle_mod.kaiser_taps(n_taps, atten)
    ref = ss.firwin(n_taps, 0.5, window=("kaiser", ss.kaiser_beta(atten)))
    # float32 rounding of each tap is the only allowed difference
    assert np.max(np.abs(h - ref)) <= 1.2e-7 * np.max(np.abs(ref))


def test_kaiser_taps_properties(oracle_mod):
    h = oracle_mod.kaiser_taps(32, 60.0).astype(np.float64)
    assert np.array_equal(h, h[::-1])                      # linear phase
    assert h.sum() == pytest.approx(1.0, abs=1e-6)         # unit DC gain
    # even T and symmetry: each polyphase branch sums to 1/2 exactly
    assert h[0::2].sum() == pytest.approx(0.5, abs=1e-6)
    assert h[1::2].sum() == pytest.approx(0.5, abs=1e-6)
    # stop band: Kaiser's design puts it at pi/2 + (A-8)/(2*2.285*(T-1));
    # his empirical beta/length formulas hold the attenuation to about 1.5 dB
    w, H = ss.freqz(h, worN=8192)
    edge = math.pi / 2 + (60.0 - 8.0) / (2 * 2.285 * 31)
    stop = 20 * np.log10(np.max(np.abs(H[w >= edge])))
    assert stop <= -58.5


# --------------------------------------------------------------------------
# Single-rate SPIIR (Sec. 2.1, Eqs. iireq0 / iireq1)
# --------------------------------------------------------------------------

def test_impulse_response_closed_form(oracle_mod):
    """x = delta[n - n0]  =>  z[n] = scale * sum_k b_k a_k^(n-n0-d_k), n-n0 >= d_k
    (Eq. equ:first-order2 with the delay of Eq. iireq0)."""
    bank = inputs.single_rate_bank(4, 64, 1023, seed=0)
    n, n0 = 4096, 17
    x = np.zeros(n, np.float32)
    x[n0] = 1.0
    z = oracle_mod.spiir_single(bank, x)
    a, b = _complex(bank)
    scale = 2.0 / 4096
    nn = np.arange(n)
    for t in range(bank.n_templates):
        ref = np.zeros(n, np.complex128)
        for k in np.nonzero(bank.template_id == t)[0]:
            q = nn - n0 - bank.delay[k]
            m = q >= 0
            ref[m] += b[k] * np.power(a[k], q[m].astype(np.float64))
        ref *= scale
        assert _rel(z[t], ref) < 1e-12


def test_matches_scipy_lfilter(oracle_mod):
    """Each filter is the textbook first-order IIR lfilter([b], [1, -a]) on
    the delayed input; the template's SNR is their scaled sum."""
    bank = inputs.single_rate_bank(3, 7, 50, seed=3)
    x = inputs.strain(1, 1000, seed=9)[0]
    z = oracle_mod.spiir_single(bank, x, scale=0.5)
    a, b = _complex(bank)
    for t in range(3):
        ref = np.zeros(1000, np.complex128)
        for k in np.nonzero(bank.template_id == t)[0]:
            d = int(bank.delay[k])
            xd = np.concatenate([np.zeros(d), x.astype(np.float64)])[:1000]
            ref += ss.lfilter([b[k]], [1.0, -a[k]], xd)
        assert _rel(z[t], 0.5 * ref) < 1e-12


def test_sinusoid_closed_form(oracle_mod):
    """x[n] = cos(theta n), n >= 0: the finite geometric sums give
    y_k[n] = b/2 [(e^{i th (P+1)} - a^{P+1})/(e^{i th} - a) + (e^{-i th (P+1)} - a^{P+1})/(e^{-i th} - a)],
    P = n - d_k >= 0."""
    bank = inputs.single_rate_bank(2, 16, 300, seed=5)
    n, th = 3000, 0.37
    x = np.cos(th * np.arange(n)).astype(np.float32)
    # the oracle sees float32(cos), the closed form exact cos: the bound below
    # is that input rounding (about 6e-8 relative per sample) times the gain
    z = oracle_mod.spiir_single(bank, x)
    a, b = _complex(bank)
    nn = np.arange(n)
    e1, e2 = np.exp(1j * th), np.exp(-1j * th)
    for t in range(2):
        ref = np.zeros(n, np.complex128)
        for k in np.nonzero(bank.template_id == t)[0]:
            P = nn - bank.delay[k]
            m = P >= 0
            Pm = P[m].astype(np.float64)
            ap = np.power(a[k], Pm + 1)
            ref[m] += 0.5 * b[k] * ((np.exp(1j * th * (Pm + 1)) - ap) / (e1 - a[k])
                                    + (np.exp(-1j * th * (Pm + 1)) - ap) / (e2 - a[k]))
        ref *= 2.0 / 4096
        assert _rel(z[t], ref) < 2e-6


def test_linearity_and_time_shift(oracle_mod):
    bank = inputs.single_rate_bank(3, 9, 40, seed=11)
    rng = np.random.default_rng(4)
    x1 = rng.integers(-8, 9, 700).astype(np.float32)
    x2 = rng.integers(-8, 9, 700).astype(np.float32)
    z1 = oracle_mod.spiir_single(bank, x1)
    z2 = oracle_mod.spiir_single(bank, x2)
    z12 = oracle_mod.spiir_single(bank, (2 * x1 - 3 * x2).astype(np.float32))
    assert _rel(z12, 2 * z1 - 3 * z2) < 1e-12
    s = 37
    zs = oracle_mod.spiir_single(bank, np.concatenate([np.zeros(s, np.float32), x1]))
    assert np.array_equal(zs[:, :s], np.zeros_like(zs[:, :s]))
    assert np.array_equal(zs[:, s:], z1)


def test_bruteforce_convolution(oracle_mod):
    """z = scale * (h_t * x) with the template's impulse response
    h_t[q] = sum_k 1[q >= d_k] b_k a_k^(q - d_k), direct convolution."""
    bank = inputs.single_rate_bank(3, 5, 20, seed=2, tau=(3.0, 30.0))
    x = inputs.strain(1, 600, seed=5)[0].astype(np.float64)
    z = oracle_mod.spiir_single(bank, x.astype(np.float32), scale=1.0)
    a, b = _complex(bank)
    q = np.arange(600)
    for t in range(3):
        h = np.zeros(600, np.complex128)
        for k in np.nonzero(bank.template_id == t)[0]:
            m = q >= bank.delay[k]
            h[m] += b[k] * np.power(a[k], (q[m] - bank.delay[k]).astype(np.float64))
        ref = np.convolve(h, x)[:600]
        assert _rel(z[t], ref) < 1e-11


def test_padding_filters_are_inert(oracle_mod):
    """Zero-coefficient filters (Sec. 5, Table 4 padding) do not change z."""
    bank = inputs.single_rate_bank(2, 6, 30, seed=8)
    x = inputs.strain(1, 500)[0]
    z = oracle_mod.spiir_single(bank, x)
    pad = inputs.single_rate_bank(2, 8, 30, seed=8)
    for t in range(2):
        src = np.nonzero(bank.template_id == t)[0]
        dst = np.nonzero(pad.template_id == t)[0]
        for f in ("a_re", "a_im", "b_re", "b_im", "delay"):
            getattr(pad, f)[dst[:6]] = getattr(bank, f)[src]
            getattr(pad, f)[dst[6:]] = 0
    assert np.array_equal(oracle_mod.spiir_single(pad, x), z)


def test_single_from_start_special_cases(oracle_mod):
    """State zero before `start`: start = 0 is the ordinary recursion bit for
    bit; z = 0 before start; strain that is zero before start leaves nothing
    to forget, so the result is the ordinary recursion's."""
    bank = inputs.single_rate_bank(3, [5, 1, 9], 40, seed=12)
    x = inputs.strain(1, 700, seed=3)[0]
    full = oracle_mod.spiir_single(bank, x)
    assert np.array_equal(oracle_mod.spiir_single_from(bank, x, start=0), full)
    z = oracle_mod.spiir_single_from(bank, x, start=300)
    assert np.all(z[:, :300] == 0)
    x0 = x.copy()
    x0[:300] = 0.0
    assert np.array_equal(oracle_mod.spiir_single_from(bank, x0, start=300)[:, 300:],
                          oracle_mod.spiir_single(bank, x0)[:, 300:])


def test_single_from_start_closed_form(oracle_mod):
    """One filter per template: the solution of y[n] = a y[n-1] + b x[n-d]
    splits at s into the zero-state solution from s plus the free response
    a^(n-s+1) y[s-1] of the state it had, so
    z_from[n] = z[n] - scale a^(n-s+1) y[s-1] with y[s-1] = z[s-1] / scale."""
    bank = inputs.single_rate_bank(4, 1, 25, seed=13)
    x = inputs.strain(1, 900, seed=4)[0]
    s0, scale = 333, 2.0 / bank.base_rate
    full = oracle_mod.spiir_single(bank, x)
    got = oracle_mod.spiir_single_from(bank, x, start=s0)
    a, _b = _complex(bank)
    n = np.arange(s0, 900)
    for t in range(4):
        free = scale * a[t] ** (n - s0 + 1) * (full[t, s0 - 1] / scale)
        assert _rel(got[t, s0:], full[t, s0:] - free) <= 1e-12


# --------------------------------------------------------------------------
# Multi-rate scheme (Sec. 2.2)
# --------------------------------------------------------------------------

def test_decimate_matches_lfilter(oracle_mod):
    h = oracle_mod.kaiser_taps(32, 60.0)
    x = inputs.strain(1, 1024, seed=3)[0].astype(np.float64)
    ref = ss.lfilter(h.astype(np.float64), [1.0], x)[0::2]
    assert _rel(oracle_mod.decimate(x, h), ref) < 1e-13


def test_upsample_matches_upfirdn(oracle_mod):
    h = oracle_mod.kaiser_taps(32, 60.0)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    ref = ss.upfirdn(2.0 * h.astype(np.float64), u, up=2)[:600]
    assert _rel(oracle_mod.upsample_add(u, h), ref) < 1e-13


def test_alignment_delays(oracle_mod):
    got = [oracle_mod.align_delay(i, 7, 32) for i in range(7)]
    assert got == [1953, 961, 465, 217, 93, 31, 0]
    assert all(oracle_mod.align_delay(i, 7, 32, align=False) == 0 for i in range(7))


def test_round_trip_delay_is_T_minus_1(oracle_mod):
    """Down x2 then up x2 (gain 2) of a band-limited tone returns it delayed by
    T-1 samples, within the 60 dB design's pass-band ripple."""
    h = oracle_mod.kaiser_taps(32, 60.0)
    n = 4096
    x = np.cos(0.1 * math.pi * np.arange(n) * 0.5)  # 0.05 of the input rate
    lo = oracle_mod.decimate(x, h)
    back = oracle_mod.upsample_add(lo.astype(np.complex128), h).real
    ref = np.concatenate([np.zeros(31), x])[:n]
    assert np.max(np.abs(back[200:] - ref[200:])) < 5e-3


def test_multirate_all_level0_equals_single_rate(oracle_mod):
    bank = inputs.single_rate_bank(3, 10, 100, seed=6)
    bank.n_levels = 3
    x = inputs.strain(1, 1024)[0]
    z1 = oracle_mod.spiir_single(bank, x)
    zm = oracle_mod.spiir_multirate(bank, x, align=False)
    assert np.array_equal(zm, z1)
    za = oracle_mod.spiir_multirate(bank, x, align=True)
    D = oracle_mod.align_delay(0, 3, 32)
    assert np.array_equal(za[:, D:], z1[:, :1024 - D])


def _scipy_multirate(bank, x, h, align=True, h_up=None):
    """The whole multi-rate chain from scipy routines: lfilter for the Kaiser
    decimator and each IIR filter, upfirdn for the interpolator. The level
    delay per round trip is the sum of the two linear-phase filters' group
    delays, (Td - 1)/2 + (Tu - 1)/2."""
    a, b = _complex(bank)
    H = bank.n_levels - 1
    hu = (h if h_up is None else h_up).astype(np.float64)
    R = (h.shape[0] + hu.shape[0]) // 2 - 1        # group delays; measured in the round-trip pins
    hd = h.astype(np.float64)
    xs = [x.astype(np.float64)]
    for i in range(1, bank.n_levels):
        xs.append(ss.lfilter(hd, [1.0], xs[-1])[0::2])
    out = []
    for t in range(bank.n_templates):
        u = None
        for i in range(H, -1, -1):
            Ni = xs[i].shape[0]
            s = np.zeros(Ni, np.complex128)
            for k in np.nonzero((bank.template_id == t) & (bank.level == i))[0]:
                d = int(bank.delay[k])
                xd = np.concatenate([np.zeros(d), xs[i]])[:Ni]
                s += ss.lfilter([b[k]], [1.0, -a[k]], xd)
            D = 0
            if align:
                for _ in range(H - i):
                    D = R + 2 * D
            cur = np.concatenate([np.zeros(D, np.complex128), s])[:Ni]
            if u is not None:
                cur = cur + ss.upfirdn(2.0 * hu, u, up=2)[:Ni]
            u = cur
        out.append(u * 2.0 / 4096)
    return np.array(out)


@pytest.mark.parametrize("align", [True, False])
def test_multirate_matches_scipy_chain(oracle_mod, align):
    counts = np.array([[3, 0, 2], [1, 2, 0], [0, 0, 4]])
    bank = inputs.multi_rate_bank(3, 3, seed=12, counts=counts, delay_max=40)
    x = inputs.strain(1, 2048, seed=2)[0]
    h = oracle_mod.kaiser_taps(32, 60.0)
    z = oracle_mod.spiir_multirate(bank, x, align=align)
    ref = _scipy_multirate(bank, x, h, align=align)
    assert _rel(z, ref) < 1e-11


@pytest.mark.parametrize("align", [True, False])
def test_multirate_long_decimator_matches_scipy_chain(oracle_mod, align):
    """The paper's resampler variant: a 384-tap 100 dB decimator with the
    32-tap 60 dB interpolator (Sec. 2.2)."""
    counts = np.array([[3, 1, 2], [1, 2, 0], [0, 2, 4]])
    bank = inputs.multi_rate_bank(3, 3, seed=13, counts=counts, delay_max=40)
    x = inputs.strain(1, 4096, seed=5)[0]
    hd = oracle_mod.kaiser_taps(384, 100.0)
    hu = oracle_mod.kaiser_taps(32, 60.0)
    z = oracle_mod.spiir_multirate(bank, x, h_down=hd, h_up=hu, align=align)
    ref = _scipy_multirate(bank, x, hd, align=align, h_up=hu)
    assert _rel(z, ref) < 1e-11


def test_round_trip_delay_long_decimator(oracle_mod):
    """Down through the 384-tap decimator and up through the 32-tap
    interpolator: a band-limited tone comes back delayed by the two group
    delays, (384 - 1)/2 + (32 - 1)/2 = 207 samples; the oracle's alignment for
    the next level up is the same 207."""
    hd = oracle_mod.kaiser_taps(384, 100.0)
    hu = oracle_mod.kaiser_taps(32, 60.0)
    n = 8192
    x = np.cos(0.05 * math.pi * np.arange(n))
    back = oracle_mod.upsample_add(oracle_mod.decimate(x, hd).astype(np.complex128), hu).real
    ref = np.concatenate([np.zeros(207), x])[:n]
    assert np.max(np.abs(back[600:] - ref[600:])) < 5e-3
    assert oracle_mod.align_delay(1, 3, 384, n_taps_up=32) == 207
    assert oracle_mod.align_delay(0, 3, 384, n_taps_up=32) == 207 + 2 * 207


def test_lower_rate_filter_approximates_base_rate(oracle_mod):
    """A slowly varying filter moved to level 1 (a' = a^2, b' = 2b, d' = d/2)
    reproduces its base-rate output on a band-limited input, delayed by the
    round trip T-1 that the alignment adds to level 0. Loose check of the
    scheme, not a parity pin."""
    rng = np.random.default_rng(0)
    n = 8192
    h = oracle_mod.kaiser_taps(32, 60.0)
    x = ss.lfilter(ss.firwin(129, 0.15), [1.0], rng.standard_normal(n)).astype(np.float32)
    a0 = np.exp(-1.0 / 400.0 + 1j * 0.05)
    b0 = 0.003 + 0.001j
    lev0 = inputs.Bank(1, 2, np.array([a0.real], np.float32), np.array([a0.imag], np.float32),
                       np.array([b0.real], np.float32), np.array([b0.imag], np.float32),
                       np.array([20], np.int32), np.zeros(1, np.int32), np.zeros(1, np.int8))
    a1 = complex(np.float32(a0.real), np.float32(a0.imag)) ** 2
    b1 = 2 * complex(np.float32(b0.real), np.float32(b0.imag))
    lev1 = inputs.Bank(1, 2, np.array([a1.real], np.float32), np.array([a1.imag], np.float32),
                       np.array([b1.real], np.float32), np.array([b1.imag], np.float32),
                       np.array([10], np.int32), np.zeros(1, np.int32), np.ones(1, np.int8))
    z0 = oracle_mod.spiir_multirate(lev0, x, h_down=h, h_up=h)[0]
    z1 = oracle_mod.spiir_multirate(lev1, x, h_down=h, h_up=h)[0]
    err = np.linalg.norm(z1[3000:] - z0[3000:]) / np.linalg.norm(z0[3000:])
    assert err < 0.05


# --------------------------------------------------------------------------
# Rate assignment (Sec. 2.2) against the paper's Table 4
# --------------------------------------------------------------------------

def test_assign_level_table4(oracle_mod):
    tab = json.load(open(os.path.join(GOLDEN, "tab_bank_config.json")))
    R0, L = tab["base_rate"], tab["n_levels"]
    for row in tab["rows"]:
        level = int(round(math.log2(R0 / row["rate_hz"])))
        hi = row["band_upper_hz"]
        for f in (0.51 * hi, 0.75 * hi, 0.999 * hi):
            arg = 2 * math.pi * f / R0
            got = oracle_mod.assign_level(math.cos(arg) * 0.99, math.sin(arg) * 0.99, R0, L)
            assert got == level, (f, got, level)
    # below the lowest band edge everything goes to the lowest rate
    assert oracle_mod.assign_level(0.99, 0.001, R0, L) == L - 1


def test_assign_level_margin(oracle_mod):
    """The margin knob: margin 0 is the paper's rule; a band edge at 95% of a
    rate's Nyquist frequency stays at that rate for margins below 1/0.95 - 1
    and moves one rate up above it (closed form); more margin never lowers
    the rate."""
    R0, L = 4096, 7
    rng = np.random.default_rng(3)
    for _ in range(500):
        th = rng.uniform(-math.pi, math.pi)
        ar, ai = 0.99 * math.cos(th), 0.99 * math.sin(th)
        assert oracle_mod.assign_level(ar, ai, R0, L, margin=0.0) == oracle_mod.assign_level(ar, ai, R0, L)
        levels = [oracle_mod.assign_level(ar, ai, R0, L, margin=m) for m in (0.0, 0.02, 0.1, 0.5, 1.0)]
        assert all(b <= a for a, b in zip(levels, levels[1:])), levels
    for lv in range(1, L):
        f = 0.95 * (R0 >> lv) / 2.0                 # 95% of level lv's Nyquist frequency
        arg = 2 * math.pi * f / R0
        ar, ai = 0.99 * math.cos(arg), 0.99 * math.sin(arg)
        edge = 1.0 / 0.95 - 1.0
        assert oracle_mod.assign_level(ar, ai, R0, L, margin=0.5 * edge) == lv
        assert oracle_mod.assign_level(ar, ai, R0, L, margin=1.5 * edge) == lv - 1


def test_cost_model_golden():
    """The cost model the roofline uses (12 flops per filter-sample) and the
    paper's worked example of it: half the filters at R/2 saves 25%."""
    g = json.load(open(os.path.join(GOLDEN, "cost_model.json")))
    N, M, R = 4096, 1024, 4096.0
    full = g["flops_per_filter_sample"] * N * M * R
    half = g["flops_per_filter_sample"] * N * (M / 2 * R + M / 2 * R / 2)
    assert 1 - half / full == pytest.approx(g["half_at_half_rate_saving"])
