"""Seeded synthetic inputs: template banks and white Gaussian strain.

This module only draws random numbers. It holds none of the SPIIR arithmetic
(no recursion, resampling or summation), so both the CUDA path and the FP64
oracle can be fed from it without sharing any of the method's code.

Recipes (the shapes of the paper's workloads, Sec. 4 and Table 4):

* filter poles  a_k = exp(-1/tau_k + i*omega_k), tau_k log-uniform in
  [tau_lo, tau_hi] samples, omega_k uniform in (omega_lo, omega_hi);
* filter gains  b_k = (n_re + i*n_im)/sqrt(2) * (1 - |a_k|), n ~ N(0, 1);
* delays        d_k uniform integers in [0, delay_max] (samples at the
  filter's own rate);
* strain        x ~ N(0, 1) white, float32, one independent stream per
  detector (seed = strain_seed + stream index).

All coefficients are rounded to complex64 (float32 real/imag parts) here, so
that the coefficient rounding is part of the input and not of the error.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

BASE_RATE = 4096


@dataclasses.dataclass
class Bank:
    """A template bank in the layout the C ABI takes (one row per filter)."""

    n_templates: int
    n_levels: int
    a_re: np.ndarray  # float32 [n_filters]
    a_im: np.ndarray
    b_re: np.ndarray
    b_im: np.ndarray
    delay: np.ndarray  # int32 [n_filters], samples at the filter's level rate
    template_id: np.ndarray  # int32 [n_filters], non-decreasing
    level: np.ndarray  # int8 [n_filters]
    base_rate: int = BASE_RATE

    @property
    def n_filters(self) -> int:
        return int(self.a_re.shape[0])

    def subset(self, templates: Sequence[int]) -> "Bank":
        """The bank restricted to `templates`, renumbered 0..len-1 in that order."""
        templates = list(int(t) for t in templates)
        idx = []
        tid = []
        for new, t in enumerate(templates):
            sel = np.nonzero(self.template_id == t)[0]
            idx.append(sel)
            tid.append(np.full(sel.shape[0], new, np.int32))
        idx = np.concatenate(idx) if idx else np.zeros(0, np.int64)
        tid = np.concatenate(tid) if tid else np.zeros(0, np.int32)
        return Bank(
            n_templates=len(templates),
            n_levels=self.n_levels,
            a_re=self.a_re[idx].copy(),
            a_im=self.a_im[idx].copy(),
            b_re=self.b_re[idx].copy(),
            b_im=self.b_im[idx].copy(),
            delay=self.delay[idx].copy(),
            template_id=tid,
            level=self.level[idx].copy(),
            base_rate=self.base_rate,
        )


def _draw(rng: np.random.Generator, n: int, tau=(10.0, 2000.0),
          omega=(0.0, math.pi), delay_max: int = 1023):
    tau_k = np.exp(rng.uniform(math.log(tau[0]), math.log(tau[1]), n))
    om = rng.uniform(omega[0], omega[1], n)
    a = np.exp(-1.0 / tau_k + 1j * om)
    g = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2.0)
    b = g * (1.0 - np.abs(a))
    d = rng.integers(0, delay_max + 1, n).astype(np.int32)
    return (a.real.astype(np.float32), a.imag.astype(np.float32),
            b.real.astype(np.float32), b.imag.astype(np.float32), d)


def single_rate_bank(n_templates: int, filters_per_template, delay_max: int,
                     seed: int = 0, tau=(10.0, 2000.0),
                     omega=(0.0, math.pi)) -> Bank:
    """Single-rate bank: every filter at level 0 (the base rate).

    `filters_per_template` is an int (same count for all templates) or a
    sequence of per-template counts (uneven banks; zero is allowed).
    """
    rng = np.random.default_rng(seed)
    if np.isscalar(filters_per_template):
        counts = np.full(n_templates, int(filters_per_template), np.int64)
    else:
        counts = np.asarray(filters_per_template, np.int64)
        assert counts.shape == (n_templates,)
    n = int(counts.sum())
    a_re, a_im, b_re, b_im, d = _draw(rng, n, tau, omega, delay_max)
    tid = np.repeat(np.arange(n_templates, dtype=np.int32), counts)
    return Bank(n_templates, 1, a_re, a_im, b_re, b_im, d, tid,
                np.zeros(n, np.int8))


def multi_rate_bank(n_templates: int, n_levels: int = 7, seed: int = 0,
                    count_range=(2.0, 300.0), delay_max: int = 1023,
                    tau=(10.0, 2000.0), counts: Optional[np.ndarray] = None) -> Bank:
    """Multi-rate bank, filters split over `n_levels` rates by frequency.

    Per (template, level) the filter count is round(log-uniform(count_range))
    unless `counts` [n_templates, n_levels] is given. A filter at level i < H
    (H = n_levels-1) has omega in (pi/2, pi] at its own rate, i.e. it lives in
    the upper half band of that rate, which is why it cannot run at the next
    lower rate; at the lowest level omega is in (0, pi]. tau and delays are in
    own-rate samples.
    """
    rng = np.random.default_rng(seed)
    H = n_levels - 1
    if counts is None:
        lo, hi = math.log(count_range[0]), math.log(count_range[1])
        counts = np.rint(np.exp(rng.uniform(lo, hi, (n_templates, n_levels)))).astype(np.int64)
    counts = np.asarray(counts, np.int64)
    parts = []
    for t in range(n_templates):
        for lev in range(n_levels):
            c = int(counts[t, lev])
            if c == 0:
                continue
            om = (0.0, math.pi) if lev == H else (math.pi / 2, math.pi)
            a_re, a_im, b_re, b_im, d = _draw(rng, c, tau, om, delay_max)
            parts.append((a_re, a_im, b_re, b_im, d,
                          np.full(c, t, np.int32), np.full(c, lev, np.int8)))
    cat = [np.concatenate([p[i] for p in parts]) for i in range(7)]
    return Bank(n_templates, n_levels, *cat)


def strain(n_streams: int, n_samples: int, seed: int = 1) -> np.ndarray:
    """White Gaussian strain, float32 [n_streams, n_samples]."""
    out = np.empty((n_streams, n_samples), np.float32)
    for s in range(n_streams):
        out[s] = np.random.default_rng(seed + s).standard_normal(n_samples).astype(np.float32)
    return out


# ---------------------------------------------------------------------------
# The five workloads. Each returns a dict with the bank, the strain and the
# run parameters; `scale_templates` shrinks the template count for tests that
# the FP64 oracle must finish in seconds.
# ---------------------------------------------------------------------------

def workload(n: int, scale_templates: Optional[int] = None,
             n_samples: Optional[int] = None) -> dict:
    if n == 0:
        T = scale_templates or 4
        bank = single_rate_bank(T, 64, 1023, seed=0)
        ns = n_samples or 4096
        return dict(name="single-rate 4x64, 1 s", bank=bank, x=strain(1, ns),
                    block_len=4096, n_streams=1)
    if n == 1:
        T = scale_templates or 1024
        bank = single_rate_bank(T, 512, 4095, seed=0)
        ns = n_samples or 16 * 4096
        return dict(name="single-rate 1024x512, 16 s", bank=bank,
                    x=strain(1, ns), block_len=4096, n_streams=1)
    if n == 2:
        T = scale_templates or 4000
        bank = multi_rate_bank(T, 7, seed=0)
        ns = n_samples or 64 * 4096
        return dict(name="multi-rate 4000 templates, 7 rates, 64 s", bank=bank,
                    x=strain(1, ns), block_len=4096, n_streams=1)
    if n == 3:
        T = scale_templates or 8000
        bank = single_rate_bank(T, 256, 1023, seed=0)
        ns = n_samples or 8 * 4096
        return dict(name="block-parallel 8000x256, 2 streams", bank=bank,
                    x=strain(2, ns), block_len=4096, n_streams=2, chunk_len=256)
    raise ValueError(f"no workload {n}")


def serving_requests(n_requests: int, seed: int = 7, rate_hz: float = 2.0,
                     templates=(50, 20000), filters=(128, 512),
                     lifetime_blocks=(10, 60), n_levels: int = 7):
    """Poisson arrivals of template-bank requests for the serving loop.

    Returns a list of dicts: arrival time (s), n_templates, filters per
    template, lifetime in 1 s blocks, and a bank seed. Per template the filter
    total is split over the levels in proportion to log-uniform weights.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        T = int(round(math.exp(rng.uniform(math.log(templates[0]), math.log(templates[1])))))
        M = int(rng.integers(filters[0], filters[1] + 1))
        life = int(rng.integers(lifetime_blocks[0], lifetime_blocks[1] + 1))
        out.append(dict(arrival_s=t, n_templates=T, filters=M, lifetime=life,
                        seed=int(rng.integers(1 << 30)), n_levels=n_levels))
    return out


def request_bank(req: dict) -> Bank:
    """The multi-rate bank of one serving request (filters split over levels)."""
    rng = np.random.default_rng(req["seed"])
    T, M, L = req["n_templates"], req["filters"], req["n_levels"]
    w = np.exp(rng.uniform(math.log(2.0), math.log(300.0), (T, L)))
    counts = np.floor(w / w.sum(axis=1, keepdims=True) * M).astype(np.int64)
    counts[:, 0] += M - counts.sum(axis=1)
    return multi_rate_bank(T, L, seed=req["seed"] + 1, counts=counts)
