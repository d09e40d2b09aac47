"""ctypes wrapper around the FP64 C oracle (spiir_oracle.c).

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import this module. The CUDA library never
does, and this module imports nothing from it.

Every function returns numpy arrays; complex SNR series come back as
complex128 [n_selected_templates, n_samples].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spiir_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libspiir_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile spiir_oracle.c with gcc (-O2, OpenMP) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
           "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, f, i32, i64 = (ctypes.c_double, ctypes.c_void_p, ctypes.c_int32,
                          ctypes.c_int64)
        p = ctypes.c_void_p
        _lib.spiir_oracle_bessel_i0.restype = d
        _lib.spiir_oracle_bessel_i0.argtypes = [d]
        _lib.spiir_oracle_kaiser_beta.restype = d
        _lib.spiir_oracle_kaiser_beta.argtypes = [d]
        _lib.spiir_oracle_kaiser_taps.restype = ctypes.c_int
        _lib.spiir_oracle_kaiser_taps.argtypes = [i32, d, p]
        _lib.spiir_oracle_assign_level.restype = i32
        _lib.spiir_oracle_assign_level.argtypes = [d, d, i32, i32]
        _lib.spiir_oracle_assign_level_margin.restype = i32
        _lib.spiir_oracle_assign_level_margin.argtypes = [d, d, i32, i32, d]
        _lib.spiir_oracle_align_delay.restype = i64
        _lib.spiir_oracle_align_delay.argtypes = [i32, i32, i32, i32, i32]
        _lib.spiir_oracle_single.restype = ctypes.c_int
        _lib.spiir_oracle_single.argtypes = [i32, p, p, p, p, p, p, p, i64, d,
                                             p, i32, p, i32]
        _lib.spiir_oracle_single_from.restype = ctypes.c_int
        _lib.spiir_oracle_single_from.argtypes = [i32, p, p, p, p, p, p, p, i64, d,
                                                  p, i32, p, i32, i64]
        _lib.spiir_oracle_decimate.restype = ctypes.c_int
        _lib.spiir_oracle_decimate.argtypes = [p, i64, p, i32, p]
        _lib.spiir_oracle_upsample_add.restype = ctypes.c_int
        _lib.spiir_oracle_upsample_add.argtypes = [p, i64, p, i32, p]
        _lib.spiir_oracle_multirate.restype = ctypes.c_int
        _lib.spiir_oracle_multirate.argtypes = [i32, p, p, p, p, p, p, p, i32,
                                                p, p, i32, i32, i32, p, i64, d, p,
                                                i32, p, i32]
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def bessel_i0(x: float) -> float:
    return lib().spiir_oracle_bessel_i0(float(x))


def kaiser_beta(atten_db: float) -> float:
    return lib().spiir_oracle_kaiser_beta(float(atten_db))


def kaiser_taps(n_taps: int = 32, atten_db: float = 60.0) -> np.ndarray:
    out = np.zeros(n_taps, np.float32)
    rc = lib().spiir_oracle_kaiser_taps(n_taps, atten_db, _ptr(out))
    if rc:
        raise ValueError("kaiser_taps failed")
    return out


def assign_level(a_re: float, a_im: float, base_rate: int, n_levels: int,
                 margin: float = 0.0) -> int:
    """Sec. 2.2: the smallest available rate >= 2 f (1 + margin), f the band
    edge |arg a| * base_rate / (2 pi); margin = 0 is the paper's rule."""
    if margin == 0.0:
        return int(lib().spiir_oracle_assign_level(float(a_re), float(a_im),
                                                   int(base_rate), int(n_levels)))
    return int(lib().spiir_oracle_assign_level_margin(float(a_re), float(a_im), int(base_rate),
                                                      int(n_levels), float(margin)))


def align_delay(level: int, n_levels: int, n_taps: int = 32, align: bool = True,
                n_taps_up: Optional[int] = None) -> int:
    """Alignment delay of level `level`: decimator of n_taps taps, interpolator
    of n_taps_up taps (default: the same)."""
    tu = n_taps if n_taps_up is None else n_taps_up
    return int(lib().spiir_oracle_align_delay(level, n_levels, n_taps, tu, int(align)))


def _csr(bank):
    tid = np.asarray(bank.template_id)
    if tid.size and np.any(np.diff(tid) < 0):
        raise ValueError("oracle wants filters grouped by template (sorted template_id)")
    ptr = np.zeros(bank.n_templates + 1, np.int64)
    np.add.at(ptr, tid.astype(np.int64) + 1, 1)
    return np.cumsum(ptr).astype(np.int64)


def _sel(bank, templates):
    if templates is None:
        return None, bank.n_templates
    t = np.ascontiguousarray(np.asarray(templates, np.int32))
    return t, int(t.shape[0])


def spiir_single(bank, x: np.ndarray, scale: Optional[float] = None,
                 templates: Optional[Sequence[int]] = None,
                 threads: Optional[int] = None) -> np.ndarray:
    """Single-rate SNR z[t, n] (Eqs. iireq0, iireq1) over the whole series x."""
    x = np.ascontiguousarray(x, np.float32)
    n = int(x.shape[0])
    scale = 2.0 / bank.base_rate if scale is None else float(scale)
    ptr = _csr(bank)
    tsel, n_sel = _sel(bank, templates)
    z = np.zeros((n_sel, n, 2), np.float64)
    arrs = [np.ascontiguousarray(v) for v in (bank.a_re, bank.a_im, bank.b_re,
                                              bank.b_im, bank.delay)]
    rc = lib().spiir_oracle_single(bank.n_templates, _ptr(ptr), *[_ptr(v) for v in arrs],
                                   _ptr(x), n, scale, _ptr(tsel), n_sel, _ptr(z),
                                   threads or default_threads())
    if rc:
        raise ValueError(f"spiir_oracle_single failed ({rc})")
    return z[..., 0] + 1j * z[..., 1]


def spiir_single_from(bank, x: np.ndarray, start: int, scale: Optional[float] = None,
                      templates: Optional[Sequence[int]] = None,
                      threads: Optional[int] = None) -> np.ndarray:
    """Single-rate SNR with every filter state zero before sample `start`
    (z = 0 there) and the recursion of Eq. iireq0 from `start` on, its delayed
    inputs x[n - d_k] read from the whole series x (a bank that joins a
    running stream)."""
    x = np.ascontiguousarray(x, np.float32)
    n = int(x.shape[0])
    scale = 2.0 / bank.base_rate if scale is None else float(scale)
    ptr = _csr(bank)
    tsel, n_sel = _sel(bank, templates)
    z = np.zeros((n_sel, n, 2), np.float64)
    arrs = [np.ascontiguousarray(v) for v in (bank.a_re, bank.a_im, bank.b_re,
                                              bank.b_im, bank.delay)]
    rc = lib().spiir_oracle_single_from(bank.n_templates, _ptr(ptr), *[_ptr(v) for v in arrs],
                                        _ptr(x), n, scale, _ptr(tsel), n_sel, _ptr(z),
                                        threads or default_threads(), int(start))
    if rc:
        raise ValueError(f"spiir_oracle_single_from failed ({rc})")
    return z[..., 0] + 1j * z[..., 1]


def decimate(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    h = np.ascontiguousarray(h, np.float32)
    out = np.zeros(x.shape[0] // 2, np.float64)
    lib().spiir_oracle_decimate(_ptr(x), x.shape[0], _ptr(h), h.shape[0], _ptr(out))
    return out


def upsample_add(u: np.ndarray, h: np.ndarray, acc: Optional[np.ndarray] = None) -> np.ndarray:
    u = np.ascontiguousarray(np.stack([u.real, u.imag], -1), np.float64)
    h = np.ascontiguousarray(h, np.float32)
    n_low = u.shape[0]
    out = np.zeros((2 * n_low, 2), np.float64)
    if acc is not None:
        out[:, 0] = acc.real
        out[:, 1] = acc.imag
    lib().spiir_oracle_upsample_add(_ptr(u), n_low, _ptr(h), h.shape[0], _ptr(out))
    return out[:, 0] + 1j * out[:, 1]


def spiir_multirate(bank, x: np.ndarray, h_down: Optional[np.ndarray] = None,
                    h_up: Optional[np.ndarray] = None, n_taps: int = 32,
                    align: bool = True, scale: Optional[float] = None,
                    templates: Optional[Sequence[int]] = None,
                    threads: Optional[int] = None) -> np.ndarray:
    """Multi-rate SNR z[t, n] at the base rate (Sec. 2.2)."""
    x = np.ascontiguousarray(x, np.float32)
    n = int(x.shape[0])
    if h_down is None:
        h_down = kaiser_taps(n_taps, 60.0)
    if h_up is None:
        h_up = kaiser_taps(n_taps, 60.0)
    h_down = np.ascontiguousarray(h_down, np.float32)
    h_up = np.ascontiguousarray(h_up, np.float32)
    scale = 2.0 / bank.base_rate if scale is None else float(scale)
    ptr = _csr(bank)
    tsel, n_sel = _sel(bank, templates)
    z = np.zeros((n_sel, n, 2), np.float64)
    arrs = [np.ascontiguousarray(v) for v in (bank.a_re, bank.a_im, bank.b_re,
                                              bank.b_im, bank.delay)]
    lev = np.ascontiguousarray(bank.level, np.int8)
    rc = lib().spiir_oracle_multirate(bank.n_templates, _ptr(ptr), *[_ptr(v) for v in arrs],
                                      _ptr(lev), bank.n_levels, _ptr(h_down), _ptr(h_up),
                                      int(h_down.shape[0]), int(h_up.shape[0]),
                                      int(bool(align)), _ptr(x), n,
                                      scale, _ptr(tsel), n_sel, _ptr(z),
                                      threads or default_threads())
    if rc:
        raise ValueError(f"spiir_oracle_multirate failed ({rc})")
    return z[..., 0] + 1j * z[..., 1]
