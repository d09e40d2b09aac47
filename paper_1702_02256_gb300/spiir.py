"""Thin ctypes binding of libspiir (include/spiir.h).

Argument marshalling only: every step of the filtering runs in the library's
CUDA kernels. PyTorch supplies device memory (tensors) and the CUDA stream.
If the shared library is missing the import fails loudly; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libspiir.so")

OK, EINVAL, ENOMEM, EBUDGET, ECUDA, ETIMEOUT, ESTATE, EUNSUPPORTED = range(8)
PLAIN_FP32, TC_FP16, TC_BF16, TC_BF16X2 = range(4)
MODES = {"plain": PLAIN_FP32, "fp16": TC_FP16, "bf16": TC_BF16, "bf16x2": TC_BF16X2}
CARRY = {"fp64": 0, "df": 1, "fp64chunk": 2}   # tensor-core forms: carried-state arithmetic

_c_void_p = ctypes.c_void_p
_i32, _i64, _f32, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double


class BankDesc(ctypes.Structure):
    _fields_ = [
        ("n_templates", _i32), ("n_levels", _i32), ("base_rate", _i32),
        ("n_streams", _i32), ("block_len", _i32), ("max_push_blocks", _i32),
        ("n_filters", _i64),
        ("a_re", _c_void_p), ("a_im", _c_void_p), ("b_re", _c_void_p), ("b_im", _c_void_p),
        ("delay", _c_void_p), ("template_id", _c_void_p), ("level", _c_void_p),
        ("h_down", _c_void_p), ("h_up", _c_void_p),
        ("n_taps", _i32), ("align", _i32), ("snr_scale", _f32), ("mode", _i32),
        ("chunk_len", _i32), ("tune", _i32), ("hbm_budget_bytes", _i64), ("n_taps_up", _i32),
        ("carry", _i32),
    ]


class BankInfo(ctypes.Structure):
    _fields_ = [
        ("footprint_bytes", _i64), ("n_slots", _i64), ("filter_samples_per_block", _i64),
        ("n_warp_tasks", _i32), ("n_cta_items", _i32), ("filters_per_lane", _i32),
        ("time_tile", _i32), ("kernel_variant", _i32), ("max_delay", _i32),
        ("tc_fir_len", _i32), ("graph_captured", _i32), ("n_units", _i32),
        ("smem_ways", _f32), ("slot_fill", _f32), ("segment_base", _i32), ("ctas_per_sm", _i32),
        ("tune_ms", _f32),
    ]


class ServerDesc(ctypes.Structure):
    _fields_ = [
        ("n_streams", _i32), ("n_levels", _i32), ("base_rate", _i32), ("block_len", _i32),
        ("max_delay", _i32), ("h_down", _c_void_p), ("h_up", _c_void_p),
        ("n_taps", _i32), ("n_taps_up", _i32), ("align", _i32), ("snr_scale", _f32),
        ("mode", _i32), ("chunk_len", _i32), ("carry", _i32), ("tune", _i32),
        ("tc_min_filters", _i32),
    ]


class ServerInfo(ctypes.Structure):
    _fields_ = [
        ("n_members", _i32), ("n_templates", _i32), ("n_filters", _i64),
        ("filter_samples_per_push", _i64), ("device_bytes", _i64), ("n_cta_items", _i32),
        ("kernel_variant", _i32), ("tc_levels", _i32), ("launches_per_push", _i32),
    ]


K_PROLOGUE, K_DECIMATE, K_RECUR, K_COMBINE, K_TC_STAGE, K_TC_FIR, K_TC_CARRY, K_OTHER = range(8)
KERNEL_NAMES = ["prologue", "decimate", "recur", "combine", "tc_stage", "tc_fir", "tc_carry", "other"]


class KernelTimes(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_int64 * 8)]


class SpiirError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"spiir status {status}: {msg}")
        self.status = status


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "spiir_bank_create": (_i32, [ctypes.POINTER(BankDesc), _c_void_p, ctypes.POINTER(_c_void_p)]),
    "spiir_push_block": (_i32, [_c_void_p, _i32, _c_void_p, _i64, _c_void_p]),
    "spiir_read_snr": (_i32, [_c_void_p, _i32, _c_void_p, _i64, _c_void_p]),
    "spiir_state_reset": (_i32, [_c_void_p, _i32, _c_void_p]),
    "spiir_read_snr_abs": (_i32, [_c_void_p, _i32, _c_void_p, _i64, _c_void_p, _c_void_p]),
    "spiir_state_bytes": (_i64, [_c_void_p, _i32]),
    "spiir_state_export": (_i32, [_c_void_p, _i32, _c_void_p, _i64, _c_void_p]),
    "spiir_state_import": (_i32, [_c_void_p, _i32, _c_void_p, _i64, _c_void_p]),
    "spiir_push_block_host": (_i32, [_c_void_p, _i32, _c_void_p, _i64, _c_void_p, _c_void_p]),
    "spiir_push_block_host_async": (_i32, [_c_void_p, _i32, _c_void_p, _i64, _c_void_p, _c_void_p]),
    "spiir_bank_host_sync": (_i32, [_c_void_p]),
    "spiir_bank_footprint": (_i64, [ctypes.POINTER(BankDesc)]),
    "spiir_bank_get_info": (_i32, [_c_void_p, ctypes.POINTER(BankInfo)]),
    "spiir_bank_plan": (_i32, [ctypes.POINTER(BankDesc), ctypes.POINTER(BankInfo)]),
    "spiir_bank_sync_status": (_i32, [_c_void_p]),
    "spiir_bank_destroy": (None, [_c_void_p]),
    "spiir_kaiser_taps": (_i32, [_i32, _f64, _c_void_p]),
    "spiir_assign_level": (_i32, [_f32, _f32, _i32, _i32]),
    "spiir_assign_level_margin": (_i32, [_f32, _f32, _i32, _i32, _f32]),
    "spiir_last_error": (ctypes.c_char_p, []),
    "spiir_filter_noalloc": (_i32, [ctypes.POINTER(BankDesc), _c_void_p, _i64, _c_void_p, _c_void_p]),
    "spiir_bank_enable_timing": (_i32, [_c_void_p, _i32]),
    "spiir_bank_test_stall": (_i32, [_c_void_p, _c_void_p, _i64, _c_void_p]),
    "spiir_bank_kernel_times": (_i32, [_c_void_p, ctypes.POINTER(KernelTimes)]),
    "spiir_server_create": (_i32, [ctypes.POINTER(ServerDesc), _c_void_p, ctypes.POINTER(_c_void_p)]),
    "spiir_server_add": (_i32, [_c_void_p, ctypes.POINTER(BankDesc), ctypes.POINTER(_i32)]),
    "spiir_server_remove": (_i32, [_c_void_p, _i32]),
    "spiir_server_member_footprint": (_i64, [_c_void_p, ctypes.POINTER(BankDesc)]),
    "spiir_server_push": (_i32, [_c_void_p, _c_void_p, _c_void_p]),
    "spiir_server_prepare": (_i32, [_c_void_p, _c_void_p]),
    "spiir_server_enable_timing": (_i32, [_c_void_p, _i32]),
    "spiir_server_kernel_times": (_i32, [_c_void_p, ctypes.POINTER(KernelTimes)]),
    "spiir_server_read": (_i32, [_c_void_p, _i32, _c_void_p, _c_void_p]),
    "spiir_server_get_info": (_i32, [_c_void_p, ctypes.POINTER(ServerInfo)]),
    "spiir_server_sync_status": (_i32, [_c_void_p]),
    "spiir_server_destroy": (None, [_c_void_p]),
    "spiir_replicas_create": (_i32, [ctypes.POINTER(BankDesc), _c_void_p, _i32, ctypes.POINTER(_c_void_p)]),
    "spiir_replicas_push_host": (_i32, [_c_void_p, _c_void_p, _i64, _c_void_p]),
    "spiir_replicas_get": (_i32, [_c_void_p, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                  ctypes.POINTER(_i32)]),
    "spiir_replicas_destroy": (None, [_c_void_p]),
}


def lib():
    """Load libspiir.so (built by __graft_entry__.build()); fail loudly if absent.
    SPIIR_LIB, if set, names another build of it (a reduction ablation)."""
    global _lib
    if _lib is None:
        path = os.environ.get("SPIIR_LIB", LIB_PATH)
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().spiir_last_error().decode()


def check(status: int):
    if status != OK:
        raise SpiirError(status, last_error())


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def kaiser_taps(n_taps: int = 32, atten_db: float = 60.0) -> np.ndarray:
    out = np.zeros(n_taps, np.float32)
    check(lib().spiir_kaiser_taps(n_taps, atten_db, out.ctypes.data))
    return out


def assign_level(a_re: float, a_im: float, base_rate: int, n_levels: int, margin: float = 0.0) -> int:
    if margin == 0.0:
        return int(lib().spiir_assign_level(a_re, a_im, base_rate, n_levels))
    return int(lib().spiir_assign_level_margin(a_re, a_im, base_rate, n_levels, margin))


def make_desc(bank, n_streams: int = 1, block_len: int = 4096, max_push_blocks: int = 1,
              mode: str = "plain", chunk_len: int = 0, tune: int = 0,
              hbm_budget_bytes: int = 0, align: Optional[bool] = None,
              h_down: Optional[np.ndarray] = None, h_up: Optional[np.ndarray] = None,
              snr_scale: float = 0.0, carry="fp64"):
    """Fill a BankDesc from an inputs.Bank. Returns (desc, keepalive arrays)."""
    keep = dict(
        a_re=_arr(bank.a_re, np.float32), a_im=_arr(bank.a_im, np.float32),
        b_re=_arr(bank.b_re, np.float32), b_im=_arr(bank.b_im, np.float32),
        delay=_arr(bank.delay, np.int32), template_id=_arr(bank.template_id, np.int32),
        level=_arr(bank.level, np.int8),
    )
    d = BankDesc()
    d.n_templates = bank.n_templates
    d.n_levels = bank.n_levels
    d.base_rate = bank.base_rate
    d.n_streams = n_streams
    d.block_len = block_len
    d.max_push_blocks = max_push_blocks
    d.n_filters = bank.n_filters
    for k, v in keep.items():
        setattr(d, k, v.ctypes.data if v.size else None)
    if h_down is not None:
        keep["h_down"] = _arr(h_down, np.float32)
        keep["h_up"] = _arr(h_up, np.float32)
        d.h_down = keep["h_down"].ctypes.data
        d.h_up = keep["h_up"].ctypes.data
        d.n_taps = int(keep["h_down"].shape[0])
        d.n_taps_up = int(keep["h_up"].shape[0])
    d.align = int(bank.n_levels > 1 if align is None else align)
    d.snr_scale = snr_scale
    d.mode = MODES[mode] if isinstance(mode, str) else int(mode)
    d.chunk_len = chunk_len
    d.tune = tune
    d.hbm_budget_bytes = hbm_budget_bytes
    d.carry = CARRY[carry] if isinstance(carry, str) else int(carry)
    return d, keep


def footprint(bank, **kw) -> int:
    d, _keep = make_desc(bank, **kw)
    return int(lib().spiir_bank_footprint(ctypes.byref(d)))


def plan(bank, **kw) -> dict:
    """Host-only packing facts for a bank description (no GPU needed)."""
    d, _keep = make_desc(bank, **kw)
    inf = BankInfo()
    check(lib().spiir_bank_plan(ctypes.byref(d), ctypes.byref(inf)))
    return {k: getattr(inf, k) for k, _ in BankInfo._fields_}


def filter_noalloc(bank, x, z_out=None, stream=None, **kw):
    """spiir_filter_noalloc: one-shot filtering of a CUDA tensor x [n] from
    zero state into z_out (complex64 [T, n]) without any device allocation by
    the library. Returns z_out."""
    import torch
    n = int(x.shape[-1])
    if z_out is None:
        z_out = torch.empty((bank.n_templates, n), dtype=torch.complex64, device=x.device)
    d, _keep = make_desc(bank, n_streams=1, block_len=n, max_push_blocks=1, **kw)
    check(lib().spiir_filter_noalloc(ctypes.byref(d), x.data_ptr(), n, z_out.data_ptr(),
                                     _stream_handle(stream)))
    return z_out


def _stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Bank:
    """A device-resident SPIIR bank (spiir_bank_t)."""

    def __init__(self, bank, n_streams: int = 1, block_len: int = 4096,
                 max_push_blocks: int = 1, stream=None, **kw):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libspiir needs a CUDA device")
        d, keep = make_desc(bank, n_streams=n_streams, block_len=block_len,
                            max_push_blocks=max_push_blocks, **kw)
        h = _c_void_p()
        check(lib().spiir_bank_create(ctypes.byref(d), _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self.n_templates = bank.n_templates
        self.n_streams = n_streams
        self.block_len = block_len
        self.max_push_blocks = max_push_blocks

    @property
    def handle(self):
        return self._h

    def push(self, x, stream_id: int = -1, stream=None):
        """x: float32 CUDA tensor [n] (one stream) or [n_streams, n] (stream_id=-1)."""
        assert x.is_cuda and x.dtype.is_floating_point and x.is_contiguous()
        n = int(x.shape[-1])
        check(lib().spiir_push_block(self._h, stream_id, x.data_ptr(), n, _stream_handle(stream)))

    def read(self, n_samples: int, stream_id: int = -1, out=None, stream=None):
        """SNR of the last push: complex64 [n_streams, T, n] (or [T, n])."""
        import torch
        shape = ((self.n_streams if stream_id < 0 else 1), self.n_templates, n_samples)
        if out is None:
            out = torch.empty(shape, dtype=torch.complex64, device="cuda")
        check(lib().spiir_read_snr(self._h, stream_id, out.data_ptr(), n_samples,
                                   _stream_handle(stream)))
        return out if stream_id < 0 else out[0]

    def push_host(self, x, stream_id: int = -1, z_out=None, stream=None):
        """Host buffers in and out (copies inside the call). x and z_out are
        numpy arrays or (pinned) CPU torch tensors."""
        if hasattr(x, "data_ptr"):
            n = int(x.shape[-1])
            xp = x.data_ptr()
        else:
            x = np.ascontiguousarray(x, np.float32)
            n = int(x.shape[-1])
            xp = x.ctypes.data
        cnt = self.n_streams if stream_id < 0 else 1
        if z_out is None:
            z_out = np.empty((cnt, self.n_templates, n), np.complex64)
        zp = z_out.data_ptr() if hasattr(z_out, "data_ptr") else z_out.ctypes.data
        check(lib().spiir_push_block_host(self._h, stream_id, xp, n, zp, _stream_handle(stream)))
        return z_out

    def push_host_async(self, x, z_out, stream_id: int = -1, stream=None):
        """As push_host, returning once the work is queued; z_out holds the
        SNR (and x may change) after host_sync(). x and z_out: pinned CPU
        torch tensors, kept alive by the caller until then."""
        n = int(x.shape[-1])
        check(lib().spiir_push_block_host_async(self._h, stream_id, x.data_ptr(), n, z_out.data_ptr(),
                                                _stream_handle(stream)))
        return z_out

    def host_sync(self):
        """Wait until every asynchronous host push has its SNR in host memory."""
        check(lib().spiir_bank_host_sync(self._h))

    def reset(self, stream_id: int = -1, stream=None):
        check(lib().spiir_state_reset(self._h, stream_id, _stream_handle(stream)))

    def read_abs(self, n_samples: int, norm=None, stream_id: int = -1, out=None, stream=None):
        """|z| / norm[t] of the last push: float32 CUDA tensor [n_streams, T, n]
        (or [T, n]). norm: float32 CUDA tensor [T] or None."""
        import torch
        shape = ((self.n_streams if stream_id < 0 else 1), self.n_templates, n_samples)
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device="cuda")
        check(lib().spiir_read_snr_abs(self._h, stream_id, out.data_ptr(), n_samples,
                                       None if norm is None else norm.data_ptr(),
                                       _stream_handle(stream)))
        return out if stream_id < 0 else out[0]

    def export_state(self, stream_id: int = -1, stream=None) -> np.ndarray:
        """Checkpoint: the state blob of one stream (or all) as uint8 host bytes."""
        n = int(lib().spiir_state_bytes(self._h, stream_id))
        if n < 0:
            raise SpiirError(EINVAL, "bad stream_id")
        buf = np.empty(n, np.uint8)
        check(lib().spiir_state_export(self._h, stream_id, buf.ctypes.data, n, _stream_handle(stream)))
        return buf

    def import_state(self, blob, stream_id: int = -1, stream=None):
        """Resume from a blob written by export_state (same description)."""
        blob = np.ascontiguousarray(blob, np.uint8)
        check(lib().spiir_state_import(self._h, stream_id, blob.ctypes.data, blob.size,
                                       _stream_handle(stream)))

    def info(self) -> dict:
        inf = BankInfo()
        check(lib().spiir_bank_get_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in BankInfo._fields_}

    def enable_timing(self, on: bool = True):
        check(lib().spiir_bank_enable_timing(self._h, int(on)))

    def kernel_times(self) -> dict:
        """{kernel name: (ms summed, launches)} since the last call."""
        kt = KernelTimes()
        check(lib().spiir_bank_kernel_times(self._h, ctypes.byref(kt)))
        return {KERNEL_NAMES[k]: (kt.ms[k], int(kt.launches[k])) for k in range(8)
                if kt.launches[k]}

    def test_stall(self, x, stream=None) -> int:
        """Failure-detection push (see spiir_bank_test_stall); returns its status."""
        return int(lib().spiir_bank_test_stall(self._h, x.data_ptr(), int(x.shape[-1]),
                                               _stream_handle(stream)))

    def sync_status_code(self) -> int:
        return int(lib().spiir_bank_sync_status(self._h))

    def sync_status(self):
        check(lib().spiir_bank_sync_status(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().spiir_bank_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Many banks filtered together (spiir_server_t): one push filters a
    block of every stream through every member with shared strain
    preprocessing and batched launches."""

    def __init__(self, n_streams: int, n_levels: int, block_len: int, max_delay: int,
                 base_rate: int = 4096, mode: str = "plain", chunk_len: int = 0,
                 carry="fp64", tune: int = 0, h_down=None, h_up=None,
                 align: Optional[bool] = None, snr_scale: float = 0.0, tc_min_filters: int = 0,
                 stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libspiir needs a CUDA device")
        d = ServerDesc()
        d.n_streams, d.n_levels, d.base_rate, d.block_len = n_streams, n_levels, base_rate, block_len
        d.max_delay = max_delay
        self._keep = {}
        if h_down is not None:
            self._keep["h_down"] = _arr(h_down, np.float32)
            self._keep["h_up"] = _arr(h_up, np.float32)
            d.h_down = self._keep["h_down"].ctypes.data
            d.h_up = self._keep["h_up"].ctypes.data
            d.n_taps = int(self._keep["h_down"].shape[0])
            d.n_taps_up = int(self._keep["h_up"].shape[0])
        d.align = int(n_levels > 1 if align is None else align)
        d.snr_scale = snr_scale
        d.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        d.chunk_len = chunk_len
        d.carry = CARRY[carry] if isinstance(carry, str) else int(carry)
        d.tune = tune
        d.tc_min_filters = tc_min_filters
        h = _c_void_p()
        check(lib().spiir_server_create(ctypes.byref(d), _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self.n_streams = n_streams
        self.block_len = block_len
        self.n_levels = n_levels
        self._templates = {}

    def _member_desc(self, bank):
        return make_desc(bank, n_streams=self.n_streams, block_len=self.block_len)

    def add(self, bank) -> int:
        """Add a member bank (inputs.Bank); it takes part from the next push."""
        d, _keep = self._member_desc(bank)
        mid = _i32()
        check(lib().spiir_server_add(self._h, ctypes.byref(d), ctypes.byref(mid)))
        self._templates[int(mid.value)] = bank.n_templates
        return int(mid.value)

    def remove(self, member_id: int):
        check(lib().spiir_server_remove(self._h, int(member_id)))
        self._templates.pop(int(member_id), None)

    def member_footprint(self, bank) -> int:
        d, _keep = self._member_desc(bank)
        return int(lib().spiir_server_member_footprint(self._h, ctypes.byref(d)))

    def prepare(self, stream=None):
        """Apply pending additions and removals ahead of the next push."""
        check(lib().spiir_server_prepare(self._h, _stream_handle(stream)))

    def push(self, x, stream=None):
        """x: float32 CUDA tensor [n_streams, block_len], contiguous."""
        assert x.is_cuda and x.is_contiguous() and tuple(x.shape) == (self.n_streams, self.block_len)
        check(lib().spiir_server_push(self._h, x.data_ptr(), _stream_handle(stream)))

    def enable_timing(self, on: bool = True):
        check(lib().spiir_server_enable_timing(self._h, int(on)))

    def kernel_times(self) -> dict:
        """{kernel name: (ms summed, launches)} since the last call."""
        kt = KernelTimes()
        check(lib().spiir_server_kernel_times(self._h, ctypes.byref(kt)))
        return {KERNEL_NAMES[k]: (kt.ms[k], int(kt.launches[k])) for k in range(8)
                if kt.launches[k]}

    def read(self, member_id: int, out=None, stream=None):
        """SNR of the last push for one member: complex64 [n_streams, T, block_len]."""
        import torch
        T = self._templates[int(member_id)]
        if out is None:
            out = torch.empty((self.n_streams, T, self.block_len), dtype=torch.complex64, device="cuda")
        check(lib().spiir_server_read(self._h, int(member_id), out.data_ptr(), _stream_handle(stream)))
        return out

    def info(self) -> dict:
        inf = ServerInfo()
        check(lib().spiir_server_get_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in ServerInfo._fields_}

    def sync_status(self):
        check(lib().spiir_server_sync_status(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().spiir_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Replicas:
    """One bank split by templates over several devices (spiir_replicas_t):
    host strain in, host SNR of the whole bank out."""

    def __init__(self, bank, devices, n_streams: int = 1, block_len: int = 4096,
                 max_push_blocks: int = 1, **kw):
        d, _keep = make_desc(bank, n_streams=n_streams, block_len=block_len,
                             max_push_blocks=max_push_blocks, **kw)
        devs = (ctypes.c_int32 * len(devices))(*devices)
        h = _c_void_p()
        check(lib().spiir_replicas_create(ctypes.byref(d), devs, len(devices), ctypes.byref(h)))
        self._h = h
        self.n_templates = bank.n_templates
        self.n_streams = n_streams
        self.n_replicas = len(devices)

    def push_host(self, x, z_out=None):
        """x: numpy float32 [n_streams, n]; returns complex64 [n_streams, T, n]."""
        x = np.ascontiguousarray(x, np.float32)
        n = int(x.shape[-1])
        if z_out is None:
            z_out = np.empty((self.n_streams, self.n_templates, n), np.complex64)
        check(lib().spiir_replicas_push_host(self._h, x.ctypes.data, n, z_out.ctypes.data))
        return z_out

    def ranges(self):
        """[(device, first template, templates)] per replica."""
        out = []
        for i in range(self.n_replicas):
            dv, t0, nt = _i32(), _i32(), _i32()
            check(lib().spiir_replicas_get(self._h, i, ctypes.byref(dv), ctypes.byref(t0), ctypes.byref(nt)))
            out.append((dv.value, t0.value, nt.value))
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().spiir_replicas_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
