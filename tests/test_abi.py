"""CPU tests of the C ABI: the library loads, exports every symbol the header
declares, and its host-only logic (validation, packing plan, footprint, taps,
rate rule) behaves. No compute call is made here: there is no GPU."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_1702_02256_gb300 import inputs, spiir

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(spiir_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_header_symbol():
    lib = spiir.lib()
    names = _header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"libspiir.so does not export {n}"


def test_library_taps_match_oracle(oracle_mod):
    for n_taps, atten in [(32, 60.0), (16, 50.0), (64, 100.0)]:
        a = spiir.kaiser_taps(n_taps, atten)
        b = oracle_mod.kaiser_taps(n_taps, atten)
        assert np.max(np.abs(a - b)) <= 2 * np.finfo(np.float32).eps * np.max(np.abs(b))


def test_assign_level_matches_oracle(oracle_mod):
    rng = np.random.default_rng(0)
    for _ in range(2000):
        th = rng.uniform(-math.pi, math.pi)
        r = rng.uniform(0.5, 1.0)
        ar, ai = np.float32(r * math.cos(th)), np.float32(r * math.sin(th))
        for L in (1, 4, 7):
            assert spiir.assign_level(ar, ai, 4096, L) == oracle_mod.assign_level(
                float(ar), float(ai), 4096, L)


def test_assign_level_margin_matches_oracle(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(2000):
        th = rng.uniform(-math.pi, math.pi)
        r = rng.uniform(0.5, 1.0)
        ar, ai = np.float32(r * math.cos(th)), np.float32(r * math.sin(th))
        m = float(np.float32(rng.choice([0.0, 0.01, 0.05, 0.2, 1.0])))
        for L in (1, 4, 7):
            assert spiir.assign_level(ar, ai, 4096, L, margin=m) == oracle_mod.assign_level(
                float(ar), float(ai), 4096, L, margin=m)
    assert spiir.lib().spiir_assign_level_margin(0.5, 0.5, 4096, 7, -0.1) == -1
    assert spiir.lib().spiir_assign_level_margin(0.5, 0.5, 4096, 0, 0.1) == -1
    assert spiir.lib().spiir_assign_level(0.5, 0.5, 0, 7) == -1


def _status(bank, **kw):
    d, _k = spiir.make_desc(bank, **kw)
    info = spiir.BankInfo()
    return spiir.lib().spiir_bank_plan(ctypes.byref(d), ctypes.byref(info))


def test_validation_rejects_bad_descriptions():
    bank = inputs.single_rate_bank(3, 5, 10, seed=1)
    assert _status(bank) == spiir.OK
    assert _status(bank, block_len=0) == spiir.EINVAL
    assert _status(bank, n_streams=0) == spiir.EINVAL
    assert _status(bank, max_push_blocks=0) == spiir.EINVAL
    bad = inputs.single_rate_bank(3, 5, 10, seed=1)
    bad.template_id[2] = 7
    assert _status(bad) == spiir.EINVAL
    bad = inputs.single_rate_bank(3, 5, 10, seed=1)
    bad.delay[0] = -1
    assert _status(bad) == spiir.EINVAL
    bad = inputs.single_rate_bank(3, 5, 10, seed=1)
    bad.a_re[1] = np.nan
    assert _status(bad) == spiir.EINVAL
    mr = inputs.multi_rate_bank(2, 3, seed=1)
    assert _status(mr, block_len=4098) == spiir.EINVAL  # not a multiple of 4
    assert _status(mr, block_len=4096, mode="fp16") == spiir.EUNSUPPORTED
    # resampler lengths: decimator up to 512 taps, interpolator up to 64, even
    hd, hu = spiir.kaiser_taps(384, 100.0), spiir.kaiser_taps(32, 60.0)
    assert _status(mr, block_len=4096, h_down=hd, h_up=hu) == spiir.OK
    assert _status(mr, block_len=4096, h_down=spiir.kaiser_taps(514, 100.0), h_up=hu) == spiir.EINVAL
    assert _status(mr, block_len=4096, h_down=hd, h_up=spiir.kaiser_taps(66, 60.0)) == spiir.EINVAL
    assert _status(mr, block_len=4096, h_down=hd, h_up=spiir.kaiser_taps(31, 60.0)) == spiir.EINVAL
    # carry arithmetic of the tensor-core forms: 0 = FP64, 1 = double-float,
    # anything else is rejected before the form is looked at
    assert _status(bank, carry="df") == spiir.OK
    assert _status(bank, carry=2) == spiir.OK
    assert _status(bank, carry=3) == spiir.EINVAL
    assert _status(bank, mode="fp16", carry=-1) == spiir.EINVAL
    d, _k = spiir.make_desc(bank)
    assert spiir.lib().spiir_bank_create(None, None, ctypes.byref(ctypes.c_void_p())) == spiir.EINVAL
    assert "NULL" in spiir.last_error()
    assert spiir.lib().spiir_bank_footprint(None) == -1
    # the queued host push and its sync refuse a NULL bank before any CUDA call
    buf = np.zeros(4096, np.float32)
    zb = np.zeros(2 * 4096, np.float32)
    assert spiir.lib().spiir_push_block_host_async(None, -1, buf.ctypes.data, 4096, zb.ctypes.data,
                                                   None) == spiir.EINVAL
    assert "NULL" in spiir.last_error()
    assert spiir.lib().spiir_bank_host_sync(None) == spiir.EINVAL


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_plan_covers_every_filter(variant):
    counts = [0, 1, 2, 3, 31, 33, 64, 129, 300, 513, 1100]
    bank = inputs.single_rate_bank(len(counts), counts, 500, seed=4)
    p = spiir.plan(bank, tune=-(variant + 1))
    assert p["kernel_variant"] == variant
    assert p["n_slots"] >= bank.n_filters
    assert p["n_slots"] % 64 == 0          # whole rounds of 32 lanes, F even
    assert 0 < p["slot_fill"] <= 1.0
    fmax = p["filters_per_lane"]
    assert fmax % 2 == 0
    # every template with filters is at least one unit; large ones split
    assert p["n_units"] >= sum(1 for c in counts if c)
    assert 1.0 <= p["smem_ways"] <= 32.0


def test_built_in_variant_follows_unit_size():
    """Without tuning, banks whose (template, rate) units hold at most 128
    filters on average run 4 filters per lane (variant 2), larger ones 8
    (variant 3); a forced variant still wins."""
    small = inputs.single_rate_bank(64, 32, 500, seed=4)
    assert spiir.plan(small)["kernel_variant"] == 2
    assert spiir.plan(inputs.single_rate_bank(8, 128, 500, seed=4))["kernel_variant"] == 2
    assert spiir.plan(inputs.single_rate_bank(8, 129, 500, seed=4))["kernel_variant"] == 3
    assert spiir.plan(inputs.single_rate_bank(16, 512, 4095, seed=4))["kernel_variant"] == 3
    # multi-rate: the same filters spread over rates make smaller units
    assert spiir.plan(inputs.multi_rate_bank(50, 7, seed=3))["kernel_variant"] == 2
    # empty templates do not count as units
    uneven = inputs.single_rate_bank(4, [0, 0, 300, 300], 500, seed=4)
    assert spiir.plan(uneven)["kernel_variant"] == 3
    assert spiir.plan(small, tune=-4)["kernel_variant"] == 3


def test_plan_multirate_and_footprint():
    bank = inputs.multi_rate_bank(50, 7, seed=3)
    p = spiir.plan(bank, max_push_blocks=2)
    assert p["max_delay"] >= 1953            # level-0 alignment folded into delays
    f1 = spiir.footprint(bank, max_push_blocks=1)
    f2 = spiir.footprint(bank, max_push_blocks=2)
    assert 0 < f1 < f2
    assert _status(bank, hbm_budget_bytes=1) == spiir.OK  # budget is checked at create


def test_tc_footprint_counts_panels_and_state():
    """The block form's footprint (HBM admission) includes the precomputed
    power panel of every 128-filter tile (32 KB) and 16 bytes of carried
    state per tile slot and stream: adding one tile to one template adds at
    least 32 KB + 128 x 16 B x streams."""
    counts = [1, 128, 129, 300, 0, 5, 256, 64, 65, 1000]
    base = inputs.single_rate_bank(len(counts), counts, 500, seed=1)
    more = inputs.single_rate_bank(len(counts), counts[:-1] + [1000 + 128], 500, seed=1)
    tiles = lambda c: sum(-(-k // 128) for k in c)
    assert tiles(counts[:-1] + [1128]) == tiles(counts) + 1
    for S in (1, 2):
        kw = dict(mode="fp16", n_streams=S, block_len=4096, max_push_blocks=1)
        f0, f1 = spiir.footprint(base, **kw), spiir.footprint(more, **kw)
        assert f0 >= tiles(counts) * (32768 + 128 * 16 * S)
        assert f1 - f0 >= 32768 + 128 * 16 * S
    assert spiir.footprint(base, mode="fp16", n_streams=1) == spiir.footprint(base, mode="bf16", n_streams=1)


def test_workload_shapes_follow_recipes():
    w = inputs.workload(0)
    assert w["bank"].n_filters == 256 and w["x"].shape == (1, 4096)
    w = inputs.workload(2, scale_templates=40)
    b = w["bank"]
    assert b.n_levels == 7 and b.level.min() >= 0 and b.level.max() <= 6
    cnt = np.bincount(b.template_id.astype(np.int64) * 7 + b.level, minlength=40 * 7)
    assert cnt.min() >= 2 and cnt.max() <= 300
    a = np.abs(b.a_re.astype(np.float64) + 1j * b.a_im)
    assert np.all(a < 1.0)
    hi = b.level < 6
    om = np.angle(b.a_re[hi] + 1j * b.a_im[hi].astype(np.float64))
    assert np.all(np.abs(om) >= math.pi / 2 - 1e-6)


@pytest.mark.parametrize("c_name,cls", [("spiir_bank_desc", "BankDesc"), ("spiir_bank_info", "BankInfo"),
                                         ("spiir_kernel_times", "KernelTimes"),
                                         ("spiir_server_desc", "ServerDesc"),
                                         ("spiir_server_info", "ServerInfo")])
def test_struct_layout_matches_the_c_header(tmp_path, c_name, cls):
    """Every field of the ABI's structs sits at the same offset for a C
    compiler (gcc on include/spiir.h) and for the ctypes binding."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    py = getattr(spiir, cls)
    names = [f for f, _ in py._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"spiir.h\"\nint main(void) {\n"
                   + "".join(f'    printf("{n} %zu\\n", offsetof({c_name}, {n}));\n' for n in names)
                   + f'    printf("sizeof %zu\\n", sizeof({c_name}));\n    return 0;\n}}\n')
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                         text=True).stdout.splitlines())
    for n in names:
        assert int(out[n]) == getattr(py, n).offset, n
    assert int(out["sizeof"]) == ctypes.sizeof(py)
