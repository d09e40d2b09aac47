#!/usr/bin/env python
"""Benchmark of the SPIIR hot path on GB300.

Default workload: single-rate bank, 1024 templates x 512 complex filters,
4096 Hz, 16 s of seeded white Gaussian strain pushed as one 16-block push per
step (the plain FP32 recursion path). One JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload single|multirate]

N > 1 (torchrun): every rank filters its own bank of the same shape (weak
scaling, no collective on the data path); the timing is the max over ranks.
--impl reference times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1702_02256_gb300 import replicas  # noqa: E402

METRIC = "real-time templates/GPU (filter-samples/s) & p99 block latency, chosen vs plain"
UNIT = "filter-samples/s"
FLOPS_PER_FS = 12          # Sec. 2.2 cost model: 12 flops per filter per sample
LANE_OPS_PER_FS = 8        # 2 FMUL + 4 FFMA + 2 FADD per filter-sample
FP32_LANES_PER_SM = 128


def _dist():
    from paper_1702_02256_gb300 import replicas
    return replicas.world()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.gpu_id],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self):
        self.marks.append(time.time())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [l for (t, l) in self.lines if t0 - 0.25 <= t <= t1 + 0.25]
        if not rows:
            rows = [l for (_, l) in self.lines[-3:]]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _gpu_id(torch, dev: int) -> str:
    try:
        p = torch.cuda.get_device_properties(dev)
        return "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[dev] if vis else str(dev)


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def _source_hash(kernel_file: str, csrc: str = "") -> str:
    """First 16 hex digits of the sha256 of the kernel file followed by the
    planner (spiir_api.cu), comments and blank lines left out: the traffic
    depends on the code of both, not on their comments."""
    csrc = csrc or os.path.join(ROOT, "paper_1702_02256_gb300", "csrc")
    h = hashlib.sha256()
    for f in (kernel_file, "spiir_api.cu"):
        src = open(os.path.join(csrc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip()).encode())
    return h.hexdigest()[:16]


def _traffic(kernel_file: str, key: str, variant=None):
    """DRAM bytes per launch from a committed ncu summary, if the kernel and
    planner sources have not changed since it was taken and, where the
    summary names a kernel variant, the run used that variant."""
    path = os.path.join(ROOT, "profiles", f"{key}_traffic.txt")
    try:
        kv = dict(tok.split("=", 1) for tok in open(path).read().split() if "=" in tok)
    except OSError:
        return None
    if kv.get("source_sha256_16") != _source_hash(kernel_file):
        return None
    if "kernel_variant" in kv and (variant is None or int(kv["kernel_variant"]) != int(variant)):
        return None
    return float(kv["dram_bytes_per_launch"])


def _workload(name: str, rank: int, templates: int = 0, seconds: int = 0):
    """The benchmark workloads: seeded synthetic banks of the configurations'
    shapes, one bank per rank (weak scaling)."""
    from paper_1702_02256_gb300 import inputs
    if name == "single":
        T = templates or 1024
        sec = seconds or 16
        bank = inputs.single_rate_bank(T, 512, 4095, seed=replicas.rank_seed(0, rank))
        return dict(bank=bank, x=inputs.strain(1, sec * 4096, seed=1 + 100 * rank),
                    block_len=4096, push_blocks=sec, n_streams=1, chunk_len=256,
                    desc=f"single-rate {T} templates x 512 filters, 4096 Hz, {sec} s per step "
                         f"(one {sec}-block push), delays 0-4095")
    if name == "multirate":
        T = templates or 4000
        sec = seconds or 16
        bank = inputs.multi_rate_bank(T, 7, seed=replicas.rank_seed(0, rank))
        return dict(bank=bank, x=inputs.strain(1, sec * 4096, seed=1 + 100 * rank),
                    block_len=4096, push_blocks=1, n_streams=1, chunk_len=256,
                    desc=f"multi-rate {T} templates, 7 rates 4096-64 Hz, {sec} s per step "
                         f"({sec} pushes of 1 s)")
    if name == "tc":
        T = templates or 8000
        sec = seconds or 8
        bank = inputs.single_rate_bank(T, 256, 1023, seed=replicas.rank_seed(0, rank))
        return dict(bank=bank, x=inputs.strain(2, sec * 4096, seed=1 + 100 * rank),
                    block_len=4096, push_blocks=1, n_streams=2, chunk_len=256,
                    desc=f"single-rate {T} templates x 256 filters, 2 streams, 4096 Hz, {sec} s "
                         f"per step ({sec} pushes of 1 s of both streams), delays 0-1023")
    raise SystemExit(f"unknown workload {name}")


def _cpu_sample(w, budget_s: float, n_templates_max: int, threads: int = 0):
    """Time the oracle on the host cores (all of them, or `threads`) over a
    bounded template sample sized to about budget_s seconds. Returns
    (filter-samples/s, sample text, cores)."""
    from oracle import oracle
    bank = w["bank"]
    x = w["x"][0]
    threads = threads or oracle.default_threads()
    multi = bank.n_levels > 1

    def run(sel):
        t0 = time.perf_counter()
        if multi:
            oracle.spiir_multirate(bank, x, h_down=w.get("h_down"), h_up=w.get("h_up"),
                                   templates=sel, threads=threads)
        else:
            oracle.spiir_single(bank, x, templates=sel, threads=threads)
        return time.perf_counter() - t0

    def fs(sel):
        cnt = np.bincount(bank.template_id, minlength=bank.n_templates)
        lev_fs = 0
        for t in sel:
            m = bank.template_id == t
            lev_fs += int(np.sum(x.shape[0] >> bank.level[m].astype(np.int64)))
        return lev_fs

    n0 = max(1, threads)
    sel = np.arange(min(n0, bank.n_templates), dtype=np.int32)
    dt = run(sel)
    rate = fs(sel) / dt
    per_t = dt / len(sel)
    n = int(min(n_templates_max, bank.n_templates, max(len(sel), budget_s / per_t)))
    n = max(threads, (n // threads) * threads) if n >= threads else n
    sel = np.arange(n, dtype=np.int32)
    dt = run(sel)
    rate = fs(sel) / dt
    sample = f"{n} of {bank.n_templates} templates, full {x.shape[0]} samples, {dt:.1f} s wall"
    _cpu_sample.last_wall_s = dt
    return rate, sample, threads


def run_sweep(args):
    """Throughput against filters per template (the paper's speed-up table,
    Table tab:spiir_speedup): single-rate banks of about 2^19 filters,
    M = 4 .. 512 filters per template, 1 s pushes of 1 s blocks, plain form
    and the fp16 block form; fraction of the FP32 roofline for the plain form."""
    import torch
    from paper_1702_02256_gb300 import inputs
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    peaks = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_fs = sms * FP32_LANES_PER_SM * sm_max * 1e6 / LANE_OPS_PER_FS
    rows = []
    for M in (4, 8, 16, 32, 64, 128, 256, 512):
        T = (1 << 19) // M
        bank = inputs.single_rate_bank(T, M, 1023, seed=5)
        w = dict(bank=bank, x=inputs.strain(1, 4 * 4096, seed=3), block_len=4096, push_blocks=1,
                 n_streams=1, chunk_len=256, desc=f"{T} templates x {M} filters")
        row = {"filters_per_template": M, "templates": T}
        for form in ("plain", "fp16"):
            m = _measure(w, form, args, dev, None, None, 0, 1)
            row[form] = {"filter_samples_per_s": m["value"], "p99_block_latency_ms": m["p99"]}
            if form == "plain":
                row[form]["roofline_frac"] = m["value"] / peak_fs
                row[form]["kernel_variant"] = m["info"]["kernel_variant"]
        rows.append(row)
    line = {"metric": "filter-samples/s by filters per template (plain and fp16 block form)",
            "value": rows[-1]["plain"]["filter_samples_per_s"], "unit": UNIT, "higher_is_better": True,
            "n_gpus": 1, "data": "synthetic", "rows": rows,
            "config": {"workload": "single-rate banks of 2^19 filters, delays 0-1023, 4 s in 1 s pushes"}}
    print(json.dumps(line), flush=True)
    return 0


def run_ratesweep(args):
    """Throughput against the number of rates (the paper's multi-rate table,
    Table tab:multirate_speedup): 4096 templates whose 1024 filters are split
    equally over R = 1, 2, 3, 4, 8 rates from 4096 Hz down (R = 1: all at full
    rate), plain form, 1 s pushes of 4 s of strain. Reports the device time per
    second of strain and its ratio to R = 1 (the paper's GPU row: 287, 220,
    199, 143, 85 s, i.e. 1.30x, 1.44x, 2.01x, 3.38x)."""
    import torch
    from paper_1702_02256_gb300 import inputs
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    T, M = 4096, 1024
    if args.tune is None:
        args.tune = 1
    rows = []
    for R in (1, 2, 3, 4, 8):
        counts = np.full((T, R), M // R, np.int64)
        counts[:, 0] += M - counts.sum(axis=1)
        bank = inputs.multi_rate_bank(T, R, seed=7, counts=counts)
        w = dict(bank=bank, x=inputs.strain(1, 4 * 4096, seed=3), block_len=4096, push_blocks=1,
                 n_streams=1, chunk_len=256, desc=f"{T} templates x {M} filters over {R} rates")
        m = _measure(w, "plain", args, dev, None, None, 0, 1)
        ms_per_s = m["ms_per_step"] / (w["x"].shape[1] / 4096.0)
        rows.append({"rates": R, "filters_per_rate": [int(c) for c in counts[0]],
                     "ms_per_second_of_strain": ms_per_s,
                     "filter_samples_per_s": m["value"], "kernel_variant": m["info"]["kernel_variant"],
                     "kernel_share": {k: round(v[0] / max(1e-9, sum(x[0] for x in m["kt"].values())), 4)
                                      for k, v in m["kt"].items()}})
    for r in rows:
        r["time_ratio_vs_1_rate"] = rows[0]["ms_per_second_of_strain"] / r["ms_per_second_of_strain"]
    line = {"metric": "device time per second of strain by number of rates (plain form)",
            "value": rows[-1]["time_ratio_vs_1_rate"], "unit": "x faster than 1 rate",
            "higher_is_better": True, "n_gpus": 1, "data": "synthetic", "rows": rows,
            "config": {"workload": f"{T} templates x {M} filters split equally over 1-8 rates "
                                   f"(4096 Hz down), delays 0-1023, 4 s in 1 s pushes, autotuned tiles",
                       "paper_gpu_ratio": {"2": 287 / 220, "3": 287 / 199, "4": 287 / 143, "8": 287 / 85}}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    w = _workload(args.workload, 0, args.templates, args.seconds)
    per_step = max(1.0, 150.0 / max(1, args.steps + args.warmup))
    rates = []
    sample = ""
    threads = 1
    walls = []
    for i in range(args.warmup + args.steps):
        rate, sample, threads = _cpu_sample(w, per_step, 64)
        if i >= args.warmup:
            rates.append(rate)
            walls.append(_cpu_sample.last_wall_s)
    value = float(np.mean(rates))
    bank = w["bank"]
    n = w["x"].shape[1]
    fs_total = w["n_streams"] * int(np.sum(n >> bank.level.astype(np.int64)))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * fs_total / value, "higher_is_better": True,
        "ms_per_step_extrapolated": True,
        "ms_per_step_basis": "not measured: the full step's filter-samples divided by the rate "
                             "measured on a bounded template sample (the oracle would take this "
                             "long for one whole step)",
        "sample_wall_ms_per_step": 1e3 * float(np.mean(walls)),
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "n_templates": bank.n_templates,
                   "n_filters": bank.n_filters},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


FORM_MODE = {"plain": "plain", "fp16": "fp16", "bf16": "bf16"}


def _measure(w, form, args, dev, dist, sampler, rank, ws, err=None):
    """Time one form of the filtering on workload w. Returns a dict of the
    device-timed throughput, per-kernel times, latency and end-to-end rate.
    err = (template indices, samples): afterwards the state is reset and the
    first samples are pushed again, and the SNR of those templates is
    returned as "err_z" (complex64 [streams, templates, samples]) for the
    comparison with the oracle."""
    import torch
    from paper_1702_02256_gb300 import spiir
    bank = w["bank"]
    S = w["n_streams"]
    n = w["x"].shape[1]
    push_len = w["block_len"] * w["push_blocks"]
    kw = dict(tune=args.tune) if form == "plain" else dict(mode=form, chunk_len=w["chunk_len"], carry=args.carry)
    if w.get("h_down") is not None:
        kw.update(h_down=w["h_down"], h_up=w["h_up"])
    # an output ring of two pushes: the end-to-end leg's asynchronous host
    # pushes alternate its halves (device pushes use the first)
    b = spiir.Bank(bank, n_streams=S, block_len=w["block_len"], max_push_blocks=2 * w["push_blocks"], **kw)
    info = b.info()
    x = torch.from_numpy(w["x"]).to(dev)
    pushes = [x[:, s0:s0 + push_len].contiguous() for s0 in range(0, n, push_len)]
    fs_per_step = S * int(np.sum(n >> bank.level.astype(np.int64)))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step():
        for p in pushes:
            b.push(p, stream_id=-1)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    b.enable_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    for i in range(args.steps):
        flush.zero_()                      # L2 flushed between timed steps (untimed)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall1 = time.time()
    kt = b.kernel_times()
    b.enable_timing(False)
    total_ms = replicas.max_over_ranks(sum(e0.elapsed_time(e1) for e0, e1 in ev), dist, dev)
    ms_per_step = total_ms / args.steps

    # per-block latency: one 1 s block of every stream per push, push -> SNR out
    blk = w["block_len"]
    xb = x[:, :blk].contiguous()
    zout = torch.empty((S, bank.n_templates, blk), dtype=torch.complex64, device=dev)
    lat = []
    for i in range(40):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.push(xb, stream_id=-1)
        b.read(blk, stream_id=-1, out=zout)
        e1.record(stream)
        e1.synchronize()
        if i >= 5:
            lat.append(e0.elapsed_time(e1))
    lat = np.array(lat)

    # end to end through the asynchronous host-buffer entry point: a step
    # queues its pushes (strain in from pinned host memory, SNR out to it)
    # and ends when the SNR of its last push is in host memory; a push
    # computes while the SNR of the one before it is copied out
    xh_pushes = [torch.from_numpy(np.ascontiguousarray(w["x"][:, s0:s0 + push_len])).pin_memory()
                 for s0 in range(0, n, push_len)]
    zh = torch.empty((S, bank.n_templates, push_len), dtype=torch.complex64).pin_memory()
    for p in xh_pushes:
        b.push_host_async(p, zh)
    b.host_sync()
    # steps are timed on the host clock in blocks of e2e_block that end when
    # the block's last SNR is in host memory (consecutive steps overlap as
    # consecutive pushes do), and the median block stands for the rate (a
    # stall of the host process shows in the maximum, not in the rate)
    e2e_block = max(2, min(args.steps, 4))
    step_s = []
    for _ in range(3):
        t0 = time.perf_counter()
        for _ in range(e2e_block):
            for p in xh_pushes:
                b.push_host_async(p, zh)
        b.host_sync()
        step_s.append((time.perf_counter() - t0) / e2e_block)
    e2e_s = replicas.max_over_ranks(float(np.median(step_s)), dist, dev)
    err_z = None
    if err is not None:
        sel, n_err = err
        b.reset()
        idx = torch.from_numpy(np.asarray(sel, np.int64)).to(dev)
        zz = torch.empty((S, bank.n_templates, push_len), dtype=torch.complex64, device=dev)
        parts = []
        for p in pushes[:max(1, n_err // push_len)]:
            b.push(p, stream_id=-1)
            b.read(push_len, stream_id=-1, out=zz)
            parts.append(zz.index_select(1, idx).cpu().numpy())
        err_z = np.concatenate(parts, axis=-1)
    b.sync_status()
    b.close()
    del flush
    torch.cuda.synchronize()
    return dict(form=form, info=info, kt=kt, ms_per_step=ms_per_step,
                value=replicas.job_rate(fs_per_step * args.steps, ws, total_ms / 1e3),
                fs_per_step=fs_per_step, steps=args.steps,
                rtt=ws * bank.n_templates * S * (n / 4096.0) / (ms_per_step / 1e3),
                p50=float(np.percentile(lat, 50)), p99=float(np.percentile(lat, 99)),
                e2e=ws * fs_per_step / e2e_s, h2d=int(S * n * 4),
                e2e_steps_ms={"median": 1e3 * float(np.median(step_s)), "min": 1e3 * min(step_s),
                              "max": 1e3 * max(step_s), "steps": len(step_s) * e2e_block,
                              "steps_per_block": e2e_block},
                d2h=int(S * bank.n_templates * n * 8), wall=(t_wall0, t_wall1), err_z=err_z)


_LINK = {}


def _host_link(torch, dev):
    """Device-to-host and host-to-device copy bandwidth of this GPU's host link
    (GB/s): 256 MB between a device buffer and a pinned host buffer, best of 3
    copies each way, CUDA events on a side stream. Measured once per run."""
    if _LINK:
        return _LINK
    nbytes = 256 << 20
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    st = torch.cuda.Stream(dev)
    out = {}
    for name, dst, src in (("d2h_gbs", h, d), ("h2d_gbs", d, h)):
        best = 0.0
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(st):
                e0.record(st)
                dst.copy_(src, non_blocking=True)
                e1.record(st)
            e1.synchronize()
            best = max(best, nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9)
        out[name] = best
    del d, h
    _LINK.update(out)
    return _LINK


def _e2e_json(m, torch, dev):
    """The end-to-end object: the host-buffer rate, its copy bytes, and the
    bound the measured host link puts on it (each step's copies at the link's
    rates, overlapped with the device step)."""
    link = _host_link(torch, dev)
    t_link = max(m["d2h"] / (link["d2h_gbs"] * 1e9), m["h2d"] / (link["h2d_gbs"] * 1e9),
                 m["ms_per_step"] / 1e3)
    bound = m["fs_per_step"] / t_link
    return {"value": m["e2e"], "unit": UNIT, "h2d_bytes_per_step": m["h2d"],
            "d2h_bytes_per_step": m["d2h"],
            "basis": "host-buffer pushes through spiir_push_block_host_async (strain in from and SNR out "
                     "to pinned host memory; a push computes while the SNR of the one before it is copied "
                     "out), timed in blocks of steps that end when the block's last SNR is in host "
                     "memory (spiir_bank_host_sync); the rate of the median block, per step",
            "step_ms": {k: (round(v, 3) if isinstance(v, float) else v) for k, v in m["e2e_steps_ms"].items()},
            "host_link": {"d2h_gbs": round(link["d2h_gbs"], 1), "h2d_gbs": round(link["h2d_gbs"], 1)},
            "link_bound": bound, "frac_of_link_bound": m["e2e"] / bound}


def _form_desc(form: str, args) -> str:
    if form == "plain":
        return "plain FP32 recursion"
    carry = {"fp64": "FP64 state anchor per chunk batch", "df": "double-float state anchor per chunk batch",
             "fp64chunk": "FP64 state at every chunk"}[args.carry]
    return f"tensor-core block form ({form}, {carry})"


def _oracle_error(w, sel, z):
    """SNR error of a GPU run against the FP64 oracle (part of the CPU
    baseline leg: the oracle runs on the host cores): per template and
    stream, RMS error over RMS oracle SNR, on the sampled templates and the
    first samples of the workload."""
    from oracle import oracle
    bank = w["bank"]
    n = z.shape[-1]
    errs = []
    for s in range(z.shape[0]):
        x = w["x"][s, :n]
        if bank.n_levels > 1:
            ref = oracle.spiir_multirate(bank, x, h_down=w.get("h_down"), h_up=w.get("h_up"),
                                         templates=sel)
        else:
            ref = oracle.spiir_single(bank, x, templates=sel)
        num = np.sqrt(np.mean(np.abs(z[s] - ref) ** 2, axis=-1))
        den = np.sqrt(np.mean(np.abs(ref) ** 2, axis=-1))
        errs.append(num / np.where(den > 0, den, 1.0))
    e = np.concatenate(errs)
    return {"max": float(e.max()), "median": float(np.median(e)), "templates": int(len(sel)),
            "streams": int(z.shape[0]), "seconds": n / 4096.0,
            "measure": "per template and stream: RMS(z - z_oracle) / RMS(z_oracle), FP64 oracle"}


def _err_sample(w, k=8, seconds=2):
    """Templates and samples of the oracle comparison: k spread templates,
    the first `seconds` seconds (at least one push)."""
    T = w["bank"].n_templates
    sel = np.unique(np.linspace(0, T - 1, k).round().astype(np.int32))
    push_len = w["block_len"] * w["push_blocks"]
    n = max(push_len, (seconds * 4096 // push_len) * push_len)
    return sel, min(n, w["x"].shape[1])


def _roofline(m, w, args, peaks, sms, wl=None):
    """Roofline of the dominant kernel of one measured form."""
    wl = wl or args.workload
    kt = m["kt"]
    bank = w["bank"]
    if m["form"] == "plain":
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        peak = sms * FP32_LANES_PER_SM * sm_max * 1e6 / LANE_OPS_PER_FS * FLOPS_PER_FS / 1e12
        ms, nl = kt.get("recur", (0.0, 0))
        ach = FLOPS_PER_FS * m["fs_per_step"] * m["steps"] / nl / (ms / nl / 1e3) / 1e12 if nl else 0.0
        return {"bound": "alu", "kernel": "recur_kernel", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak if peak else None,
                "traffic": _traffic("spiir_plain.cu", f"recur_{wl}",
                                    m["info"].get("kernel_variant")),
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_max:.0f} MHz "
                              f"(sm_max_mhz of measured peaks) / {LANE_OPS_PER_FS} lane-ops x "
                              f"{FLOPS_PER_FS} flops per filter-sample"}
    # tensor-core form: algorithmic contraction flops of the dominant kernel
    S = w["n_streams"]
    samples = S * w["x"].shape[1] * m["steps"]
    F = m["info"]["tc_fir_len"]
    L = w["chunk_len"]
    passes = 3 if m["form"] == "bf16x2" else 1                     # split bf16: hi*hi + hi*lo + lo*hi
    fir_flops = passes * 4.0 * (F + L) * bank.n_templates * samples   # 2 real rows x 2 flops x K
    carry_flops = 12.0 * bank.n_filters * samples                 # 4M state + 8M output
    fir_ms, fir_n = kt.get("tc_fir", (0.0, 0))
    car_ms, car_n = kt.get("tc_carry", (0.0, 0))
    peak = float(peaks.get("bf16_tflops", 1890.7))
    if fir_ms >= car_ms:
        name, ach = "tc_fir_kernel", fir_flops / (fir_ms / 1e3) / 1e12 if fir_ms else 0.0
    else:
        name, ach = "tc_carry_kernel", carry_flops / (car_ms / 1e3) / 1e12 if car_ms else 0.0
    key = ("tc_fir" if name == "tc_fir_kernel" else "tc_carry") + f"_{wl}"
    return {"bound": "tensor", "kernel": name, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": _traffic("spiir_tc.cu", key),
            "peak_basis": "measured dense bf16 burst (cuBLAS) of MEASURED_PEAKS; fp16 has the same "
                          "nominal dense rate" + ("; the split-bf16 FIR counts its three passes"
                                                  if passes > 1 else ""),
            "fir_tflops": fir_flops / (fir_ms / 1e3) / 1e12 if fir_ms else None,
            "carry_tflops": carry_flops / (car_ms / 1e3) / 1e12 if car_ms else None}


def _workload_desc(name):
    return {"tc": "single-rate 8000 templates x 256 filters, 2 streams, 4096 Hz, 8 s per step "
                  "(8 pushes of 1 s of both streams), delays 0-1023, chunk length 256"}[name]


def _leg_json(m, w, wl, args, peaks, sms, plain=None, err=None):
    """One measured form of a workload as a JSON object: rate, step time,
    latency, roofline of its dominant kernel, end-to-end rate and SNR error
    against the oracle; speed-up over the plain form's leg when given."""
    import torch
    o = {
        "form": _form_desc(m["form"], args),
        "value": m["value"], "unit": UNIT, "ms_per_step": m["ms_per_step"], "steps": m["steps"],
        "real_time_templates": m["rtt"],
        "p50_block_latency_ms": m["p50"], "p99_block_latency_ms": m["p99"],
        "roofline": _roofline(m, w, args, peaks, sms, wl),
        "e2e": _e2e_json(m, torch, torch.cuda.current_device()),
        "kernel_ms": {k: v[0] for k, v in m["kt"].items()},
        "gpu_launches": int(sum(c for _, c in m["kt"].values())),
    }
    if plain is not None:
        o["speedup_vs_plain"] = m["value"] / plain["value"]
    if m.get("err_z") is not None and err is not None:
        o["snr_error_vs_oracle"] = _oracle_error(w, err[0], m["err_z"])
    return o


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = _workload(args.workload, rank, args.templates, args.seconds)
    if args.resampler == "paper":
        # Sec. 2.2's pair: a 384-tap 100 dB decimator, a 32-tap 60 dB interpolator
        from paper_1702_02256_gb300 import spiir
        w["h_down"], w["h_up"] = spiir.kaiser_taps(384, 100.0), spiir.kaiser_taps(32, 60.0)
        w["desc"] += ", resampler: 384-tap 100 dB decimator, 32-tap 60 dB interpolator"
    sampler = ClockSampler(_gpu_id(torch, local)) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.5)
    form = args.form or ("fp16" if args.workload == "tc" else "plain")
    lead = rank == 0 and ws == 1      # oracle comparisons: one GPU, rank 0
    err = _err_sample(w) if lead else None
    main = _measure(w, form, args, dev, dist, sampler, rank, ws, err=err)
    chosen = None
    if args.chosen and args.chosen != form and w["bank"].n_levels == 1:
        chosen = _measure(w, args.chosen, args, dev, dist, sampler, rank, ws, err=err)
    # the block-parallel configuration (8000 x 256 filters, 2 streams, 1 s
    # pushes): the plain form and every requested tensor-core form
    # the multi-rate bank (4000 templates, 7 rates), autotuned, 16 s in 1 s pushes
    c2 = None
    if args.workload == "single" and args.config2:
        w2 = _workload("multirate", rank)
        err2 = _err_sample(w2) if lead else None
        tune_keep = args.tune
        args.tune = 1
        c2 = ("plain", _measure(w2, "plain", args, dev, dist, sampler, rank, ws, err=err2))
        args.tune = tune_keep
    c3 = []
    if args.workload == "single" and args.config3:
        w3 = _workload("tc", rank)
        err3 = _err_sample(w3) if lead else None
        for f3 in ["plain"] + [f for f in args.config3.split(",") if f]:
            c3.append((f3, _measure(w3, f3, args, dev, dist, sampler, rank, ws, err=err3)))
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    sampler.stop()
    clocks = sampler.summary(*main["wall"])
    peaks = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    kt = main["kt"]
    tot = max(1e-9, sum(v[0] for v in kt.values()))
    shares = {k: round(v[0] / tot, 4) for k, v in kt.items()}
    cpu_rate, cpu_sample, cores = _cpu_sample(w, 10.0, 256)
    cpu1_rate, cpu1_sample, _ = _cpu_sample(w, 3.0, 64, threads=1)
    bank = w["bank"]
    line = {
        "metric": METRIC,
        "value": main["value"],
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": main["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if form == "plain" else form,
        "data": "synthetic",
        "config": {
            "workload": w["desc"],
            "n_templates": bank.n_templates,
            "n_filters": bank.n_filters,
            "n_streams": w["n_streams"],
            "samples_per_step": int(w["x"].shape[1]),
            "form": _form_desc(form, args),
            "kernel_variant": main["info"]["kernel_variant"],
            "variant_choice": {1: "autotuned at bank creation", 0: "default"}.get(
                args.tune, f"forced {-args.tune - 1}") if form == "plain" else "n/a",
            "filters_per_lane": main["info"]["filters_per_lane"],
            "time_tile": main["info"]["time_tile"],
            "l2": "flushed between timed steps (256 MB write, untimed)",
            "parallelism": f"{ws} independent bank replicas" if ws > 1 else "1 GPU",
            "reduction": args.ablation,
            "segment_base": main["info"].get("segment_base"),
            "ctas_per_sm": main["info"].get("ctas_per_sm"),
            "tune_ms": main["info"].get("tune_ms"),
        },
        "real_time_templates": main["rtt"],
        "p50_block_latency_ms": main["p50"],
        "p99_block_latency_ms": main["p99"],
        "kernel_share": shares,
        "roofline": _roofline(main, w, args, peaks, sms),
        "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": cpu_sample},
        "cpu_baseline_single_thread": {"value": cpu1_rate, "unit": UNIT, "cores": 1,
                                       "kind": "oracle", "sample": cpu1_sample},
        "e2e": _e2e_json(main, torch, dev),
        "gpu_launches": int(sum(c for _, c in kt.values())),
        "clocks": clocks,
    }
    if main["err_z"] is not None:
        line["snr_error_vs_oracle"] = _oracle_error(w, err[0], main["err_z"])
    if chosen:
        line["chosen"] = _leg_json(chosen, w, args.workload, args, peaks, sms, main, err)
    if c2:
        line["config2"] = {
            "workload": w2["desc"],
            "variant_choice": "autotuned at bank creation",
            "kernel_variant": c2[1]["info"]["kernel_variant"],
            "segment_base": c2[1]["info"].get("segment_base"),
            "ctas_per_sm": c2[1]["info"].get("ctas_per_sm"),
            "tune_ms": c2[1]["info"].get("tune_ms"),
            "legs": {"plain": _leg_json(c2[1], w2, "multirate", args, peaks, sms, None, err2)},
        }
    if args.workload == "single" and args.serving and ws == 1:
        line["serving"] = _serve_line(args)
    if c3:
        plain3 = c3[0][1]
        line["config3"] = {
            "workload": _workload_desc("tc"),
            "legs": {f: _leg_json(m, w3, "tc", args, peaks, sms, plain3 if f != "plain" else None, err3)
                     for f, m in c3},
        }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def _serve_trial(kind, form, scale, n_blocks, seed, budget, batched=True, warm=2):
    """One serving run of the configuration-4 request process (Poisson
    arrivals 2/s, template counts log-uniform 50-20000 times `scale`,
    128-512 filters, lifetimes 10-60 blocks, 3 streams, 1 s blocks), started
    from the steady-state population. batched: all requests are members of
    one libspiir server (one push per block); else each request is a bank of
    its own on its own CUDA stream. Returns the latency and load summary."""
    import torch
    from paper_1702_02256_gb300 import inputs, serve, spiir
    block = 4096
    reqs = inputs.serving_requests(int(2 * n_blocks + 200), seed=seed)
    t0 = 40.0     # requests arriving in the 40 s before block 0 may still be alive
    n_levels = 7 if kind == "multirate" else 1
    if batched:
        engine = spiir.Server(3, n_levels, block, 1023, mode=form,
                              chunk_len=256 if form != "plain" else 0)
        srv = serve.BatchedServer(budget, 3, block, engine)
    else:
        make, fp = serve.device_bank_factory(form, block_len=block, n_streams=3)
        srv = serve.Server(budget, 3, block, make, fp)
    for i, r in enumerate(reqs):
        t = r["arrival_s"] - t0
        if t >= n_blocks:
            break
        first = max(0, int(np.ceil(t)))
        # a request that arrived before block 0 has already served part of
        # its lifetime
        life = r["lifetime"] - (int(np.ceil(-t)) if t < 0 else 0)
        if life <= 0:
            continue
        T = max(1, int(round(r["n_templates"] * scale)))
        q = dict(r, n_templates=T)
        if kind == "multirate":
            bank = inputs.request_bank(q)
        else:
            bank = inputs.single_rate_bank(T, r["filters"], 1023, seed=r["seed"])
        srv.submit(serve.Request(i, bank, first, life))
    x = torch.from_numpy(inputs.strain(3, n_blocks * block, seed=seed + 1)).cuda()
    t_wall = time.perf_counter()
    for b in range(n_blocks):
        srv.step(x[:, b * block:(b + 1) * block].contiguous())
    t_wall = time.perf_counter() - t_wall
    srv.drain()
    out = serve.summarize(srv, warm_blocks=warm)
    out["wall_s"] = t_wall
    prep = [r.get("prepare_ms", 0.0) for r in srv.log[warm:]]
    if prep:
        out["p50_prepare_ms"] = float(np.percentile(prep, 50))
        out["max_prepare_ms"] = float(np.max(prep))
    if batched:
        engine.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def _serve_search(kind, form, args, budget, batched=True):
    """Largest template scale whose p99 block latency stays under 10 ms. Short
    runs steer the scale (each step rescales by the latency it saw, then a
    geometric bisection between the largest passing and smallest failing
    scale); one confirmation run of args.serve_confirm blocks at the scale
    found gives the reported numbers (its p99 is a percentile of at least
    200 blocks); if that run misses the SLO, the scale is lowered 10% and
    confirmed once more."""
    trials = []
    scale = args.serve_scale0
    lo, hi, best = None, None, None
    for _ in range(args.serve_trials):
        r = _serve_trial(kind, form, scale, args.serve_blocks, 7, budget, batched)
        r["scale"] = scale
        trials.append(r)
        p99 = r.get("p99_block_latency_ms", 1e9) if r.get("blocks", 0) else 1e9
        if p99 < 10.0:
            lo, best = scale, r
        else:
            hi = scale
        if lo is not None and hi is not None:
            if hi / lo < 1.06:
                break
            scale = (lo * hi) ** 0.5
        else:
            step = 8.5 / max(p99, 0.5)
            scale = scale * (min(4.0, max(1.25, step)) if hi is None else max(0.25, min(0.8, step)))
    confirm, last = None, None
    if lo is not None and args.serve_confirm > 0:
        sc = lo
        for _ in range(3):
            r = _serve_trial(kind, form, sc, args.serve_confirm, 7, budget, batched)
            r["scale"] = sc
            last = r
            if r.get("blocks", 0) and r["p99_block_latency_ms"] < 10.0:
                confirm = r
                break
            # the longer run saw a heavier load: rescale by its p99 (block
            # time is close to proportional to the templates served)
            sc *= 9.5 / max(r.get("p99_block_latency_ms", 20.0), 1.0)
    return {"search": trials, "at_slo": best, "confirm": confirm or last}


def _serve_summary(res):
    """Real-time templates at the SLO from the confirmation run (or the best
    search run): the offered load that was served, with p50/p99 latency."""
    r = res["confirm"] or res["at_slo"]
    if not r:
        return {"real_time_templates": 0.0}
    return {
        "real_time_templates": 3 * r["mean_active_templates"],
        "real_time_templates_basis": "templates x 3 streams served in real time (1 s blocks, "
                                     "every block finished) with p99 block latency < 10 ms; "
                                     "mean over the run",
        "p50_block_latency_ms": r["p50_block_latency_ms"],
        "p99_block_latency_ms": r["p99_block_latency_ms"],
        "blocks": r["blocks"], "scale": r["scale"],
        "max_active_templates": r["max_active_templates"],
        "slo_met": r["p99_block_latency_ms"] < 10.0,
    }


def run_serve(args):
    """Largest sustained load (real-time templates, 3 streams) with p99 block
    latency under 10 ms, plain form versus tensor-core form, on the
    configuration-4 request process, through the batched server."""
    import torch
    torch.cuda.set_device(0)
    line = _serve_line(args)
    print(json.dumps(line), flush=True)
    return 0


def _serve_line(args):
    import torch
    budget = int(torch.cuda.get_device_properties(0).total_memory * 0.8)
    kind = args.serve_kind
    forms = ["plain"] + [f for f in args.serve_forms.split(",") if f and f != "plain"]
    res = {f: _serve_search(kind, f, args, budget) for f in forms}
    out = {
        "metric": "real-time templates/GPU at p99 block latency < 10 ms (3 streams, 1 s blocks)",
        "unit": "templates", "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
        "config": {"workload": "serving loop: Poisson bank requests 2/s, template counts "
                               "log-uniform 50-20000 x scale, 128-512 filters per template "
                               + ("split over 7 rates 4096-64 Hz" if kind == "multirate" else "single rate")
                               + ", lifetimes 10-60 blocks, 3 streams, 1 s blocks, HBM budget 80% of "
                               "the device, all requests batched in one server",
                   "requests": kind},
        "plain": _serve_summary(res["plain"]),
    }
    for f in forms[1:]:
        o = _serve_summary(res[f])
        if out["plain"]["real_time_templates"]:
            o["ratio_vs_plain"] = o["real_time_templates"] / out["plain"]["real_time_templates"]
        out[f] = o
    out["value"] = max(v["real_time_templates"] for k, v in out.items() if k in forms)
    out["trials"] = {f: [dict((k, t.get(k)) for k in ("scale", "blocks", "p50_block_latency_ms",
                                                        "p99_block_latency_ms", "mean_active_templates"))
                         for t in res[f]["search"]] for f in forms}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="single", choices=["single", "multirate", "tc", "serve", "sweep", "ratesweep"])
    ap.add_argument("--serve-kind", default="multirate", choices=["single", "multirate"],
                    help="serving requests: multi-rate (configuration 4) or single-rate banks")
    ap.add_argument("--serve-forms", default="fp16",
                    help="serving: forms compared with the plain form (comma-separated)")
    ap.add_argument("--serve-blocks", type=int, default=16,
                    help="blocks per SLO-search run")
    ap.add_argument("--serve-confirm", type=int, default=210,
                    help="blocks of the confirmation run at the scale found (0: none)")
    ap.add_argument("--serve-trials", type=int, default=5)
    ap.add_argument("--serving", type=int, default=1,
                    help="default workload only: add the serving comparison (configuration-4 "
                         "requests, batched server, plain and --serve-forms) to the line")
    ap.add_argument("--serve-scale0", type=float, default=0.02)
    ap.add_argument("--form", default="", choices=["", "plain", "fp16", "bf16", "bf16x2"],
                    help="compute form of the headline number (default: plain; fp16 for tc)")
    ap.add_argument("--chosen", default="fp16", choices=["", "plain", "fp16", "bf16", "bf16x2"],
                    help="second form measured on the same workload and reported as 'chosen'")
    ap.add_argument("--config2", type=int, default=1,
                    help="default workload only: also measure the multi-rate bank (4000 templates, "
                         "7 rates, autotuned) with the plain form")
    ap.add_argument("--config3", default="fp16,bf16x2",
                    help="default workload only: also measure the 8000 x 256 two-stream "
                         "configuration with the plain form and these tensor-core forms "
                         "(comma-separated; empty: skip)")
    ap.add_argument("--resampler", default="default", choices=["default", "paper"],
                    help="multi-rate: 32/32-tap 60 dB pair (default) or the paper's "
                         "384-tap 100 dB decimator with the 32-tap interpolator")
    ap.add_argument("--carry", default="fp64", choices=["fp64", "df", "fp64chunk"],
                    help="tensor-core forms: carried-state arithmetic: FP64 per chunk batch "
                         "(default), double-float pairs on the FP32 pipe, or FP64 per chunk")
    ap.add_argument("--tune", type=int, default=None,
                    help="plain-form kernel variant: 1 = autotune at bank creation, 0 = default, "
                         "-(v+1) = variant v (default: autotune for multirate, else 0)")
    ap.add_argument("--templates", type=int, default=0,
                    help="template count (0 = the workload's full size); small cases for ncu")
    ap.add_argument("--seconds", type=int, default=0,
                    help="seconds of strain per step (0 = the workload's 16 s)")
    ap.add_argument("--ablation", default="adopted",
                    choices=["adopted", "shuffle", "smem", "atomics"],
                    help="recursion kernel's reduction (rebuilds libspiir with that "
                         "SPIIR_REDUCE_ABLATION): adopted, shuffle butterfly for every group, "
                         "shared-memory column sums for every group, cross-warp atomics")
    args = ap.parse_args()
    if args.ablation != "adopted" and args.impl == "ours":
        from paper_1702_02256_gb300 import build as lib_build
        os.environ["SPIIR_LIB"] = lib_build.build_ablation(args.ablation)
    if args.tune is None:
        args.tune = 1 if args.workload == "multirate" else 0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "ratesweep":
        return run_ratesweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
