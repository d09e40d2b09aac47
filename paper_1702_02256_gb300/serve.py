"""Streaming serving loop for SPIIR template banks (continuous batching).

Detector strain arrives in blocks (1 s at 4096 Hz by default) on several
streams at once. Template-bank requests of uneven sizes arrive over time and
stay for a number of blocks. The server

* admits a request when its device footprint (spiir_bank_footprint, computed
  on the host) fits the HBM budget next to the requests already resident;
  requests that do not fit wait in arrival order and are admitted as soon as
  retiring requests free enough memory;
* keeps every admitted bank, its filter state and its strain history resident
  on the device between blocks;
* pushes each block of all streams to every active request: BatchedServer
  makes the requests members of one device-side server, so a block is one
  batched push for all of them (continuous batching); Server keeps a bank per
  request, each on its own CUDA stream (the unbatched baseline);
* records, per request and block, the device time from the push to the SNR
  being in the output buffer (CUDA events on the request's stream), and per
  block the time until every active request is done.

All filtering runs in libspiir's kernels; this module schedules and measures.
"""
from __future__ import annotations

import collections
import dataclasses
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    bank: object            # inputs.Bank
    arrival_block: int      # first block the request may take part in
    lifetime: int           # blocks it stays for once admitted
    keep_snr: bool = False  # keep the SNR of every block (for tests)


@dataclasses.dataclass
class Active:
    req: Request
    handle: object          # device bank (spiir.Bank) or a test double
    footprint: int
    admitted_block: int
    blocks_done: int = 0
    stream: object = None
    out: object = None
    snr: list = dataclasses.field(default_factory=list)


class Server:
    """Admission, residency and per-block scheduling of template banks.

    make_bank(request) -> device bank; footprint(request) -> bytes. Both are
    injectable so that the scheduling can be exercised without a GPU."""

    def __init__(self, hbm_budget: int, n_streams: int, block_len: int,
                 make_bank: Callable, footprint: Callable, use_cuda: bool = True):
        self.budget = int(hbm_budget)
        self.n_streams = n_streams
        self.block_len = block_len
        self.make_bank = make_bank
        self.footprint = footprint
        self.use_cuda = use_cuda
        self.pending: collections.deque = collections.deque()
        self.active: List[Active] = []
        self.used = 0
        self.block = 0
        self.log: List[dict] = []
        self.rejected: List[int] = []
        self.finished: Dict[int, Active] = {}

    # -- admission --------------------------------------------------------
    def submit(self, req: Request):
        fp = int(self.footprint(req))
        if fp < 0 or fp > self.budget:
            self.rejected.append(req.rid)      # can never fit
            return False
        self.pending.append((req, fp))
        return True

    def _admit(self):
        admitted = []
        while self.pending:
            req, fp = self.pending[0]
            if req.arrival_block > self.block or self.used + fp > self.budget:
                break                           # arrival order: no overtaking
            self.pending.popleft()
            a = Active(req=req, handle=self.make_bank(req), footprint=fp,
                       admitted_block=self.block)
            if self.use_cuda:
                import torch
                a.stream = torch.cuda.Stream()
                a.out = torch.empty((self.n_streams, req.bank.n_templates, self.block_len),
                                    dtype=torch.complex64, device="cuda")
            self.active.append(a)
            self.used += fp
            admitted.append(req.rid)
        return admitted

    def _retire(self):
        keep = []
        for a in self.active:
            if a.blocks_done >= a.req.lifetime:
                self.used -= a.footprint
                close = getattr(a.handle, "close", None)
                if close:
                    close()
                a.handle = None
                self.finished[a.req.rid] = a
            else:
                keep.append(a)
        self.active = keep

    # -- one block --------------------------------------------------------
    def step(self, x_block) -> dict:
        """Process one block (x_block: CUDA tensor [n_streams, block_len])."""
        admitted = self._admit()
        rec = {"block": self.block, "admitted": admitted, "active": [a.req.rid for a in self.active],
               "templates": int(sum(a.req.bank.n_templates for a in self.active)),
               "used_bytes": self.used, "pending": len(self.pending)}
        if self.use_cuda and self.active:
            import torch
            main = torch.cuda.current_stream()
            ev_x = torch.cuda.Event(enable_timing=True)
            ev_x.record(main)                       # the block is on the device
            events = []
            for a in self.active:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(a.stream):
                    a.stream.wait_event(ev_x)
                    e0.record(a.stream)
                    a.handle.push(x_block, stream_id=-1, stream=a.stream)
                    a.handle.read(self.block_len, stream_id=-1, out=a.out, stream=a.stream)
                    e1.record(a.stream)
                events.append((a, e0, e1))
            lat = []
            for a, e0, e1 in events:
                e1.synchronize()
                lat.append(e0.elapsed_time(e1))
                if a.req.keep_snr:
                    a.snr.append(a.out.cpu().numpy().copy())
            # block latency: from the block being on the device to the last
            # request's SNR being ready
            block_ms = max(ev_x.elapsed_time(e1) for _, _, e1 in events) if events else 0.0
            rec["latency_ms"] = lat
            rec["block_ms"] = block_ms
        elif not self.use_cuda:
            for a in self.active:
                a.handle.push(x_block)
        for a in self.active:
            a.blocks_done += 1
        self.block += 1
        self._retire()
        self.log.append(rec)
        return rec

    def drain(self):
        for a in self.active:
            close = getattr(a.handle, "close", None)
            if close:
                close()
        self.active = []


class BatchedServer(Server):
    """Continuous batching on one libspiir server (spiir_server_t).

    Same admission and retirement as Server (HBM budget, arrival order, no
    overtaking), but every admitted request is a member of one device-side
    server: each block is a single push that filters all of them together
    (one shared strain update and decimation, one recursion launch over every
    member's work items, one upsample-and-add launch, replayed from a CUDA
    graph while the membership is unchanged), followed by one device copy of
    each member's SNR. Requests join and leave between blocks; their filter
    states stay on the device meanwhile.

    engine: the device server (spiir.Server) or a test double with add,
    remove, push, read and member_footprint."""

    def __init__(self, hbm_budget: int, n_streams: int, block_len: int, engine,
                 use_cuda: bool = True):
        self.engine = engine
        super().__init__(hbm_budget, n_streams, block_len, make_bank=lambda r: engine.add(r.bank),
                         footprint=lambda r: engine.member_footprint(r.bank), use_cuda=use_cuda)

    def _admit(self):
        admitted = []
        while self.pending:
            req, fp = self.pending[0]
            if req.arrival_block > self.block or self.used + fp > self.budget:
                break
            self.pending.popleft()
            a = Active(req=req, handle=self.engine.add(req.bank), footprint=fp,
                       admitted_block=self.block)
            if self.use_cuda:
                import torch
                a.out = torch.empty((self.n_streams, req.bank.n_templates, self.block_len),
                                    dtype=torch.complex64, device="cuda")
            self.active.append(a)
            self.used += fp
            admitted.append(req.rid)
        return admitted

    def _retire(self):
        keep = []
        for a in self.active:
            if a.blocks_done >= a.req.lifetime:
                self.used -= a.footprint
                self.engine.remove(a.handle)
                self.finished[a.req.rid] = a
            else:
                keep.append(a)
        self.active = keep

    def step(self, x_block) -> dict:
        admitted = self._admit()
        rec = {"block": self.block, "admitted": admitted, "active": [a.req.rid for a in self.active],
               "templates": int(sum(a.req.bank.n_templates for a in self.active)),
               "used_bytes": self.used, "pending": len(self.pending)}
        # every block enters the server's strain history, with or without
        # requests, so that a request joining later reads the continuous stream
        if self.use_cuda:
            import time
            import torch
            main = torch.cuda.current_stream()
            # membership changes (placement, uploads, work lists, graph) are
            # made between blocks, before the block arrives
            t0 = time.perf_counter()
            prep = getattr(self.engine, "prepare", None)
            if prep:
                prep()
            rec["prepare_ms"] = 1e3 * (time.perf_counter() - t0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(main)                          # the block is on the device
            self.engine.push(x_block)
            for a in self.active:
                self.engine.read(a.handle, out=a.out)
            e1.record(main)
            e1.synchronize()
            if self.active:
                ms = e0.elapsed_time(e1)
                rec["latency_ms"] = [ms] * len(self.active)
                rec["block_ms"] = ms
            for a in self.active:
                if a.req.keep_snr:
                    a.snr.append(a.out.cpu().numpy().copy())
        elif self.active:
            self.engine.push(x_block)
            for a in self.active:
                out = self.engine.read(a.handle)
                if a.req.keep_snr:
                    a.snr.append(out)
        for a in self.active:
            a.blocks_done += 1
        self.block += 1
        self._retire()
        self.log.append(rec)
        return rec

    def drain(self):
        for a in self.active:
            self.engine.remove(a.handle)
        self.active = []


def device_bank_factory(form: str = "plain", block_len: int = 4096, n_streams: int = 3,
                        chunk_len: int = 256):
    """make_bank / footprint callables backed by libspiir."""
    from . import spiir

    def kw(req):
        bank = req.bank
        d = dict(n_streams=n_streams, block_len=block_len, max_push_blocks=1)
        if form != "plain":
            d.update(mode=form, chunk_len=chunk_len)
        return bank, d

    def make(req):
        bank, d = kw(req)
        return spiir.Bank(bank, **d)

    def fp(req):
        bank, d = kw(req)
        return spiir.footprint(bank, **d)

    return make, fp


def summarize(server: Server, warm_blocks: int = 2) -> dict:
    """Latency percentiles and sustained load over the logged blocks."""
    lat, blk, tmpl = [], [], []
    for rec in server.log[warm_blocks:]:
        if "latency_ms" in rec:
            lat.extend(rec["latency_ms"])
            blk.append(rec["block_ms"])
            tmpl.append(rec["templates"])
    if not blk:
        return {"blocks": 0}
    return {
        "blocks": len(blk),
        "p50_request_latency_ms": float(np.percentile(lat, 50)),
        "p99_request_latency_ms": float(np.percentile(lat, 99)),
        "p50_block_latency_ms": float(np.percentile(blk, 50)),
        "p99_block_latency_ms": float(np.percentile(blk, 99)),
        "mean_active_templates": float(np.mean(tmpl)),
        "max_active_templates": int(np.max(tmpl)),
        "rejected": len(server.rejected),
    }
