"""Serving loop: estimator requests of mixed grid sizes and bin sets,
continuous batching on CUDA streams, admission by an HBM budget.

A request asks for B_l^m of one seeded synthetic field on an N_g grid, for
a run of k1 bins of that grid's default 30-bin edges and l <= l_max.  The
server keeps one plan per grid size resident on the device (30 bins, l <= 6:
binning is per bin and the moment axis is ordered by l, so a request's
answer is a slice of that plan's output).  Requests wait in arrival order;
whenever a stream is free, the oldest waiting request's grid size is served
with up to `max_batch` waiting requests of that size in one batched launch
(every stage runs once for all its fields), in a slot (field buffer +
workspace) taken from a pool bounded by the HBM budget.  Launches on
different streams overlap on the GPU; requests that arrive meanwhile join
the next batch of their size.

Launches of one plan run at the same time on different streams; the C ABI
allows that because each slot has its own workspace and output (an estimate
only reads the plan's tables), and each launch's wait status is read from its
own workspace, so a request is told of a failure in its own launch only.

`Scheduler` holds the decisions and nothing of the GPU (tested on the CPU);
`Server` runs them on the device.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import synth

# default serving mix: grid sizes, weights and box lengths (Mpc/h)
GRIDS = (64, 128, 256, 512)
WEIGHTS = (0.4, 0.3, 0.2, 0.1)
BOXES = {32: 500.0, 64: 1000.0, 128: 500.0, 256: 1000.0, 512: 2000.0}
N_K1, N_MU, L_MAX = 30, 10, 6          # resident plans: 30 k1 bins, (mu, t) step 0.05, l <= 6


@dataclasses.dataclass
class Request:
    rid: int
    t_arrive: float       # seconds from the start of the trace
    ng: int
    k1_lo: int            # first k1 bin of the run (of the grid's 30 default bins)
    n_k1: int             # bins in the run, 4..30
    l_max: int            # 2, 4 or 6
    seed: int

    def n_lm(self) -> int:
        return (self.l_max // 2 + 1) ** 2

    def n_bins(self) -> int:
        return self.n_k1 * N_MU * N_MU


def make_trace(n: int = 300, rate: float = 20.0, seed: int = 0, grids=GRIDS, weights=WEIGHTS) -> list[Request]:
    """A seeded Poisson trace: exponential gaps of mean 1/rate; N_g by the
    weights; a run of 4-30 consecutive k1 bins at a random offset; l_max in
    {2, 4, 6}; one field seed per request."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        ng = int(rng.choice(grids, p=np.asarray(weights) / np.sum(weights)))
        nk = int(rng.integers(4, N_K1 + 1))
        lo = int(rng.integers(0, N_K1 - nk + 1))
        out.append(Request(i, t, ng, lo, nk, int(rng.choice((2, 4, 6))), 10_000 + i))
    return out


@dataclasses.dataclass
class Slot:
    """Device buffers for one batched launch of one grid size."""
    ng: int
    bytes: int
    max_batch: int = 1
    busy: bool = False
    handle: object = None          # executor's buffers


class Scheduler:
    """Admission and batching decisions.

    max_batch[ng]: fields per launch; slot_bytes[ng]: HBM of one slot (field
    buffer + workspace + output for max_batch fields); budget: HBM the slots
    may take together; streams: launches in flight at once."""

    def __init__(self, max_batch: dict, slot_bytes: dict, budget: int, streams: int):
        self.max_batch = dict(max_batch)
        self.slot_bytes = dict(slot_bytes)
        self.budget = int(budget)
        self.streams = int(streams)
        self.waiting: collections.deque[Request] = collections.deque()
        self.slots: list[Slot] = []
        self.in_flight = 0
        for ng, b in self.slot_bytes.items():
            if b > self.budget:
                raise ValueError(f"one slot of N_g={ng} ({b} bytes) exceeds the HBM budget")

    def used(self) -> int:
        return sum(s.bytes for s in self.slots)

    def arrive(self, req: Request):
        self.waiting.append(req)

    def _slot_for(self, ng: int):
        for s in self.slots:
            if s.ng == ng and not s.busy:
                return s
        need = self.slot_bytes[ng]
        # free idle slots of other sizes (largest first) until the new one fits
        if self.used() + need > self.budget:
            for s in sorted((s for s in self.slots if not s.busy and s.ng != ng), key=lambda s: -s.bytes):
                self.slots.remove(s)
                if self.used() + need <= self.budget:
                    break
        if self.used() + need > self.budget:
            return None
        s = Slot(ng, need, self.max_batch[ng])
        self.slots.append(s)
        return s

    def next_launch(self):
        """(slot, requests) to launch now, or None.  The oldest waiting
        request decides the grid size; later requests of that size join it
        (in arrival order) up to max_batch.  A size that cannot get a slot
        waits: it is not overtaken, so no request starves."""
        if not self.waiting or self.in_flight >= self.streams:
            return None
        ng = self.waiting[0].ng
        slot = self._slot_for(ng)
        if slot is None:
            return None
        batch = []
        for r in list(self.waiting):
            if r.ng == ng:
                batch.append(r)
                if len(batch) == self.max_batch[ng]:
                    break
        for r in batch:
            self.waiting.remove(r)
        slot.busy = True
        self.in_flight += 1
        return slot, batch

    def done(self, slot: Slot):
        slot.busy = False
        self.in_flight -= 1


class Server:
    """Runs a trace on the GPU with resident plans, a stream pool and the
    scheduler above; records each request's completion time and result."""

    def __init__(self, grids=GRIDS, precision: str = "mixed_tc", max_batch=None, budget_gb: float = 160.0,
                 streams: int = 4, device="cuda"):
        import torch

        from . import api
        self.torch, self.api = torch, api
        self.device = torch.device(device)
        self.precision = precision
        self.grids = tuple(grids)
        mb = max_batch or {32: 16, 64: 16, 128: 8, 256: 4, 512: 1}
        self.max_batch = {ng: mb[ng] for ng in self.grids}
        self.plans = {ng: api.Plan(ng, BOXES[ng], synth.default_k1_edges(ng, BOXES[ng], N_K1), N_MU, N_MU, L_MAX,
                                   precision=precision, max_batch=self.max_batch[ng]) for ng in self.grids}
        fsize = 8 if precision == "fp64" else 4
        slot_bytes = {ng: self.plans[ng].workspace_bytes(self.max_batch[ng]) + self.max_batch[ng] * ng ** 3 * fsize
                      + self.max_batch[ng] * int(np.prod(self.plans[ng].out_shape(1))) * 8 for ng in self.grids}
        self.sched = Scheduler(self.max_batch, slot_bytes, int(budget_gb * 2 ** 30), streams)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(streams)]

    def _buffers(self, slot: Slot):
        torch = self.torch
        if slot.handle is None:
            ng, mb = slot.ng, slot.max_batch
            p = self.plans[ng]
            dt = torch.float64 if self.precision == "fp64" else torch.float32
            slot.handle = {"field": torch.empty((mb, ng, ng, ng), dtype=dt, device=self.device),
                           "ws": p.workspace(mb, device=self.device),
                           "out": torch.empty(p.out_shape(mb), dtype=torch.float64, device=self.device)}
        return slot.handle

    def _launch(self, slot: Slot, batch: list, stream):
        torch = self.torch
        buf = self._buffers(slot)
        p = self.plans[slot.ng]
        k = len(batch)
        with torch.cuda.stream(stream):
            for i, r in enumerate(batch):
                buf["field"][i].copy_(synth.make_field_torch(r.ng, BOXES[r.ng], r.seed, device=self.device))
            out = buf["out"][:k]
            p.estimate(buf["field"][:k], buf["ws"], out=out, stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        return ev

    def answer(self, r: Request, out_row):
        """The request's slice of its plan's output [n_k1][n_mu][n_t][n_lm]."""
        return out_row[r.k1_lo:r.k1_lo + r.n_k1, :, :, :r.n_lm()]

    def run(self, trace: list[Request], one_by_one: bool = False, keep_results: bool = False):
        """Serve the trace in real time (arrival times from its start).
        one_by_one: a single stream, one request per launch, no overlap (the
        plain single-job form).  Returns per-request latencies (s), the
        makespan (s), and the results when asked.  self.status[rid] is the
        status code of the launch that served request rid (0: success)."""
        torch = self.torch
        sched = self.sched
        if one_by_one:
            sched = Scheduler({ng: 1 for ng in self.grids}, self.sched.slot_bytes, self.sched.budget, 1)
        lat, res = {}, {}
        self.status = {}
        self.log = []           # (N_g, fields) of every launch
        pending = []            # (event, slot, batch, stream index)
        free_streams = list(range(len(self.streams) if not one_by_one else 1))
        i = 0
        t0 = time.perf_counter()
        while i < len(trace) or sched.waiting or pending:
            now = time.perf_counter() - t0
            while i < len(trace) and trace[i].t_arrive <= now:
                sched.arrive(trace[i])
                i += 1
            still = []
            for ev, slot, batch, si in pending:
                if ev.query():
                    t_done = time.perf_counter() - t0
                    out = slot.handle["out"]
                    st = self.plans[slot.ng].workspace_status(slot.handle["ws"], len(batch), self.streams[si])
                    for j, r in enumerate(batch):
                        lat[r.rid] = t_done - r.t_arrive
                        self.status[r.rid] = st
                        if keep_results:
                            res[r.rid] = self.answer(r, out[j]).cpu().numpy()
                    sched.done(slot)
                    free_streams.append(si)
                else:
                    still.append((ev, slot, batch, si))
            pending = still
            launched = False
            while free_streams:
                nxt = sched.next_launch()
                if nxt is None:
                    break
                slot, batch = nxt
                si = free_streams.pop()
                self.log.append((slot.ng, len(batch)))
                ev = self._launch(slot, batch, self.streams[si])
                pending.append((ev, slot, batch, si))
                launched = True
            if not launched:
                time.sleep(2e-4)
        makespan = time.perf_counter() - t0
        torch.cuda.synchronize(self.device)
        return lat, makespan, res

    def close(self):
        for p in self.plans.values():
            p.close()
        self.plans = {}


def summary(trace: list[Request], lat: dict, makespan: float) -> dict:
    """configs/s (output bins of all requests / makespan) and latency percentiles."""
    v = np.array([lat[r.rid] for r in trace])
    bins = sum(r.n_bins() for r in trace)
    return {"requests": len(trace), "configs": int(bins), "makespan_s": makespan, "configs_per_s": bins / makespan,
            "p50_s": float(np.percentile(v, 50)), "p99_s": float(np.percentile(v, 99)), "max_s": float(v.max())}
