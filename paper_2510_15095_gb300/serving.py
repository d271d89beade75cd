"""Continuous-batching serving loop over many device-resident Hive tables.

Requests (an op range on one table; payload in device memory, or in pinned
host memory that the kernels read and write in place) arrive over time.  The server keeps a FIFO of arrived requests and, whenever fewer than
`depth` batches are in flight, coalesces the oldest admissible requests into
one multi-table batch (hive_multi_execute in asynchronous mode, replayed from
a captured CUDA graph) and queues it on its stream.  A request is admissible
when

* no earlier request of its table is still waiting (per-table FIFO order, so
  every request sees exactly the table state it would see served alone, in
  arrival order),
* its table has no other request in the batch being formed (the batch
  contract holds per request, not across requests), and
* the committed bucket memory of all tables, counting the growth this
  request may trigger (its inserts at the 0.9 load threshold), stays within
  the HBM budget.

Completion times come from CUDA events recorded after each batch on the
serving stream, relative to an event recorded at start, so latency =
completion - arrival needs no host polling precision.  The FIFO mode runs one
hive_execute per request instead, as the plain bulk-launch reference.

Host orchestration only: every op runs in the library's CUDA kernels.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import hive as H

SLOT_BYTES = 8.0 + 8.0 / 32  # a bucket slot plus its share of free mask and lock words


@dataclass
class Request:
    rid: int
    table: int
    arrival: float  # seconds after the run starts
    ops: object  # uint8 tensor: CUDA, or pinned host memory used in place
    keys: object  # int32 tensor, same memory as ops
    vals: object  # int32 tensor, same memory as ops
    n_insert: int
    vals_out: object = None
    status: object = None
    done_at: float = field(default=float("nan"))
    rejected: bool = False  # could never fit the HBM budget; not executed

    @property
    def n(self) -> int:
        return int(self.keys.numel())


class HiveServer:
    def __init__(self, tables, hbm_budget_bytes: float, max_batch_ops: int = 1 << 22,
                 max_batch_reqs: int = 256, depth: int = 2, use_graph: bool = True,
                 grow_num: int = 9, grow_den: int = 10, stream=None):
        import torch
        self.torch = torch
        self.tables = list(tables)
        self.budget = float(hbm_budget_bytes)
        self.max_ops = int(max_batch_ops)
        self.max_reqs = int(max_batch_reqs)
        self.depth = int(depth)
        self.grow = (grow_num, grow_den)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.multi = H.HiveMulti(self.tables, max_segments=self.max_reqs, max_ops=self.max_ops,
                                 use_graph=use_graph, asynchronous=True, stream=self.stream)
        # upper bounds of sizes and capacities, kept on the host between
        # batches and refreshed from the library before each batch is formed;
        # a table grows in steps of K bucket pairs, so a growth may overshoot
        # by K buckets
        self.size_ub = [t.size() for t in self.tables]
        self.cap_slots = [t.capacity() for t in self.tables]
        self.slack = [32 * int(t.config.resize_batch) for t in self.tables]

    def close(self):
        self.multi.close()

    # -- admission --------------------------------------------------------
    def _needed_slots(self, t: int, extra: int) -> int:
        g_num, g_den = self.grow
        need = (self.size_ub[t] + extra) * g_den // g_num + 1
        if need <= self.cap_slots[t]:
            return self.cap_slots[t]
        return need + self.slack[t]

    def _committed_bytes(self) -> float:
        return sum(self.cap_slots) * SLOT_BYTES

    def _sync_bounds(self):
        """Take the size bounds the library keeps (the size gathered after each
        table's newest completed batch plus the inserts queued since, so erases
        lower them again) and the tables' capacities (which include the growth
        planned for batches in flight)."""
        self.size_ub = self.multi.bounds()
        self.cap_slots = [t.capacity() for t in self.tables]

    def _form_batch(self, pending: deque, reqs):
        chosen, tables_in, blocked = [], set(), set()
        ops = 0
        committed = self._committed_bytes()
        keep = deque()
        while pending:
            rid = pending.popleft()
            r = reqs[rid]
            t = r.table
            if (t in tables_in or t in blocked or len(chosen) >= self.max_reqs
                    or ops + r.n > self.max_ops):
                blocked.add(t)
                keep.append(rid)
                continue
            need = self._needed_slots(t, r.n_insert)
            add = (need - self.cap_slots[t]) * SLOT_BYTES
            if committed + add > self.budget:
                blocked.add(t)
                keep.append(rid)
                continue
            committed += add
            chosen.append(rid)
            tables_in.add(t)
            ops += r.n
        pending.extend(keep)
        # restore arrival order of the kept requests
        if keep:
            tmp = sorted(pending)
            pending.clear()
            pending.extend(tmp)
        return chosen

    def _note_launch(self, chosen, reqs):
        """Host bookkeeping of a batch about to be queued: its tables' bounds
        rise by the batch's inserts and their capacities by the growth it may
        need, until the next _sync_bounds()."""
        for rid in chosen:
            r = reqs[rid]
            self.cap_slots[r.table] = self._needed_slots(r.table, r.n_insert)
            self.size_ub[r.table] += r.n_insert

    def _launch(self, chosen, reqs):
        segs = []
        for rid in chosen:
            r = reqs[rid]
            segs.append({"table": r.table, "ops": r.ops, "keys": r.keys, "vals": r.vals,
                         "vals_out": r.vals_out, "status": r.status, "n_insert": r.n_insert})
        self._note_launch(chosen, reqs)
        self.multi.execute(segs, stream=self.stream)
        ev = self.torch.cuda.Event(enable_timing=True)
        ev.record(self.stream)
        return ev

    # -- serving ----------------------------------------------------------
    def run(self, reqs, time_scale: float = 1.0):
        """Serve `reqs` (sorted by arrival).  Returns a summary dict; each
        request's done_at is filled in (seconds after start)."""
        torch = self.torch
        for r in reqs:
            # results go where the payload is: device memory, or pinned host
            # memory that the kernels write in place
            pin = not r.keys.is_cuda
            if r.vals_out is None:
                r.vals_out = torch.empty(r.n, dtype=torch.int32, device=r.keys.device,
                                         pin_memory=pin)
            if r.status is None:
                r.status = torch.empty(r.n, dtype=torch.uint8, device=r.keys.device,
                                       pin_memory=pin)
        start = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(self.stream)
        t0 = time.perf_counter()
        pending, inflight = deque(), deque()
        i, n_done, batches, batch_reqs = 0, 0, 0, []
        N = len(reqs)
        while n_done < N:
            now = (time.perf_counter() - t0) / time_scale
            while i < N and reqs[i].arrival <= now:
                pending.append(i)
                i += 1
            while inflight and inflight[0][0].query():
                ev, ids = inflight.popleft()
                done_at = start.elapsed_time(ev) / 1e3 / time_scale
                for rid in ids:
                    reqs[rid].done_at = done_at
                n_done += len(ids)
            if pending and len(inflight) < self.depth:
                self._sync_bounds()
                chosen = self._form_batch(pending, reqs)
                if chosen:
                    inflight.append((self._launch(chosen, reqs), chosen))
                    batches += 1
                    batch_reqs.append(len(chosen))
                    continue
                if not inflight:
                    # nothing runs and the oldest request still does not fit:
                    # it never will (capacity only grows), so reject it
                    rid = pending.popleft()
                    reqs[rid].rejected = True
                    n_done += 1
                    continue
            if not pending and not inflight and i < N:
                gap = (reqs[i].arrival - now) * time_scale
                if gap > 2e-4:
                    time.sleep(gap - 1e-4)
            else:
                time.sleep(2e-5)
        torch.cuda.synchronize()
        return self._summary(reqs, batches, batch_reqs)

    @staticmethod
    def _summary(reqs, batches, batch_reqs):
        served = [r for r in reqs if not r.rejected]
        lat = np.array([r.done_at - r.arrival for r in served]) if served else np.zeros(1)
        ops = sum(r.n for r in served)
        span = (max(r.done_at for r in served) - min(r.arrival for r in served)) if served else 1.0
        return {"requests": len(served), "rejected": len(reqs) - len(served), "ops": ops,
                "batches": batches,
                "mean_batch_requests": float(np.mean(batch_reqs)) if batch_reqs else 0.0,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "makespan_s": span,
                "gops": ops / span / 1e9}


def run_fifo(tables, reqs, stream=None, time_scale: float = 1.0):
    """Reference: one hive_execute per request, in arrival order, each started
    when it has arrived and the previous one has finished."""
    import torch
    stream = stream if stream is not None else torch.cuda.current_stream()
    for r in reqs:
        if r.vals_out is None:
            r.vals_out = torch.empty(r.n, dtype=torch.int32, device=r.keys.device)
        if r.status is None:
            r.status = torch.empty(r.n, dtype=torch.uint8, device=r.keys.device)
    start = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    t0 = time.perf_counter()
    for r in reqs:
        now = (time.perf_counter() - t0) / time_scale
        if r.arrival > now:
            time.sleep((r.arrival - now) * time_scale)
        vo, st = tables[r.table].execute(r.ops, r.keys, r.vals, stream=stream)
        r.vals_out.copy_(vo)
        r.status.copy_(st)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        ev.synchronize()
        r.done_at = start.elapsed_time(ev) / 1e3 / time_scale
    return HiveServer._summary(reqs, len(reqs), [1] * len(reqs))


def make_trace(torch, n_tables: int, n_requests: int, rate_per_s: float, seed: int,
               counts, max_log2_ops: int = 20, ins_frac=(2, 5), erase_frac=(1, 5),
               device="cuda"):
    """Poisson arrivals at `rate_per_s`, each request log-uniform in
    [1, 2^max_log2_ops] ops on a uniform random table, ops insert:erase:find =
    ins_frac : erase_frac : rest (default 40/20/40).  `counts[t]` is the number
    of keys table t was preloaded with (stream positions [0, count) of seed
    1000 + t); it is advanced as inserts are generated."""
    from . import workload as W
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    tables = rng.integers(0, n_tables, n_requests)
    sizes = np.exp(rng.uniform(0, max_log2_ops * np.log(2), n_requests)).astype(np.int64)
    sizes = np.maximum(sizes, 1)
    reqs = []
    for k in range(n_requests):
        t = int(tables[k])
        ops, keys, vals, counts[t], n_ins = W.mixed_step_t(
            torch, 1000 + t, counts[t], int(sizes[k]), device, ins_frac=ins_frac,
            erase_frac=erase_frac, salt=k)
        reqs.append(Request(k, t, float(arrivals[k]), ops, keys, vals, n_ins))
    return reqs
