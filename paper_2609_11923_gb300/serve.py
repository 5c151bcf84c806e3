"""Continuous-batching solve server over the batched CFR+ kernels.

Requests (game specs with arrival times) are compiled on arrival by worker
threads, admitted into a device memory pool by their footprint (cfr_plan)
whenever a slot and enough pool memory are free, and solved together: every
round is ONE batched launch that runs `check_every` iterations of every
active solve (one CTA per solve), followed by ONE batched exploitability
launch. Solves that reach `target * pot` exploitability (or `max_iters`)
retire, free their memory, and the next arrivals are admitted before the
next round, so work that arrives while others are on the GPU overlaps with
them. Requests of at least `big_edges` edges run as thread-block clusters of
`cluster` CTAs (a second batched launch on a side stream, concurrent with
the one-CTA launch of the rest), so one large subgame no longer holds every
round to the speed of a single SM. Whether a request is large depends only
on the request, so a solve's iterates do not depend on what else is in the
batch.
"""
from __future__ import annotations

import bisect
import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import cfr

ALIGN = 256


class DevicePool:
    """First-fit sub-allocator over one device tensor (256-byte blocks)."""

    def __init__(self, nbytes: int, device="cuda"):
        if device is None:  # bookkeeping only (host tests)
            self.buf, self.base = None, 0
        else:
            import torch

            self.buf = torch.empty(nbytes + ALIGN, dtype=torch.uint8, device=device)
            self.base = (self.buf.data_ptr() + ALIGN - 1) & ~(ALIGN - 1)
        self.size = nbytes - (nbytes % ALIGN)
        self.free = [(0, self.size)]  # sorted (offset, length)
        self.used = 0

    def alloc(self, n: int) -> Optional[int]:
        n = (n + ALIGN - 1) & ~(ALIGN - 1)
        for i, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, ln - n)
                self.used += n
                return off
        return None

    def release(self, off: int, n: int) -> None:
        n = (n + ALIGN - 1) & ~(ALIGN - 1)
        self.used -= n
        i = bisect.bisect_left(self.free, (off, 0))
        self.free.insert(i, (off, n))
        # coalesce with neighbours
        if i + 1 < len(self.free) and self.free[i][0] + self.free[i][1] == self.free[i + 1][0]:
            self.free[i] = (self.free[i][0], self.free[i][1] + self.free[i + 1][1])
            self.free.pop(i + 1)
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            self.free.pop(i)

    def ptr(self, off: int) -> int:
        return self.base + off


@dataclass
class Request:
    rid: int
    spec: object
    arrival: float = 0.0  # seconds after the start of serve()


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    iterations: int
    exploitability: float
    pot: float
    edges: int
    strategy: Optional[np.ndarray] = field(default=None, repr=False)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Active:
    req: Request
    h: int
    off: int
    nbytes: int
    admitted: float
    big: bool = False
    done: int = 0


class Server:
    def __init__(self, pool_bytes: int, max_active: int = 256, precision: int = cfr.P32, threads: int = 256,
                 lanes: int = 4, check_every: int = 50, max_iters: int = 5000, target: float = 1e-3,
                 compile_workers: int = 8, keep_strategies: bool = False, device="cuda",
                 big_edges: int = 200_000, cluster: int = 8, big_threads: int = 1024, big_lanes: int = 8):
        import torch

        self.torch = torch
        self.pool = DevicePool(pool_bytes, device)
        self.max_active = max_active
        self.opts = cfr.make_options(precision=precision, exec_form=cfr.EXEC_LEVELS)
        self.threads, self.lanes = threads, lanes
        self.big_edges, self.cluster = big_edges, cluster
        self.big_threads, self.big_lanes = big_threads, big_lanes
        self.check_every, self.max_iters, self.target = check_every, max_iters, target
        self.keep = keep_strategies
        self.table_bytes = cfr.cfr_batch_table_bytes(max_active)
        self.table = torch.empty(self.table_bytes + 16, dtype=torch.uint8, device=device)
        self.table_ptr = (self.table.data_ptr() + 15) & ~15
        self.table2 = torch.empty(self.table_bytes + 16, dtype=torch.uint8, device=device)
        self.table2_ptr = (self.table2.data_ptr() + 15) & ~15
        self.side = torch.cuda.Stream(device=device)
        self.workers = ThreadPoolExecutor(max_workers=compile_workers)
        self.rounds = 0

    def is_big(self, spec) -> bool:
        return self.cluster > 1 and int(spec.n_edges) >= self.big_edges

    def _stream(self) -> int:
        return int(self.torch.cuda.current_stream().cuda_stream)

    def _compile(self, spec):
        return cfr.cfr_compile(spec, self.opts)

    def bind(self, h: int):
        nbytes = cfr.cfr_plan(h)
        off = self.pool.alloc(nbytes)
        if off is None:
            return None
        cfr.cfr_bind(h, self.pool.ptr(off), nbytes, self._stream())
        return off, nbytes

    def serve(self, requests: List[Request]) -> List[Result]:
        s = self._stream()
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting: deque = deque()  # (request, future) in arrival order
        active: List[_Active] = []
        results: List[Result] = []
        t0 = time.perf_counter()
        while pending or waiting or active:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                waiting.append((r, self.workers.submit(self._compile, r.spec)))
            # admit in arrival order while a slot and pool memory are free
            while waiting and len(active) < self.max_active and waiting[0][1].done():
                r, fut = waiting[0]
                h = fut.result()
                got = self.bind(h)
                if got is None:
                    break  # memory full: wait for retirements
                waiting.popleft()
                active.append(_Active(r, h, got[0], got[1], time.perf_counter() - t0, self.is_big(r.spec)))
            if not active:
                nxt = pending[0].arrival if pending else now + 1e-3
                time.sleep(max(0.0, min(nxt - (time.perf_counter() - t0), 2e-3)))
                continue
            active.sort(key=lambda a: a.big)  # one-CTA solves first, clusters after
            hs = [a.h for a in active]
            iters = [min(self.check_every, self.max_iters - a.done) for a in active]
            nb = sum(1 for a in active if a.big)
            ns = len(active) - nb
            if nb:  # the large solves as clusters on the side stream, concurrently
                self.side.wait_stream(self.torch.cuda.current_stream())
                cfr.cfr_batch_iterate(hs[ns:], 0, self.table2_ptr, self.table_bytes, self.big_threads, self.big_lanes,
                                      int(self.side.cuda_stream), iters=iters[ns:], cluster=self.cluster)
            if ns:
                cfr.cfr_batch_iterate(hs[:ns], 0, self.table_ptr, self.table_bytes, self.threads, self.lanes, s,
                                      iters=iters[:ns])
            if nb:
                self.torch.cuda.current_stream().wait_stream(self.side)
            ex = cfr.cfr_batch_exploitability(hs, self.table_ptr, self.table_bytes, self.threads, self.lanes, s)
            self.rounds += 1
            keep = []
            t_now = time.perf_counter() - t0
            for a, n_it, row in zip(active, iters, ex):
                a.done += n_it
                pot = float(getattr(a.req.spec, "pot", 1.0))
                if row[0] <= self.target * pot or a.done >= self.max_iters:
                    strat = None
                    if self.keep:
                        strat = np.empty(cfr.cfr_get_counts(a.h)["n_slots"])
                        cfr.cfr_avg_strategy(a.h, strat, False, s)
                    results.append(Result(a.req.rid, a.req.arrival, a.admitted, t_now, a.done, float(row[0]), pot,
                                          int(a.req.spec.n_edges), strat))
                    self.pool.release(a.off, a.nbytes)
                    cfr.cfr_destroy(a.h)
                else:
                    keep.append(a)
            active = keep
        return results

    def close(self):
        self.workers.shutdown(wait=True)


def autotune_batch(specs, precision: int = cfr.P32, iters: int = 20, device="cuda"):
    """Pick (threads, lanes) of the batched kernel by timing a sample batch."""
    import torch

    opts = cfr.make_options(precision=precision, exec_form=cfr.EXEC_LEVELS)
    hs = [cfr.cfr_compile(sp, opts) for sp in specs]
    sizes = [cfr.cfr_plan(h) for h in hs]
    pool = DevicePool(sum(((n + ALIGN - 1) & ~(ALIGN - 1)) for n in sizes) + ALIGN, device)
    s = int(torch.cuda.current_stream().cuda_stream)
    for h, n in zip(hs, sizes):
        cfr.cfr_bind(h, pool.ptr(pool.alloc(n)), n, s)
    tb = cfr.cfr_batch_table_bytes(len(hs))
    table = torch.empty(tb + 16, dtype=torch.uint8, device=device)
    tp = (table.data_ptr() + 15) & ~15
    best, best_t = (256, 4), float("inf")
    timings = {}
    for threads in (256, 1024):
        for lanes in (2, 4, 8, 32):
            cfr.cfr_batch_iterate(hs, 2, tp, tb, threads, lanes, s)
            torch.cuda.synchronize()
            t = time.perf_counter()
            cfr.cfr_batch_iterate(hs, iters, tp, tb, threads, lanes, s)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            timings[(threads, lanes)] = dt
            if dt < best_t:
                best, best_t = (threads, lanes), dt
    for h in hs:
        cfr.cfr_destroy(h)
    return best, timings


def solve_alone(spec, check_every: int = 50, max_iters: int = 5000, target: float = 1e-3,
                precision: int = cfr.P32):
    """The per-instance baseline: one solver per game (its own arena, the
    single-game execution form chosen by size), the same check schedule."""
    s = cfr.Solver(spec, precision=precision, exec_form=cfr.EXEC_AUTO)
    done, e = 0, float("inf")
    pot = float(getattr(spec, "pot", 1.0))
    while done < max_iters:
        n = min(check_every, max_iters - done)
        s.iterate(n)
        done += n
        e = s.exploitability()
        if e <= target * pot:
            break
    s.close()
    return done, e
