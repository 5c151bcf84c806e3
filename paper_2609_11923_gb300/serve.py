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

Admission (``admit``): requests are taken in arrival order. A request whose
footprint exceeds the whole pool can never be admitted and is answered at
once with a ``rejected`` result. When the request at the head of the queue
does not fit the free memory yet, later requests that fit are admitted
around it (backfill), but only for ``hol_rounds`` rounds: after that nothing
passes the head until it fits, so a large request cannot starve behind a
stream of small ones. ``cancel(rid)`` (thread-safe) drops a request that is
still queued, or retires an active solve at the next round boundary, when
none of its kernels is in flight; its result carries the iterations done.
A spec the compiler refuses is answered with an ``error`` result.
"""
from __future__ import annotations

import bisect
import threading
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
    # "solved" (reached target * pot), "capped" (max_iters first), "rejected"
    # (footprint larger than the pool), "cancelled" or "error" (compile failed)
    status: str = "solved"
    message: str = ""

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def admit(queue, n_free_slots: int, pool: DevicePool, footprint, head=(None, 0), hol_rounds: int = 8, key=id):
    """One admission pass (host logic only). queue: entries in arrival order
    whose compile has finished; footprint(entry) gives its device bytes.
    Entries larger than the whole pool are rejected. The others are admitted
    first-fit while slots last; once one does not fit (the blocked head),
    later entries are still admitted around it unless that same head has
    already waited hol_rounds passes. head = (key of the blocked head, passes
    it has waited) from the previous pass. Returns (admitted [(entry, offset,
    nbytes)], rejected [(entry, reason)], head for the next pass)."""
    admitted, rejected = [], []
    blocked = None
    for ent in queue:
        nbytes = int(footprint(ent))
        if nbytes > pool.size:
            rejected.append((ent, "footprint %d bytes exceeds the pool's %d bytes" % (nbytes, pool.size)))
            continue
        if len(admitted) >= n_free_slots:
            break
        if blocked is not None and head[0] == key(blocked) and head[1] >= hol_rounds:
            break  # the head has waited long enough: nothing passes it
        off = pool.alloc(nbytes)
        if off is None:
            if blocked is None:
                blocked = ent
            continue
        admitted.append((ent, off, nbytes))
    if blocked is None:
        return admitted, rejected, (None, 0)
    k = key(blocked)
    return admitted, rejected, (k, head[1] + 1 if head[0] == k else 1)


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
                 big_edges: int = 200_000, cluster: int = 8, big_threads: int = 1024, big_lanes: int = 8,
                 hol_rounds: int = 8, on_round=None):
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
        self.hol_rounds = hol_rounds
        self.on_round = on_round  # called after every round with the active request ids
        self._cancel_lock = threading.Lock()
        self._cancelled = set()

    def cancel(self, rid) -> None:
        """Cancels request rid (any thread): dropped if still queued, retired
        at the next round boundary if active."""
        with self._cancel_lock:
            self._cancelled.add(rid)

    def _take_cancelled(self):
        with self._cancel_lock:
            out, self._cancelled = self._cancelled, set()
        return out

    def is_big(self, spec) -> bool:
        return self.cluster > 1 and int(spec.n_edges) >= self.big_edges

    def _stream(self) -> int:
        return int(self.torch.cuda.current_stream().cuda_stream)

    def _compile(self, spec):
        return cfr.cfr_compile(spec, self.opts)

    def _compile_or_error(self, spec):
        try:
            return self._compile(spec)
        except cfr.CfrError as e:
            return e

    def serve(self, requests: List[Request]) -> List[Result]:
        s = self._stream()
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting: List = []  # (request, future) in arrival order
        active: List[_Active] = []
        results: List[Result] = []
        head = (None, 0)  # the blocked head of the queue and the passes it has waited
        t0 = time.perf_counter()

        def answer(r, status, msg="", h=None):
            t = time.perf_counter() - t0
            results.append(Result(r.rid, r.arrival, t, t, 0, float("nan"), float(getattr(r.spec, "pot", 1.0)),
                                  int(r.spec.n_edges), None, status, msg))
            if h is not None:
                cfr.cfr_destroy(h)

        while pending or waiting or active:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                waiting.append((r, self.workers.submit(self._compile_or_error, r.spec)))
            cancelled = self._take_cancelled()
            if cancelled:  # queued requests leave now; active ones at this round boundary
                for r in [r for r in pending if r.rid in cancelled]:
                    answer(r, "cancelled")
                pending = deque(r for r in pending if r.rid not in cancelled)
                keep_w = []
                for r, fut in waiting:
                    if r.rid in cancelled:
                        h = fut.result()
                        answer(r, "cancelled", h=h if not isinstance(h, Exception) else None)
                    else:
                        keep_w.append((r, fut))
                waiting = keep_w
                keep_a = []
                for a in active:
                    if a.req.rid in cancelled:
                        self._retire(a, results, time.perf_counter() - t0, float("nan"), "cancelled", s)
                    else:
                        keep_a.append(a)
                active = keep_a
            # compile failures are answered; the rest is admitted in arrival order
            ready, errored = [], set()
            for r, fut in waiting:
                if not fut.done():
                    break  # keep arrival order: later compiles wait for earlier ones
                h = fut.result()
                if isinstance(h, Exception):
                    answer(r, "error", str(h))
                    errored.add(id(r))
                    continue
                ready.append((r, fut, h))
            if errored:
                waiting = [(r, fut) for r, fut in waiting if id(r) not in errored]
            if ready:
                adm, rej, head = admit(ready, self.max_active - len(active), self.pool,
                                       lambda e: cfr.cfr_plan(e[2]), head, self.hol_rounds, key=lambda e: e[0].rid)
                gone = set()
                for (r, fut, h), why in rej:
                    answer(r, "rejected", why, h)
                    gone.add(id(r))
                for (r, fut, h), off, nbytes in adm:
                    cfr.cfr_bind(h, self.pool.ptr(off), nbytes, s)
                    active.append(_Active(r, h, off, nbytes, time.perf_counter() - t0, self.is_big(r.spec)))
                    gone.add(id(r))
                waiting = [(r, fut) for r, fut in waiting if id(r) not in gone]
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
                if row[0] <= self.target * pot:
                    self._retire(a, results, t_now, float(row[0]), "solved", s)
                elif a.done >= self.max_iters:
                    self._retire(a, results, t_now, float(row[0]), "capped", s)
                else:
                    keep.append(a)
            active = keep
            if self.on_round is not None:
                self.on_round(self, [a.req.rid for a in active])
        return results

    def _retire(self, a: _Active, results: List[Result], t_now: float, expl: float, status: str, s: int) -> None:
        """Result of an active solve, then its memory back to the pool (no
        kernel of it is in flight between rounds)."""
        pot = float(getattr(a.req.spec, "pot", 1.0))
        strat = None
        if self.keep:
            strat = np.empty(cfr.cfr_get_counts(a.h)["n_slots"])
            cfr.cfr_avg_strategy(a.h, strat, False, s)
        results.append(Result(a.req.rid, a.req.arrival, a.admitted, t_now, a.done, expl, pot,
                              int(a.req.spec.n_edges), strat, status))
        self.pool.release(a.off, a.nbytes)
        cfr.cfr_destroy(a.h)

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
