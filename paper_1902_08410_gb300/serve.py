"""Continuous-batching request loop for grid simulations.

Requests (parameters, seed, number of steps, arrival time) are admitted while
the device-memory ledger has room for their footprint; admitted networks stay
resident on the GPU and every active network advances together, one fused
kernel per time step for the whole set (``run_batch``), in chunks of
``chunk_steps``.  Requests that arrive while others run join at the next chunk
boundary; finished networks leave, their spikes and rate counts are copied to
the host and their memory is released.  Each network's results are identical
to running it alone (integer-exact accumulation, counter-based randomness).
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field

import numpy as np

from . import Network, footprint, run_batch

EQUIV_PER_SPIKE_EXTRA = 400   # external synapses per neuron counted per spike (Table S1: N_ext)


@dataclass
class Request:
    rid: int
    params: dict
    seed: int
    steps: int
    arrival_s: float = 0.0


@dataclass
class Result:
    rid: int
    arrival_s: float
    admitted_s: float
    completed_s: float
    steps: int
    spike_steps: np.ndarray
    spike_ids: np.ndarray
    rates: np.ndarray
    stats: dict
    state: tuple | None = None          # final (V, c, refractory steps) when the server keeps states

    @property
    def latency_s(self) -> float:
        return self.completed_s - self.arrival_s


@dataclass
class _Active:
    req: Request
    net: Network
    bytes: int
    left: int
    admitted_s: float


@dataclass
class Server:
    memory_budget: int                      # device bytes available to resident networks
    chunk_steps: int = 1000                 # steps between admission points
    max_active: int = 1024
    realtime: bool = True                   # arrivals on the wall clock; else on completed chunks
    keep_state: bool = False                # return each network's final neuron state with its result
    _queue: list = field(default_factory=list)
    _next_rid: int = 0

    def submit(self, params: dict, seed: int, steps: int, arrival_s: float = 0.0) -> int:
        rid = self._next_rid
        self._next_rid += 1
        heapq.heappush(self._queue, (arrival_s, rid, Request(rid, params, seed, int(steps), arrival_s)))
        return rid

    def run(self) -> dict:
        """Serve every submitted request; returns results and summary statistics."""
        active: list[_Active] = []
        waiting: list[Request] = []
        results: list[Result] = []
        ledger = 0
        t_start = time.perf_counter()
        chunks = 0
        events = 0

        def now() -> float:
            return time.perf_counter() - t_start if self.realtime else chunks * 1.0

        while self._queue or waiting or active:
            clock = now()
            while self._queue and self._queue[0][0] <= clock:
                waiting.append(heapq.heappop(self._queue)[2])
            # admit in arrival order while memory and slots allow
            still = []
            for req in waiting:
                need = footprint(req.params)
                if need > self.memory_budget:
                    raise ValueError(f"request {req.rid} needs {need} bytes, more than the whole budget")
                if ledger + need <= self.memory_budget and len(active) < self.max_active and not still:
                    net = Network(req.params, req.seed)
                    ledger += need
                    active.append(_Active(req, net, need, req.steps, now()))
                else:
                    still.append(req)
            waiting = still
            if not active:
                if self._queue:
                    if self.realtime:
                        time.sleep(max(0.0, self._queue[0][0] - now()))
                    else:
                        chunks += 1
                continue
            steps = [min(a.left, self.chunk_steps) for a in active]
            run_batch([a.net for a in active], steps)
            chunks += 1
            for a, s in zip(active, steps):
                a.left -= s
            done = [a for a in active if a.left == 0]
            active = [a for a in active if a.left > 0]
            t_done = now()
            for a in done:
                st, ids = a.net.spikes()
                rates = a.net.rates()
                stats = a.net.stats()
                state = a.net.state() if self.keep_state else None
                events += stats["spikes"] * (a.net.M + EQUIV_PER_SPIKE_EXTRA)
                results.append(Result(a.req.rid, a.req.arrival_s, a.admitted_s, t_done, a.req.steps, st, ids,
                                      rates, stats, state))
                a.net.close()
                ledger -= a.bytes
        wall = time.perf_counter() - t_start
        lat = np.array([r.latency_s for r in results]) if results else np.zeros(1)
        results.sort(key=lambda r: r.rid)
        return {
            "results": results,
            "wall_s": wall,
            "events": events,
            "events_per_s": events / wall if wall > 0 else 0.0,
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "chunks": chunks,
        }
