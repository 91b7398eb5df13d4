"""Continuous-batching request loop for grid simulations.

Requests (parameters, seed, number of steps, arrival time) are admitted in
arrival order while the device-memory ledger has room for their footprint;
admitted networks stay resident on the GPU and every active network advances
together, one fused kernel per time step for the whole set (``run_batch``), in
chunks of at most ``chunk_steps``.  Requests that arrive while others run join
at the next chunk boundary; finished networks leave, their spikes and rate
counts are read into host memory and their device memory is released.

With ``overlap`` (the default) the host work around the GPU runs on a helper
thread while the next chunk runs: admitted networks are built there (each on a
CUDA stream of its own, so their construction kernels overlap the running
batch) and finished ones are released there; the ledger gives a network's
bytes back only once its memory is actually free.  In real-time mode a chunk
is shortened when the next request is due before a full chunk would end, so
that it waits at most about one short chunk before it joins.  Each network's
results are identical to running it alone (integer-exact accumulation,
counter-based randomness).
"""
from __future__ import annotations

import concurrent.futures as cf
import heapq
import threading
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


class _Ledger:
    """Device bytes held by networks that are built, being built, or not yet
    freed; released bytes come back from the helper thread."""

    def __init__(self):
        self._lock = threading.Lock()
        self.used = 0

    def take(self, n: int) -> None:
        with self._lock:
            self.used += n

    def give(self, n: int) -> None:
        with self._lock:
            self.used -= n


class _Inline:
    """Runs helper work on the calling thread (overlap off)."""

    def submit(self, fn, *args):
        f = cf.Future()
        try:
            f.set_result(fn(*args))
        except BaseException as e:   # noqa: BLE001 - handed to the waiting side
            f.set_exception(e)
        return f

    def shutdown(self, wait=True):
        pass


def _own_stream():
    """A CUDA stream for one served network (None without torch or a GPU)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.Stream()
    except ImportError:
        pass
    return None


@dataclass
class Server:
    memory_budget: int                      # device bytes available to resident networks
    chunk_steps: int = 1000                 # longest run between admission points
    min_chunk_steps: int = 100              # shortest chunk when an arrival is due (real time)
    max_active: int = 1024
    realtime: bool = True                   # arrivals on the wall clock; else on completed chunks
    keep_state: bool = False                # return each network's final neuron state with its result
    overlap: bool = True                    # build and release networks on a helper thread
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
        building: list[tuple[Request, int, cf.Future]] = []
        releasing: list[cf.Future] = []
        results: list[Result] = []
        ledger = _Ledger()
        helper = cf.ThreadPoolExecutor(max_workers=1) if self.overlap else _Inline()
        t_start = time.perf_counter()
        chunks = 0
        events = 0
        sec_per_step = None

        def now() -> float:
            return time.perf_counter() - t_start if self.realtime else chunks * 1.0

        def build(req: Request) -> Network:
            stream = _own_stream()
            net = Network(req.params, req.seed, stream=None if stream is None else stream.cuda_stream)
            net._served_stream = stream          # keeps the stream alive as long as the network
            return net

        def release(net: Network, nbytes: int) -> None:
            try:
                net.close()
            finally:
                ledger.give(nbytes)

        try:
            while self._queue or waiting or building or active:
                clock = now()
                while self._queue and self._queue[0][0] <= clock:
                    waiting.append(heapq.heappop(self._queue)[2])
                # admit in arrival order while memory and slots allow
                still = []
                for req in waiting:
                    need = footprint(req.params)
                    if need > self.memory_budget:
                        raise ValueError(f"request {req.rid} needs {need} bytes, more than the whole budget")
                    if (still or ledger.used + need > self.memory_budget
                            or len(active) + len(building) >= self.max_active):
                        still.append(req)
                        continue
                    ledger.take(need)
                    building.append((req, need, helper.submit(build, req)))
                waiting = still
                # built networks join the batch
                pending = []
                for req, need, fut in building:
                    if fut.done():
                        active.append(_Active(req, fut.result(), need, req.steps, now()))
                    else:
                        pending.append((req, need, fut))
                building = pending
                releasing = [f for f in releasing if not f.done()]
                if not active:
                    if building:
                        building[0][2].result()          # the oldest build; it joins on the next pass
                    elif waiting and releasing:
                        releasing[0].result()            # memory comes back as networks are freed
                    elif self._queue:
                        if self.realtime:
                            time.sleep(max(0.0, self._queue[0][0] - now()))
                        else:
                            chunks += 1
                    continue
                n = self.chunk_steps
                if self.realtime and self._queue and sec_per_step:
                    due = int((self._queue[0][0] - now()) / sec_per_step)
                    n = max(self.min_chunk_steps, min(self.chunk_steps, due))
                steps = [min(a.left, n) for a in active]
                t0 = time.perf_counter()
                run_batch([a.net for a in active], steps)
                sec_per_step = (time.perf_counter() - t0) / max(steps)
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
                    releasing.append(helper.submit(release, a.net, a.bytes))
        except BaseException:
            helper.shutdown(wait=True)
            for a in active:
                a.net.close()
            for _, _, fut in building:
                if fut.done() and fut.exception() is None:
                    fut.result().close()
            raise
        helper.shutdown(wait=True)
        for f in releasing:
            f.result()
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
