"""Host logic of the serving loop (no GPU): admission by device-memory
footprint in arrival order, chunked stepping of every resident network,
retirement and latency bookkeeping, with fake networks in place of the
library."""
import numpy as np
import pytest

import paper_1902_08410_gb300.serve as serve


class FakeNet:
    live = 0
    peak = 0
    log = []

    def __init__(self, params, seed, stream=None):
        self.params, self.seed = params, seed
        self.N = params["n"]
        self.M = 3
        self.t = 0
        FakeNet.live += 1
        FakeNet.peak = max(FakeNet.peak, FakeNet.live)
        FakeNet.log.append(("admit", seed))

    def spikes(self):
        return np.arange(self.t, dtype=np.uint32), np.full(self.t, self.seed, np.uint32)

    def rates(self):
        return np.zeros((1, 1, 3), np.uint32)

    def stats(self):
        return {"spikes": self.t, "t": self.t}

    def close(self):
        FakeNet.live -= 1
        FakeNet.log.append(("free", self.seed))


def fake_run_batch(nets, steps):
    assert len(nets) == len(steps)
    for n, s in zip(nets, steps):
        assert s > 0
        n.t += s


@pytest.fixture()
def fakes(monkeypatch):
    FakeNet.live, FakeNet.peak, FakeNet.log = 0, 0, []
    monkeypatch.setattr(serve, "Network", FakeNet)
    monkeypatch.setattr(serve, "run_batch", fake_run_batch)
    monkeypatch.setattr(serve, "footprint", lambda p: p["bytes"])
    monkeypatch.setattr(serve, "_own_stream", lambda: None)
    return FakeNet


def test_admission_by_footprint_in_arrival_order(fakes):
    srv = serve.Server(memory_budget=100, chunk_steps=10, realtime=False)
    sizes = [60, 30, 50, 20, 40]        # bytes of each request
    steps = [25, 10, 40, 5, 15]
    for i, (b, st) in enumerate(zip(sizes, steps)):
        srv.submit({"n": 10, "bytes": b}, seed=i, steps=st, arrival_s=0.0)
    out = srv.run()
    res = out["results"]
    assert [r.rid for r in res] == list(range(5))
    for r, st in zip(res, steps):
        assert r.steps == st and r.stats["t"] == st          # every network advanced exactly its steps
        assert len(r.spike_steps) == st
    admits = [s for ev, s in fakes.log if ev == "admit"]
    assert admits == list(range(5))                           # first come, first admitted
    assert fakes.live == 0                                    # every network freed
    # the ledger never exceeds the budget: replay the admit/free log
    used, size = 0, dict(enumerate(sizes))
    for ev, s in fakes.log:
        used += size[s] if ev == "admit" else -size[s]
        assert used <= 100
    assert out["p50_latency_s"] <= out["p99_latency_s"]


def test_later_arrivals_join_between_chunks(fakes):
    # builds on the calling thread: join times are exact on the chunk clock
    srv = serve.Server(memory_budget=1000, chunk_steps=10, realtime=False, overlap=False)
    srv.submit({"n": 10, "bytes": 1}, seed=0, steps=50, arrival_s=0.0)
    srv.submit({"n": 10, "bytes": 1}, seed=1, steps=10, arrival_s=2.0)   # arrives after two chunks
    out = srv.run()
    r0, r1 = out["results"]
    assert r1.admitted_s >= 2.0 and r1.completed_s < r0.completed_s     # joined the running batch
    assert fakes.peak == 2


@pytest.mark.parametrize("overlap", [True, False])
def test_overlap_keeps_order_ledger_and_results(fakes, overlap):
    """With the helper thread (builds and releases off the main thread) and
    without it, admission stays in arrival order, the ledger never exceeds the
    budget and every request advances exactly its steps."""
    srv = serve.Server(memory_budget=70, chunk_steps=7, realtime=False, overlap=overlap)
    sizes = [30, 30, 30, 20, 50, 10]
    for i, b in enumerate(sizes):
        srv.submit({"n": 10, "bytes": b}, seed=i, steps=11 + 3 * i, arrival_s=float(i % 3))
    out = srv.run()
    assert [r.stats["t"] for r in out["results"]] == [11 + 3 * i for i in range(6)]
    arrival_order = sorted(range(6), key=lambda i: (i % 3, i))
    assert [s for ev, s in fakes.log if ev == "admit"] == arrival_order
    used = 0
    for ev, s in fakes.log:
        used += sizes[s] if ev == "admit" else -sizes[s]
        assert used <= 70
    assert fakes.live == 0


def test_request_larger_than_budget(fakes):
    srv = serve.Server(memory_budget=10, chunk_steps=10, realtime=False)
    srv.submit({"n": 10, "bytes": 11}, seed=0, steps=5)
    with pytest.raises(ValueError):
        srv.run()
