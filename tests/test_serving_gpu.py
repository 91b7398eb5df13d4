"""Serving: networks admitted by memory footprint, stepped together with
networks already on the GPU, retired when done.  Every request's raster, rate
counts, counters and final state must equal the oracle's run of the same
network, and those of the same network run alone through the library."""
import numpy as np
import pytest

import workloads as W
from parity import assert_same, gpu_results

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1902_08410_gb300 as snn
    snn.build()
    return snn


def test_served_results_equal_oracle_and_solo_runs(snn, oracle_mod):
    from paper_1902_08410_gb300.serve import Server
    specs = [  # (gx, gy, regime, format, seed, steps, arrival chunk)
        (2, 2, "SWA", W.REC_I16, 31, 900, 0), (1, 1, "AW", W.REC_F32, 32, 400, 0),
        (3, 2, "AW", W.REC_I16, 33, 1300, 1), (2, 3, "SWA", W.REC_F32, 34, 500, 2),
        (1, 2, "AW", W.REC_I16, 35, 700, 2), (3, 3, "SWA", W.REC_I16, 36, 600, 4),
        (2, 1, "AW", W.REC_F32, 37, 1000, 5), (1, 1, "SWA", W.REC_I16, 38, 350, 7),
    ]
    fps = [snn.footprint(W.base_params(gx, gy, 1.0, reg, record_format=fmt)) for gx, gy, reg, fmt, *_ in specs]
    budget = sum(sorted(fps)[-3:])        # at most about three networks resident at once
    srv = Server(memory_budget=budget, chunk_steps=200, realtime=False, keep_state=True)
    for gx, gy, reg, fmt, seed, steps, arr in specs:
        srv.submit(W.base_params(gx, gy, 1.0, reg, record_format=fmt), seed, steps, arrival_s=arr)
    out = srv.run()
    assert len(out["results"]) == len(specs)
    # continuous batching: some requests joined while others were on the device
    res = out["results"]
    assert any(a.admitted_s < b.admitted_s < a.completed_s for a in res for b in res)
    for r, (gx, gy, reg, fmt, seed, steps, arr) in zip(out["results"], specs):
        p = W.base_params(gx, gy, 1.0, reg, record_format=fmt)
        V, c, ref = r.state
        served = {"steps": r.spike_steps, "ids": r.spike_ids, "rates": r.rates, "V": V, "c": c, "ref": ref,
                  "stats": r.stats}
        assert_same(served, oracle_mod.simulate(p, seed, steps), steps, f"served request {r.rid}")
        solo = snn.Network(p, seed)
        solo.run(steps)
        alone = gpu_results(solo)
        solo.close()
        for k in ("steps", "ids", "rates", "V", "c", "ref"):
            assert np.array_equal(alone[k], served[k]), (r.rid, k)
        assert r.stats["t"] == steps and r.latency_s >= 0
    assert out["p99_latency_s"] >= out["p50_latency_s"] > 0


def test_request_larger_than_budget_is_rejected(snn):
    from paper_1902_08410_gb300.serve import Server
    p = W.base_params(2, 2, 1.0)
    srv = Server(memory_budget=snn.footprint(p) - 1, chunk_steps=100, realtime=False)
    srv.submit(p, 1, 100)
    with pytest.raises(ValueError):
        srv.run()
