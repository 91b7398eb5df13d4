"""Comparison of a GPU run with the oracle's run of the same network.

Spike rasters, rate counts, refractory counters and event counters are
integer results and must be identical.  V and c are binary32 results of the
same operation sequence on both sides; the bar is |a - b| <= 1e-6 * max(1, |b|)
(identical bits are expected: both sides round every operation once, with no
fused multiply-add)."""
import numpy as np

REL_TOL = 1e-6


def gpu_results(net) -> dict:
    """Everything the comparison reads from a network built by the library."""
    ts, ids = net.spikes()
    V, c, ref = net.state()
    return {"steps": ts, "ids": ids, "rates": net.rates(), "V": V, "c": c, "ref": ref, "stats": net.stats()}


def oracle_results(o) -> dict:
    ts, ids = o.raster()
    V, c, ref = o.state()
    return {"t": o.t, "steps": ts, "ids": ids, "rates": o.rates(), "V": V, "c": c, "ref": ref,
            "counters": o.counters()}


def assert_same(g: dict, o: dict, steps: int, what: str = "") -> None:
    """g: gpu_results(...) (or a served result in the same form); o: the
    oracle's results (oracle.simulate or oracle_results)."""
    assert len(g["steps"]) == len(o["steps"]), (what, len(g["steps"]), len(o["steps"]))
    assert np.array_equal(g["steps"], o["steps"]) and np.array_equal(g["ids"], o["ids"]), what
    assert np.array_equal(g["rates"], o["rates"]), what
    assert np.array_equal(g["ref"], o["ref"]), what
    for key in ("V", "c"):
        a, b = g[key], o[key]
        assert np.all(np.abs(a - b) <= REL_TOL * np.maximum(1.0, np.abs(b))), (what, key)
    s, c = g["stats"], o["counters"]
    assert s["spikes"] == c["spikes"] and s["ext_events"] == c["ext_events"], what
    assert s["rec_events"] == c["rec_events"] and s["t"] == steps, what
