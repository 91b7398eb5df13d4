"""The seeded synthetic workloads follow their stated recipes (sizes, value
ranges and distributions), are reproducible, and carry no method arithmetic
beyond parameter sets."""
import math

import numpy as np
import pytest

import workloads as W


def test_named_grids():
    for reg in ("SWA", "AW"):
        w = W.grid_24x24(reg)
        p = w["params"]
        assert (p["gx"], p["gy"], p["lambda"], p["record_format"]) == (24, 24, 1.0, W.REC_F32)
        assert W.n_neurons(p) == 720_000 and W.n_neurons(p) * p["out_degree"] == 810_000_000
        assert w["steps"] == 100_000 and w["seed"] == 1
    for lam in (0.4, 1.0, 2.0):
        for fmt in (W.REC_F32, W.REC_I16):
            p = W.grid_64x64("SWA", lam, fmt)["params"]
            assert W.n_neurons(p) * p["out_degree"] == 5_760_000_000 and p["record_format"] == fmt
    p = W.grid_4x4_swa()["params"]
    assert W.n_neurons(p) == 20_000 and p["lambda"] == 0.4 and p["p_local"] == 0.8


def test_batched_sweep_recipe():
    a, b = W.batched_sweep(), W.batched_sweep()
    assert [x["params"] for x in a] == [x["params"] for x in b]          # reproducible
    assert len(a) == 256 and [x["seed"] for x in a] == list(range(1000, 1256))
    sides = np.array([x["params"]["gx"] for x in a])
    assert sides.min() == 2 and sides.max() == 8 and np.all(sides == [x["params"]["gy"] for x in a])
    nu = np.array([x["params"]["nu_ext"][0] for x in a])
    assert nu.min() >= 2.0 and nu.max() <= 8.0 and abs(nu.mean() - 5.0) < 0.3
    g = sorted({x["params"]["g_c"][0] for x in a})
    grid = np.linspace(W.REGIMES["SWA"]["g_c"], W.REGIMES["AW"]["g_c"], 16)
    assert all(np.min(np.abs(grid - v)) < 1e-12 for v in g) and len(g) >= 14
    assert all(x["params"]["g_c"][2] == 0.0 and x["params"]["record_format"] == W.REC_I16 for x in a)
    n = sum(W.n_neurons(x["params"]) for x in a)
    assert n == 8_516_250                                               # the sweep of the benchmark


def test_serving_request_recipe():
    r = W.serving_requests()
    assert len(r) == 2000 and r == W.serving_requests()
    t = np.array([x["arrival_s"] for x in r])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() - 0.1) < 0.01               # Poisson at 10 requests/s
    sides = np.array([x["params"]["gx"] for x in r])
    assert sides.min() == 2 and sides.max() == 16
    # log-uniform side: P(side <= 4) = P(U(1, 4) <= log2(4.5)) for the rounding
    frac = np.mean(sides <= 4)
    assert abs(frac - (math.log2(4.5) - 1.0) / 3.0) < 0.04
    dur = np.array([x["steps"] for x in r]) * W.DT_MS * 1e-3
    assert dur.min() >= 0.5 - 1e-9 and dur.max() <= 10.0 + 1e-9 and abs(dur.mean() - 5.25) < 0.3
    swa = np.mean([x["regime"] == "SWA" for x in r])
    assert abs(swa - 0.5) < 0.04


@pytest.mark.parametrize("state", ["SW_3.1Hz", "AW_2.8Hz", "AW_8.8Hz"])
def test_table_s1_parameter_sets(state):
    p = W.table_s1_params(24, 24, 0.6, state)
    J = np.array(p["J"])
    assert np.all(J[:, :2] > 0) and np.all(J[:, 2] == -1.5) and p["p_local"] < 0
    assert p["g_c"] == [0.02, 0.02, 0.0] and p["N_ext"] == [400.0, 400.0, 400.0]
