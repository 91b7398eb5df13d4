"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Spike rasters, synapse rows, rate counts, counters and the refractory state are
integer results and must match bit for bit.  V and c are binary32 results of
the same operation sequence on both sides; the bar is |a - b| <= 1e-6 * max(1, |b|)
(identical bits are expected: both sides round every operation once, with no
fused multiply-add).  The benchmarked grids at length are in
test_long_parity_gpu.py.
"""
import numpy as np
import pytest

import workloads as W
from parity import assert_same, gpu_results, oracle_results

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1902_08410_gb300 as snn
    snn.build()
    return snn


def _oracle(oracle_mod, params, seed, steps):
    o = oracle_mod.OracleNet(params, seed)
    o.run(steps)
    return o


def _assert_same_run(g, o, steps):
    assert_same(gpu_results(g), oracle_results(o), steps)


# ---------------------------------------------------------------------------
# construction (Eq. 1 rows) -- bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", [
    dict(g=(2, 2), lam=0.4, pl=0.8, fmt=W.REC_F32),
    dict(g=(3, 2), lam=1.0, pl=0.8, fmt=W.REC_I16),
    dict(g=(5, 5), lam=0.6, pl=-1.0, fmt=W.REC_F32),
    dict(g=(1, 1), lam=0.4, pl=0.8, fmt=W.REC_F32),
])
def test_rows_bit_exact(snn, oracle_mod, case):
    p = W.base_params(*case["g"], case["lam"], record_format=case["fmt"], p_local=case["pl"])
    g = snn.Network(p, 17)
    o = oracle_mod.OracleNet(p, 17)
    N = g.N
    rng = np.random.default_rng(0)
    sample = np.unique(np.concatenate([[0, 249, 250, 999, 1000, 1249, N - 1], rng.integers(0, N, 60)]))
    for s in sample:
        gk, gw = g.row(int(s))
        ok, ow = o.row(int(s))
        assert np.array_equal(gk, ok), s
        if case["fmt"] == W.REC_I16:
            q = np.clip(np.rint(ow * np.float32(1024.0)), -32768, 32767).astype(np.float32) / np.float32(1024.0)
            assert np.array_equal(gw, q), s
        else:
            assert np.array_equal(gw, ow), s
    g.close()


@pytest.mark.parametrize("out_degree", [7, 2048])
def test_unusual_out_degree_rows_and_run(snn, oracle_mod, out_degree):
    """Smallest padded row (7 records, M_pad 8) and the largest out-degree
    (2048): construction layout, sort and delivery at the edges."""
    p = W.base_params(2, 2, 0.6, "AW", record_format=W.REC_I16)
    p["out_degree"] = out_degree
    g = snn.Network(p, 23)
    o = oracle_mod.OracleNet(p, 23)
    for s in (0, 250, 1249, 2500, g.N - 1):
        gk, gw = g.row(s)
        ok, ow = o.row(s)
        assert np.array_equal(gk, ok), s
        q = np.clip(np.rint(ow * np.float32(1024.0)), -32768, 32767).astype(np.float32) / np.float32(1024.0)
        assert np.array_equal(gw, q), s
    g.run(300)
    o.run(300)
    _assert_same_run(g, o, 300)
    g.close()


def test_rows_bit_exact_full_size_sample(snn, oracle_mod):
    """24x24 grid (720k neurons, 0.81G synapses): sampled rows."""
    p = W.base_params(24, 24, 1.0)
    g = snn.Network(p, 1)
    o = oracle_mod.OracleNet(p, 1)
    rng = np.random.default_rng(1)
    for s in np.concatenate([[0, g.N - 1], rng.integers(0, g.N, 40)]):
        gk, gw = g.row(int(s))
        ok, ow = o.row(int(s))
        assert np.array_equal(gk, ok) and np.array_equal(gw, ow), s
    g.close()


# ---------------------------------------------------------------------------
# whole runs -- raster bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("fmt", [W.REC_F32, W.REC_I16])
def test_run_4x4_swa(snn, oracle_mod, path, fmt):
    p = W.base_params(4, 4, 0.4, "SWA", record_format=fmt)
    steps = 3000
    g = snn.Network(p, 1)
    g.launch = {"path": path}
    g.run(1234)
    g.run(steps - 1234)       # two calls: windows and rate bins restart mid-bin
    o = _oracle(oracle_mod, p, 1, steps)
    assert o.counters()["spikes"] > 1000
    _assert_same_run(g, o, steps)
    g.close()


def test_run_4x4_swa_full_second(snn, oracle_mod):
    """The 4x4 SWA workload over its full 1 s (10,000 steps)."""
    wl = W.grid_4x4_swa()
    g = snn.Network(wl["params"], wl["seed"])
    g.run(wl["steps"])
    o = _oracle(oracle_mod, wl["params"], wl["seed"], wl["steps"])
    _assert_same_run(g, o, wl["steps"])
    g.close()


@pytest.mark.parametrize("grid,regime", [((1, 1), "AW"), ((3, 2), "AW"), ((2, 3), "SWA")])
def test_run_small_grids(snn, oracle_mod, grid, regime):
    p = W.base_params(*grid, 1.0, regime)
    g = snn.Network(p, 5)
    for n in (1, 7, 50, 443):
        g.run(n)
    o = _oracle(oracle_mod, p, 5, 501)
    _assert_same_run(g, o, 501)


@pytest.mark.parametrize("n_delay,bin_steps,dt_ms", [(1, 50, 0.1), (254, 7, 0.1), (20, 50, 0.05)])
def test_delay_range_bins_and_time_step(snn, oracle_mod, n_delay, bin_steps, dt_ms):
    """Ring depth at both ends (every delay one step: D = 2; delays up to 254
    steps: D = 255), rate bins that do not divide the windows, and a finer time
    step (propagators, Poisson rate and refractory steps all change), over runs
    split across windows, on both record formats."""
    for fmt in (W.REC_F32, W.REC_I16):
        p = W.base_params(2, 2, 0.6, "AW", record_format=fmt)
        p["n_delay"], p["bin_steps"], p["dt_ms"] = n_delay, bin_steps, dt_ms
        g = snn.Network(p, 29)
        for n in (3, 400, 97):
            g.run(n)
        o = _oracle(oracle_mod, p, 29, 500)
        ok, _ = o.row(1000)
        gk, _ = g.row(1000)
        assert np.array_equal(gk, ok)
        assert int((ok >> 24).max()) <= n_delay
        _assert_same_run(g, o, 500)
        g.close()


@pytest.mark.parametrize("n_delay,min_delay", [(20, 10), (7, 4), (20, 20)])
def test_min_delay_exchange_periods(snn, oracle_mod, n_delay, min_delay):
    """Delays on min_delay..n_delay: the spikes of min_delay consecutive steps
    are delivered in one pass after the last of them (Sec. 2.1.1; the paper's
    exchange step of 1 ms = 10 steps).  Both launch paths, both record formats,
    runs and windows that start at every phase of an exchange period."""
    for fmt in (W.REC_F32, W.REC_I16):
        p = W.base_params(2, 3, 0.6, "AW", record_format=fmt)
        p["n_delay"], p["min_delay"] = n_delay, min_delay
        o = _oracle(oracle_mod, p, 41, 700)
        assert o.counters()["spikes"] > 1000
        for path, window in ((0, 33), (0, 351), (1, 64)):
            g = snn.Network(p, 41)
            g.launch = {"path": path, "window_steps": window}
            for n in (3, 401, 96, 200):
                g.run(n)
            _assert_same_run(g, o, 700)
            g.close()
    # the tuner and the kernel timing keep results at a minimum delay too
    p = W.base_params(2, 3, 0.6, "AW")
    p["n_delay"], p["min_delay"] = n_delay, min_delay
    o = _oracle(oracle_mod, p, 41, 700)
    g = snn.Network(p, 41)
    g.run(203)
    g.autotune(30)
    tk = g.time_kernels(97)
    assert tk["update_ms"] > 0 and tk["deliver_ms"] > 0
    g.run(400)
    _assert_same_run(g, o, 700)
    g.close()


def test_run_table_s1_pure_kernel(snn, oracle_mod):
    """Table S1 three-population efficacies with the pure Eq. 1 kernel."""
    p = W.table_s1_params(3, 3, 0.6, "AW_8.8Hz")
    g = snn.Network(p, 3)
    g.run(800)
    o = _oracle(oracle_mod, p, 3, 800)
    _assert_same_run(g, o, 800)


def test_zero_steps_and_no_spike_input(snn, oracle_mod):
    p = W.base_params(1, 1, 1.0, "AW")
    p["nu_ext"] = [0.0, 0.0, 0.0]
    p["V_th"] = [1000.0, 1000.0, 1000.0]
    g = snn.Network(p, 9)
    g.run(0)
    assert g.stats()["t"] == 0
    g.run(300)
    st, ids = g.spikes()
    assert len(st) == 0 and g.stats()["ext_events"] == 0
    o = _oracle(oracle_mod, p, 9, 300)
    _assert_same_run(g, o, 300)


# ---------------------------------------------------------------------------
# batching -- each network identical alone and in the batch
# ---------------------------------------------------------------------------
def test_batch_matches_oracle(snn, oracle_mod):
    specs = [((2, 2), "SWA", W.REC_F32, 11), ((3, 3), "AW", W.REC_I16, 12),
             ((1, 1), "AW", W.REC_F32, 13), ((2, 3), "SWA", W.REC_I16, 14)]
    steps = [900, 600, 900, 350]
    nets, params = [], []
    for (g2, reg, fmt, seed) in specs:
        p = W.base_params(*g2, 1.0, reg, record_format=fmt)
        params.append((p, seed))
        nets.append(snn.Network(p, seed))
    snn.run_batch(nets, steps)
    for (p, seed), n, st in zip(params, nets, steps):
        o = _oracle(oracle_mod, p, seed, st)
        _assert_same_run(n, o, st)
    # a second batch call continues every network from where it stopped
    snn.run_batch(nets, [100] * 4)
    for (p, seed), n, st in zip(params, nets, steps):
        o = _oracle(oracle_mod, p, seed, st + 100)
        _assert_same_run(n, o, st + 100)
    # the batch tuner restores every network: results continue unchanged
    cfg = snn.autotune_batch(nets, 30)
    assert cfg["path"] == 1 and all(n.launch == cfg for n in nets)
    snn.run_batch(nets, [150] * 4)
    for (p, seed), n, st in zip(params, nets, steps):
        o = _oracle(oracle_mod, p, seed, st + 250)
        _assert_same_run(n, o, st + 250)


# ---------------------------------------------------------------------------
# concurrent two-kernel runs on several streams
# ---------------------------------------------------------------------------
def test_run_concurrent_matches_oracle(snn, oracle_mod):
    import torch
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    cases = [(W.base_params(3, 3, 0.4, "SWA"), 21, s1, 600, {}),
             (W.base_params(2, 3, 1.0, "AW", record_format=W.REC_I16), 5, s2, 450, {"window_steps": 100}),
             (W.base_params(2, 2, 1.0, "AW"), 9, s2, 300, {"l2_persist": 0, "window_steps": 64})]
    nets = []
    for p, seed, st, _, launch in cases:
        g = snn.Network(p, seed, stream=st.cuda_stream)
        g.launch = launch
        nets.append(g)
    first = [c[3] // 3 for c in cases]
    snn.run_concurrent(nets, first)
    shapes = snn.autotune_concurrent(nets, 30)   # the pair tuner restores every network
    assert all(sh["path"] == 0 for sh in shapes)
    snn.run_concurrent(nets, [c[3] - f for c, f in zip(cases, first)])
    for g, (p, seed, _, steps, _) in zip(nets, cases):
        _assert_same_run(g, _oracle(oracle_mod, p, seed, steps), steps)
        g.close()
    g = snn.Network(W.base_params(2, 2, 1.0, "AW"), 3)
    g.launch = {"path": 1}
    with pytest.raises(snn.SnnError):
        snn.run_concurrent([g], [10])
    with pytest.raises(snn.SnnError):
        snn.autotune_concurrent([g], 10)
    g.close()


# ---------------------------------------------------------------------------
# launch shapes and the tuner never change results
# ---------------------------------------------------------------------------
def test_launch_shapes_and_autotune_keep_results(snn, oracle_mod):
    p = W.base_params(3, 3, 0.4, "SWA")
    o = _oracle(oracle_mod, p, 21, 700)
    shapes = [dict(path=0, update_block=128, update_groups=1, deliver_warps=2, window_steps=33, deliver_lanes=4),
              dict(path=0, update_block=512, update_groups=2, deliver_warps=8, window_steps=700, deliver_lanes=32),
              dict(path=0, update_block=256, update_groups=4, deliver_warps=1, window_steps=50, deliver_lanes=16),
              dict(path=0, update_block=128, update_groups=4, deliver_warps=4, window_steps=384, deliver_lanes=8),
              dict(path=0, update_block=256, update_groups=1, deliver_warps=2, window_steps=128, deliver_lanes=32,
                   l2_persist=1),
              dict(path=0, update_block=256, update_groups=1, deliver_warps=4, window_steps=90, deliver_lanes=8,
                   deliver_blocks=16),
              dict(path=0, update_block=128, update_groups=2, deliver_warps=8, window_steps=70, deliver_lanes=4,
                   deliver_blocks=1, l2_persist=0),
              dict(path=0, update_block=128, update_groups=1, deliver_warps=4, window_steps=45, deliver_lanes=8,
                   overlap=0),
              dict(path=0, update_block=512, update_groups=1, deliver_warps=16, window_steps=97, deliver_lanes=16,
                   deliver_blocks=32, overlap=1),
              dict(path=1, fused_block=128, fused_items_per_sm=1, window_steps=64, deliver_lanes=8),
              dict(path=1, fused_block=512, fused_items_per_sm=4, window_steps=128, deliver_lanes=4),
              dict(path=1, fused_block=128, fused_items_per_sm=16, window_steps=300, deliver_lanes=32)]
    for sh in shapes:
        g = snn.Network(p, 21)
        g.launch = sh
        g.run(700)
        _assert_same_run(g, o, 700)
        g.close()
    g = snn.Network(p, 21)
    g.run(200)
    g.autotune(50)
    g.run(500)
    _assert_same_run(g, o, 700)
    # kernel timing (a captured graph with event nodes) advances like a run
    g = snn.Network(p, 21)
    g.run(150)
    tk = g.time_kernels(100)
    assert tk["update_ms"] > 0 and tk["deliver_ms"] > 0
    g.run(450)
    _assert_same_run(g, o, 700)


# ---------------------------------------------------------------------------
# the persisting L2 set-aside is raised while a network with the window lives
# and the context's previous limit comes back when the last one is freed
# ---------------------------------------------------------------------------
def test_l2_set_aside_restored(snn):
    import ctypes
    import os
    cudart = None
    for cand in (os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcudart.so"),
                 "libcudart.so"):
        try:
            cudart = ctypes.CDLL(cand)
            break
        except OSError:
            continue
    if cudart is None:
        pytest.skip("libcudart.so not found")
    limit_persisting_l2 = 0x06   # cudaLimitPersistingL2CacheSize

    def limit():
        v = ctypes.c_size_t(0)
        assert cudart.cudaDeviceGetLimit(ctypes.byref(v), limit_persisting_l2) == 0
        return v.value

    before = limit()
    p = W.base_params(2, 2, 1.0, "AW")
    a, b = snn.Network(p, 1), snn.Network(p, 2)
    a.launch = {"l2_persist": 1}
    b.launch = {"l2_persist": 1}
    a.run(20)
    b.run(20)
    raised = limit()
    assert raised >= before and raised > 0
    a.close()
    assert limit() == raised          # b still holds the window
    b.close()
    assert limit() == before


@pytest.mark.parametrize("fmt", [W.REC_F32, W.REC_I16])
def test_rows_bit_exact_64x64_sample(snn, oracle_mod, fmt):
    """64x64 grid (5.12M neurons, 5.76G synapses): sampled rows, both formats
    (whole runs of this grid are compared in test_long_parity_gpu.py)."""
    p = W.base_params(64, 64, 1.0, "AW", record_format=fmt)
    g = snn.Network(p, 1)
    o = oracle_mod.OracleNet(p, 1)
    rng = np.random.default_rng(2)
    for s in np.concatenate([[0, g.N - 1], rng.integers(0, g.N, 20)]):
        gk, gw = g.row(int(s))
        ok, ow = o.row(int(s))
        assert np.array_equal(gk, ok), s
        if fmt == W.REC_I16:
            ow = np.clip(np.rint(ow * np.float32(1024.0)), -32768, 32767).astype(np.float32) / np.float32(1024.0)
        assert np.array_equal(gw, ow), s
    g.close()
