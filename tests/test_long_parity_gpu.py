"""Bit-exact parity with the oracle on the benchmarked configurations, at length.

* 24x24 grid (720k neurons, 0.81G synapses, lambda 1.0, f32 records), the SWA and
  the AW network: 2400 steps each, advanced in both ways the benchmark can
  advance them (the default launch shape alone first, then the two-kernel
  shapes the tuners pick, each network alone and then both together, with
  both networks concurrently on their own streams through snn_run_concurrent,
  then both in one fused kernel per step with the shape the batch tuner picks,
  through snn_run_batch).
* 64x64 grid (5.12M neurons, 5.76G synapses, AW, lambda 1.0): 250 steps on both
  record formats, tuned after the first 100 steps.
* 8x8 grid over the full 2 s of the batched sweep (20,000 steps, SWA, i16
  records) on the fused batch path, next to a 3x5 network, tuned after 2000 steps.
* 24x24 AW network with the paper's 1 ms minimum delay (delays of 10..20 steps,
  one delivery pass per 10 steps): 1500 steps, tuned on the two-kernel path
  after 500.

The oracle runs of all of them start together in spawned worker processes when
the first test of this module asks for them, and compute while the GPU runs.
The 64x64 oracle generates the rows a step needs on several threads and keeps
none (caching every row would take ~46 GB); rows are pure functions of (seed,
source), so neither setting changes its results.
"""
import concurrent.futures
import multiprocessing as mp
import os

import pytest

import workloads as W
from parity import assert_same, gpu_results

pytestmark = pytest.mark.gpu

C2_STEPS, C2_ALONE, C2_CONCURRENT = 2400, 600, 900
C3_STEPS, C3_TUNE_AT = 250, 100
C4_STEPS, C4_TUNE_AT = 20_000, 2000
COMPANION_STEPS = 7000
MD_STEPS, MD_TUNE_AT = 1500, 500


def _c2(regime):
    return W.grid_24x24(regime)["params"], W.grid_24x24(regime)["seed"]


def _c3(fmt):
    return W.base_params(64, 64, 1.0, "AW", record_format=fmt), 1


def _c4():
    return W.base_params(8, 8, 1.0, "SWA", record_format=W.REC_I16), 1000


def _companion():
    return W.base_params(3, 5, 0.4, "AW", record_format=W.REC_F32), 1001


def _md10():
    p = dict(W.grid_24x24("AW")["params"])
    p["min_delay"] = 10
    return p, W.grid_24x24("AW")["seed"]


@pytest.fixture(scope="module")
def snn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1902_08410_gb300 as snn
    snn.build()
    return snn


@pytest.fixture(scope="module")
def oracle_runs(snn, oracle_mod):
    """Futures of every oracle run this module compares with, longest first."""
    cores = os.cpu_count() or 4
    row_threads = max(1, (cores - 4) // 2)
    jobs = {
        "c3_f32": (*_c3(W.REC_F32), C3_STEPS, row_threads, False),
        "c3_i16": (*_c3(W.REC_I16), C3_STEPS, row_threads, False),
        "c2_SWA": (*_c2("SWA"), C2_STEPS, 1, True),
        "c2_AW": (*_c2("AW"), C2_STEPS, 1, True),
        "c4": (*_c4(), C4_STEPS, 1, True),
        "companion": (*_companion(), COMPANION_STEPS, 1, True),
        "md10": (*_md10(), MD_STEPS, 1, True),
    }
    ex = concurrent.futures.ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn"))
    futs = {k: ex.submit(oracle_mod.simulate, *args) for k, args in jobs.items()}
    yield futs
    ex.shutdown(wait=False, cancel_futures=True)


def _oracle(futs, key):
    return futs[key].result(timeout=1500)


def test_grid24x24_swa_aw_as_benchmarked(snn, oracle_runs):
    """Both 24x24 networks as the benchmark runs them, in both forms."""
    import torch
    nets = []
    for reg in ("SWA", "AW"):
        p, seed = _c2(reg)
        st = torch.cuda.Stream()
        g = snn.Network(p, seed, stream=st.cuda_stream)
        g._keep_stream = st
        nets.append(g)
    default = nets[0].launch
    assert default["path"] == 0 and default["l2_persist"] == 1
    for g in nets:
        g.run(C2_ALONE)
        g.autotune(50, path=0)
    snn.autotune_concurrent(nets, 50)
    snn.run_concurrent(nets, C2_CONCURRENT)
    cfg = snn.autotune_batch(nets, 50)
    assert cfg["path"] == 1
    snn.run_batch(nets, [C2_STEPS - C2_ALONE - C2_CONCURRENT] * 2)
    for g, reg in zip(nets, ("SWA", "AW")):
        assert_same(gpu_results(g), _oracle(oracle_runs, f"c2_{reg}"), C2_STEPS, f"24x24 {reg}")
        g.close()


@pytest.mark.parametrize("fmt", [W.REC_F32, W.REC_I16])
def test_grid64x64_250_steps(snn, oracle_runs, fmt):
    p, seed = _c3(fmt)
    g = snn.Network(p, seed)
    g.run(C3_TUNE_AT)
    g.autotune(20)
    g.run(C3_STEPS - C3_TUNE_AT)
    got = gpu_results(g)
    g.close()
    assert_same(got, _oracle(oracle_runs, "c3_f32" if fmt == W.REC_F32 else "c3_i16"), C3_STEPS,
                f"64x64 fmt {fmt}")


def test_grid8x8_full_two_seconds_batched(snn, oracle_runs):
    nets = [snn.Network(*_c4()), snn.Network(*_companion())]
    for g in nets:
        g.launch = {"path": 1}
    snn.run_batch(nets, [C4_TUNE_AT, C4_TUNE_AT])
    snn.autotune_batch(nets, 50)
    snn.run_batch(nets, [C4_STEPS - C4_TUNE_AT, COMPANION_STEPS - C4_TUNE_AT])
    assert_same(gpu_results(nets[0]), _oracle(oracle_runs, "c4"), C4_STEPS, "8x8 SWA i16, 2 s")
    assert_same(gpu_results(nets[1]), _oracle(oracle_runs, "companion"), COMPANION_STEPS, "3x5 AW f32")
    for g in nets:
        g.close()


def test_grid24x24_one_ms_exchange_step(snn, oracle_runs):
    """The paper's exchange step at the benchmarked size: delays of 10..20
    steps, a delivery pass after every 10th step filling the next 10 inputs."""
    p, seed = _md10()
    g = snn.Network(p, seed)
    g.run(MD_TUNE_AT)
    g.autotune(50, path=0)
    before = g.stats()["kernel_launches"]
    g.run(MD_STEPS - MD_TUNE_AT)
    launches = g.stats()["kernel_launches"] - before
    # one update per step and one pass per 10 steps (window graphs count whole windows): ~1.1 per step
    assert launches < 1.25 * (MD_STEPS - MD_TUNE_AT)
    assert_same(gpu_results(g), _oracle(oracle_runs, "md10"), MD_STEPS, "24x24 AW min_delay 10")
    g.close()
