"""Seeded synthetic workloads for the DPSNN-style grid simulation.

This module is the only code shared by the CUDA path, the CPU oracle, the
tests and ``bench.py``.  It holds parameter values and seeded recipes for the
workloads (grid sizes, connectivity scale, regimes, batched sweeps, serving
request streams) and none of the method's arithmetic: no propagators, no
probability tables, no random numbers that the simulation itself consumes.
Each side turns these plain dictionaries into its own parameter struct.

Parameter sources (Pastorelli et al. 2019, "Scaling of a large-scale
simulation of synchronous slow-wave and asynchronous awake-like activity of a
cortical model with long-range interconnections"):

* module of K = 1250 neurons split F 250 / B 750 / I 250 (Sec. 2.2);
* out-degree M = 0.9 K = 1125 recurrent synapses per neuron (Sec. 2.2);
* neuron parameters tau_m, C_m, E, V_theta, V_r, tau_arp, alpha, tau, g and the
  external drive J_ext, nu_ext, N_ext = 400 (Table S1);
* efficacy spread Delta J = 0.25 J (Sec. 2.2).

The benchmark workloads replace Table S1's 3x3 efficacies by a single
excitatory efficacy of +0.5 mV and an inhibitory one of -2.0 mV, 80% of the
excitatory out-degree kept in the source module and the rest spread over the
other modules with probability proportional to exp(-d/lambda), and delays
uniform on 1..20 steps of 0.1 ms.
"""
from __future__ import annotations

import copy
import math
import random

K = 1250                      # neurons per module (Sec. 2.2)
POP_SIZES = (250, 750, 250)   # F, B, I (Sec. 2.2)
POPS = ("F", "B", "I")
OUT_DEGREE = 1125             # M_t = 0.9 K_t (Sec. 2.2; Table 2 counts)
N_DELAY = 20                  # delays uniform on 1..20 steps
DT_MS = 0.1
BIN_STEPS = 50                # 5 ms rate bins (Sec. 2.3)

REC_F32 = 0                   # record: u32 (delay<<24 | target) + f32 weight
REC_I16 = 1                   # record: u32 (delay<<24 | target) + i16 weight (2^-10 mV)

# Table S1, neural dynamics parameters, per population F, B, I.
# Inhibitory neurons have no adaptation (alpha = g = 0).
TABLE_S1_NEURON = {
    "tau_m":   [20.0, 20.0, 10.0],     # ms
    "C_m":     [1.0, 1.0, 1.0],        # pF
    "E_L":     [0.0, 0.0, 0.0],        # mV
    "V_th":    [20.0, 20.0, 20.0],     # mV
    "V_r":     [15.0, 15.0, 15.0],     # mV
    "tau_arp": [2.0, 2.0, 1.0],        # ms
    "alpha_c": [1.0, 1.0, 0.0],        # mV
    "tau_c":   [1000.0, 1000.0, 1000.0],  # ms (unused for I: alpha = 0)
    "g_c":     [0.02, 0.02, 0.0],      # nS
}

# Table S1, recurrent efficacies J[target][source], order F, B, I.
# The inhibitory column of the SW row is printed as +3.17, +3.17, +3.0 (the
# nu_ext values); it is read as negative, with the AW value -1.5 mV.
TABLE_S1_J = {
    "SW_3.1Hz": [[0.600, 0.382, -1.5], [0.382, 0.429, -1.5], [0.560, 0.560, -1.5]],
    "AW_2.8Hz": [[0.515, 0.412, -1.5], [0.412, 0.429, -1.5], [0.560, 0.560, -1.5]],
    "AW_8.8Hz": [[0.515, 0.412, -1.5], [0.412, 0.429, -1.5], [0.560, 0.560, -1.5]],
}
TABLE_S1_EXT = {
    "SW_3.1Hz": {"J_ext": [0.832, 0.858, 1.120], "nu_ext": [3.17, 3.17, 3.0]},
    "AW_2.8Hz": {"J_ext": [0.858, 0.858, 1.120], "nu_ext": [3.17, 3.17, 3.0]},
    "AW_8.8Hz": {"J_ext": [1.416, 1.416, 1.120], "nu_ext": [3.17, 3.17, 3.0]},
}

# Benchmark efficacies: every excitatory source +0.5 mV, inhibitory -2.0 mV.
J_EXC = 0.5
J_INH = -2.0

# Regime knobs for the simplified-efficacy benchmark network, chosen on the
# 4x4 grid with the oracle: SWA = strong adaptation and weak external drive
# (Up/Down alternation), AW = weak adaptation and stronger external drive
# (stationary asynchronous firing).  Values are per-train rates in Hz and
# adaptation conductances in nS.
REGIMES = {
    "SWA": {"g_c": 0.02, "nu_ext": 1.6},   # volleys separated by ~0.25-0.5 s Down states, ~4 Hz mean
    "AW": {"g_c": 0.005, "nu_ext": 4.5},   # stationary asynchronous firing, ~8.7 Hz mean
}


def base_params(gx: int, gy: int, lam: float, regime: str = "SWA",
                record_format: int = REC_F32, p_local: float = 0.8) -> dict:
    """Parameter dictionary of the benchmark network (simplified efficacies)."""
    reg = REGIMES[regime]
    p = {
        "gx": int(gx), "gy": int(gy), "lambda": float(lam), "p_local": float(p_local),
        "out_degree": OUT_DEGREE, "n_delay": N_DELAY, "min_delay": 1, "dt_ms": DT_MS,
        "record_format": int(record_format), "bin_steps": BIN_STEPS,
        "dJ_frac": 0.25, "dJ_ext_frac": 0.25,
        "J": [[J_EXC, J_EXC, J_INH] for _ in range(3)],
        "J_ext": [0.858, 0.858, 1.120],
        "nu_ext": [reg["nu_ext"]] * 3,
        "N_ext": [400.0, 400.0, 400.0],
    }
    for k, v in TABLE_S1_NEURON.items():
        p[k] = list(v)
    p["g_c"] = [reg["g_c"], reg["g_c"], 0.0]
    return p


def table_s1_params(gx: int, gy: int, lam: float, state: str = "AW_8.8Hz",
                    record_format: int = REC_F32) -> dict:
    """Table S1 three-population parameter set with the pure Eq. 1 kernel."""
    p = base_params(gx, gy, lam, "SWA", record_format, p_local=-1.0)
    p["J"] = copy.deepcopy(TABLE_S1_J[state])
    p["J_ext"] = list(TABLE_S1_EXT[state]["J_ext"])
    p["nu_ext"] = list(TABLE_S1_EXT[state]["nu_ext"])
    p["g_c"] = [0.02, 0.02, 0.0]
    return p


def with_overrides(p: dict, **kw) -> dict:
    q = copy.deepcopy(p)
    q.update(kw)
    return q


# ---------------------------------------------------------------------------
# Named workloads.  `steps` is the simulated duration in 0.1 ms steps.
# ---------------------------------------------------------------------------
def grid_4x4_swa() -> dict:
    """4x4 grid, 20k neurons, lambda 0.4, SWA, 1 s, seed 1."""
    return {"name": "grid4x4_swa", "params": base_params(4, 4, 0.4, "SWA"),
            "seed": 1, "steps": 10_000}


def grid_24x24(regime: str) -> dict:
    """24x24 grid, 720k neurons, 0.81G recurrent synapses, lambda 1.0, 10 s."""
    return {"name": f"grid24x24_{regime.lower()}", "params": base_params(24, 24, 1.0, regime),
            "seed": 1, "steps": 100_000}


def grid_64x64(regime: str, lam: float, record_format: int) -> dict:
    """64x64 grid, 5.12M neurons, 5.76G recurrent synapses, 5 s."""
    fmt = "i16" if record_format == REC_I16 else "f32"
    return {"name": f"grid64x64_{regime.lower()}_l{lam}_{fmt}",
            "params": base_params(64, 64, lam, regime, record_format),
            "seed": 1, "steps": 50_000}


def batched_sweep(n_nets: int = 256, sample_seed: int = 7, steps: int = 20_000,
                  record_format: int = REC_I16) -> list[dict]:
    """Independent networks for a SWA->AW sweep.

    Grid side uniform on 2..8, adaptation g_c on a 16-point linear grid from the
    SWA to the AW value, external per-train rate uniform on [2, 8] Hz, network
    i seeded 1000 + i.
    """
    rng = random.Random(sample_seed)
    g_hi, g_lo = REGIMES["SWA"]["g_c"], REGIMES["AW"]["g_c"]
    g_grid = [g_hi + (g_lo - g_hi) * k / 15.0 for k in range(16)]
    nets = []
    for i in range(n_nets):
        side = rng.randint(2, 8)
        g = g_grid[rng.randrange(16)]
        nu = rng.uniform(2.0, 8.0)
        p = base_params(side, side, 1.0, "SWA", record_format)
        p["g_c"] = [g, g, 0.0]
        p["nu_ext"] = [nu, nu, nu]
        nets.append({"name": f"sweep{i}", "params": p, "seed": 1000 + i, "steps": steps})
    return nets


def serving_requests(n_req: int = 2000, seed: int = 11, rate_hz: float = 10.0,
                     min_side: int = 2, max_side: int = 16,
                     min_s: float = 0.5, max_s: float = 10.0,
                     record_format: int = REC_I16) -> list[dict]:
    """Poisson-arrival stream of simulation requests.

    Grid side round(2^U(log2 min, log2 max)) (log-uniform), duration uniform on
    [min_s, max_s] simulated seconds, SWA/AW 50/50.  `arrival_s` is the
    request's arrival time in wall seconds from the start of the stream.
    """
    rng = random.Random(seed)
    t = 0.0
    reqs = []
    lo, hi = math.log2(min_side), math.log2(max_side)
    for i in range(n_req):
        t += rng.expovariate(rate_hz)
        side = int(round(2.0 ** rng.uniform(lo, hi)))
        dur = rng.uniform(min_s, max_s)
        regime = "SWA" if rng.random() < 0.5 else "AW"
        p = base_params(side, side, 1.0, regime, record_format)
        reqs.append({"name": f"req{i}", "params": p, "seed": 5000 + i,
                     "steps": int(round(dur / (DT_MS * 1e-3))), "arrival_s": t,
                     "regime": regime})
    return reqs


def n_neurons(p: dict) -> int:
    return p["gx"] * p["gy"] * K
