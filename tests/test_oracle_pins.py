"""Pins of the CPU oracle against things other than itself.

Each test checks one oracle function against a closed form of Eq. 2, a value
printed in the paper, a library routine (cuRAND's host Philox, SciPy's normal
and Poisson functions), a statistical law of the construction (Eq. 1, the
Gaussian efficacies, uniform delays) or a plain definition evaluated directly
(input at step t = sum of the weights of synapses whose source fired at t-d).
None of them calls the CUDA path.
"""
import ctypes
import json
import math
import os

import numpy as np
import pytest
import scipy.special
import scipy.stats

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# Philox4x32-10: against cuRAND's host generator (a library routine)
# ---------------------------------------------------------------------------
def _curand_host_blocks(seed, n_blocks):
    path = None
    for cand in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            path = ctypes.CDLL(cand)
            break
        except OSError:
            continue
    if path is None:
        pytest.skip("libcurand not available")
    lib = path
    g = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(g), 161) != 0:   # CURAND_RNG_PSEUDO_PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(4 * n_blocks, dtype=np.uint32)
        assert lib.curandGenerate(g, ctypes.c_void_p(out.ctypes.data), ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(g)
    return out.reshape(-1, 4)


def test_philox_matches_curand_host(oracle_mod):
    # cuRAND's host Philox4x32-10 writes block i from counter (i >> 16, 0, i & 0xFFFF, 0)
    # with key = seed (low word, high word).
    for seed in (0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF):
        blocks = _curand_host_blocks(seed, 70000)
        k0, k1 = seed & 0xFFFFFFFF, seed >> 32
        for i in list(range(0, 40)) + [4095, 4096, 65535, 65536, 65537, 69999]:
            ctr = [i >> 16, 0, i & 0xFFFF, 0]
            got = oracle_mod.philox(ctr, k0, k1)
            assert (got == blocks[i]).all(), (seed, i, got, blocks[i])


# ---------------------------------------------------------------------------
# Tables
# ---------------------------------------------------------------------------
def test_ztable_equals_scipy_ndtri(oracle_mod):
    net = oracle_mod.OracleNet(W.base_params(1, 1, 1.0), 1)
    z = net.ztab()
    ref = scipy.special.ndtri((np.arange(4096) + 0.5) / 4096.0).astype(np.float32)
    assert np.array_equal(z, ref)
    assert z[0] < -3.4 and z[-1] > 3.4 and np.all(np.diff(z) > 0)


def test_poisson_thresholds_match_scipy(oracle_mod):
    for nu in (0.0, 1.6, 4.5, 8.0):
        p = W.base_params(1, 1, 1.0)
        p["nu_ext"] = [nu, nu, nu]
        net = oracle_mod.OracleNet(p, 1)
        # parameters cross the ABI as binary32 values
        lam = 400.0 * float(np.float32(nu)) * float(np.float32(0.1)) / 1000.0
        thr = net.pop_tables(0)["thr"].astype(np.float64)
        cdf = scipy.stats.poisson.cdf(np.arange(16), lam) if lam > 0 else np.ones(16)
        # thresholds on a 20-bit uniform
        assert np.all(np.abs(thr - np.floor(cdf * 2.0 ** 20)) <= 1.0), (nu, thr, cdf)


def test_external_amplitude_table_law(oracle_mod):
    p = W.base_params(1, 1, 1.0)
    net = oracle_mod.OracleNet(p, 1)
    z = net.ztab().astype(np.float64)
    for pop, jext in enumerate(p["J_ext"]):
        amp = net.pop_tables(pop)["amp"].astype(np.float64) / 65536.0
        # quantile table of N(J_ext, (0.25 J_ext)^2) rounded to 2^-16 mV
        assert abs(amp.mean() - jext) < 2e-5
        assert abs(amp.std() - 0.25 * jext * z.std()) < 2e-5
        assert np.all(np.diff(amp) >= 0)


def test_table_s1_values_in_workloads():
    g = _golden("paper_table_s1.json")
    exc, inh = g["neuron"]["Exc"], g["neuron"]["Inh"]
    n = W.TABLE_S1_NEURON
    for i in (0, 1):
        assert n["tau_m"][i] == exc["tau_m"] and n["V_th"][i] == exc["V_th"] and n["V_r"][i] == exc["V_r"]
        assert n["tau_arp"][i] == exc["tau_arp"] and n["alpha_c"][i] == exc["alpha_w"]
        assert n["tau_c"][i] == exc["tau_w"] and n["g_c"][i] == exc["g_w"] and n["C_m"][i] == exc["C_m"]
    assert n["tau_m"][2] == inh["tau_m"] and n["tau_arp"][2] == inh["tau_arp"]
    assert n["alpha_c"][2] == 0.0 and n["g_c"][2] == 0.0
    for state, v in g["external"].items():
        assert W.TABLE_S1_EXT[state]["J_ext"] == v["J_ext"]
        assert W.TABLE_S1_EXT[state]["nu_ext"] == v["nu_ext"]
        cols = g["recurrent_exc_columns_J_FF_BF_IF_FB_BB_IB"][state]
        J = W.TABLE_S1_J[state]
        assert [J[0][0], J[1][0], J[2][0], J[0][1], J[1][1], J[2][1]] == cols


def test_table2_counts():
    # Table 2: neurons = G*K, recurrent = N*M, total = N*(M + N_ext).
    for row in _golden("paper_table2.json")["rows"]:
        G = row["grid"] ** 2
        N = G * W.K
        assert G == row["columns"]
        assert round(N / 1e6, 2) == row["neurons_M"]
        assert abs(N * W.OUT_DEGREE / 1e9 - row["recurrent_G"]) <= 0.065
        assert abs(N * (W.OUT_DEGREE + 400) / 1e9 - row["total_G"]) <= 0.065


# ---------------------------------------------------------------------------
# Eq. 2: closed forms of the neuron update
# ---------------------------------------------------------------------------
def _exc_params(g=0.02, alpha=1.0):
    p = W.base_params(1, 1, 1.0)
    p["g_c"] = [g, g, 0.0]
    p["alpha_c"] = [alpha, alpha, 0.0]
    return p


def test_subthreshold_closed_form(oracle_mod):
    """Free evolution of Eq. 2 (no input): V and c against the FP64 solution."""
    p = _exc_params()
    steps = 3000
    dt, tm, tc, gC = 0.1, 20.0, 1000.0, 0.02
    V0, c0 = 12.0, 30.0
    V, c, s = oracle_mod.neuron_trace(p, 0, V0, c0, np.zeros(steps, np.int32))
    t = dt * np.arange(1, steps + 1)
    c_ref = c0 * np.exp(-t / tc)
    V_ref = V0 * np.exp(-t / tm) - gC * c0 * tm * tc / (tc - tm) * (np.exp(-t / tc) - np.exp(-t / tm))
    assert not s.any()
    assert np.max(np.abs(c - c_ref) / c_ref) < steps * 2.0 ** -23
    # Binary32 propagators carry a relative error <= 2^-24 each; exp(-dt/tau_c) is
    # 1 - 1e-4, so the decay rate of c is off by up to ~3e-4 and the c-driven part of
    # V (about 12 mV here) by up to steps * 2^-24 relative: bound 3000*6e-8*(12+12) mV.
    assert np.max(np.abs(V - V_ref)) < 4.3e-3, np.max(np.abs(V - V_ref))
    # With the closed-form constants rounded to binary32, an FP64 recursion of the
    # same linear map stays within the accumulated per-step rounding of V.
    em, ec = math.exp(-dt / tm), math.exp(-dt / tc)
    Pvv = float(np.float32(em))
    Pcc = float(np.float32(ec))
    Pvc = float(np.float32(-gC * tm * tc / (tc - tm) * (ec - em)))
    v, cc, rec = V0, c0, np.zeros(steps)
    for k in range(steps):
        v, cc = Pvv * v + Pvc * cc, Pcc * cc
        rec[k] = v
    assert np.max(np.abs(V - rec)) < 2e-5, np.max(np.abs(V - rec))
    # the adaptation term matters: without it V would stay positive
    assert V[-1] < -5.0
    # inhibitory population has no adaptation: c does not act on V
    Vi, ci, _ = oracle_mod.neuron_trace(p, 2, V0, c0, np.zeros(steps, np.int32))
    Vi_ref = V0 * np.exp(-t / 10.0)
    assert np.max(np.abs(Vi - Vi_ref)) < 1e-5
    # a resting potential E != 0: V relaxes to E (Eq. 2)
    pE = _exc_params()
    pE["E_L"] = [-3.0, -3.0, 4.0]
    V, c, s = oracle_mod.neuron_trace(pE, 0, V0, c0, np.zeros(steps, np.int32))
    V_ref = -3.0 + (V0 + 3.0) * np.exp(-t / tm) - gC * c0 * tm * tc / (tc - tm) * (np.exp(-t / tc) - np.exp(-t / tm))
    assert np.max(np.abs(V - V_ref)) < 4.3e-3
    Vi, _, _ = oracle_mod.neuron_trace(pE, 2, V0, 0.0, np.zeros(steps, np.int32))
    # near E the decay stalls once (1-P)|V-E| < ulp(E)/2: |V-E| <= 2^-22 / (1 - P) = 2.4e-5 mV
    stall = 2.0 ** -22 / (1 - math.exp(-dt / 10.0))
    assert np.max(np.abs(Vi - (4.0 + (V0 - 4.0) * np.exp(-t / 10.0)))) < stall + 1e-6


def _isi_steps(spikes):
    idx = np.flatnonzero(spikes)
    return np.diff(idx)


def test_lif_isi_constant_drive(oracle_mod):
    """Constant fixed-point drive x per step, no adaptation.

    V_k = V_inf + (V_r - V_inf) P^k with V_inf = x/(1-P), so the ISI in steps is
    n_arp + min{k : V_k > V_theta}; the continuous f-I curve
    nu = 1/(tau_arp + tau_m ln((mu - V_r)/(mu - V_theta))) agrees within one step per ISI.
    """
    p = _exc_params(g=0.0, alpha=0.0)
    P = math.exp(-0.1 / 20.0)
    for x_mv in (0.11, 0.12, 0.15, 0.2, 0.35):
        I = int(round(x_mv * 65536))
        x = I / 65536.0
        V, c, s = oracle_mod.neuron_trace(p, 0, 15.0, 0.0, np.full(20000, I, np.int32))
        isi = _isi_steps(s)
        assert len(isi) > 5
        vinf = x / (1 - P)
        L = math.log((vinf - 20.0) / (vinf - 15.0)) / math.log(P)
        k_star = math.floor(L) + 1
        expect = 20 + k_star
        near_int = abs(L - round(L)) < 1e-3
        ok = (isi[1:] == expect) | (near_int & (np.abs(isi[1:] - expect) <= 1))
        assert ok.all(), (x_mv, isi[:5], expect)
        mu = vinf
        isi_cont_ms = 2.0 + 20.0 * math.log((mu - 15.0) / (mu - 20.0))
        assert abs(isi[1:].mean() * 0.1 - isi_cont_ms) <= 0.1 + 0.0026 * isi_cont_ms


def test_sfa_adapted_rate(oracle_mod):
    """Adapted steady rate: nu = f_LIF(mu - tau_m (g/C) alpha tau_c nu) (tau_c >> ISI)."""
    p = _exc_params(g=0.02, alpha=1.0)
    P = math.exp(-0.1 / 20.0)
    for mu0 in (30.0, 40.0):
        x = mu0 * (1 - P)
        I = int(round(x * 65536))
        mu0 = (I / 65536.0) / (1 - P)
        steps = 200000
        V, c, s = oracle_mod.neuron_trace(p, 0, 0.0, 0.0, np.full(steps, I, np.int32))
        tail = s[steps // 2:]
        rate_hz = tail.sum() / (len(tail) * 1e-4)

        def f(nu_hz):
            mu = mu0 - 20.0 * 0.02 * 1.0 * 1000.0 * nu_hz / 1000.0
            if mu <= 20.0:
                return 0.0
            return 1000.0 / (2.0 + 20.0 * math.log((mu - 15.0) / (mu - 20.0)))

        import scipy.optimize
        nu_star = scipy.optimize.brentq(lambda v: f(v) - v, 1e-3, 500.0)
        assert abs(rate_hz - nu_star) / nu_star < 0.03, (mu0, rate_hz, nu_star)
        # and adaptation lowered the rate well below the unadapted one
        assert rate_hz < 0.8 * f(0.0)
        # mean adaptation variable ~ alpha * tau_c * nu
        assert abs(c[steps // 2:].mean() - nu_star) / nu_star < 0.05


def test_refractory_clamp(oracle_mod):
    p = _exc_params(g=0.0, alpha=0.0)
    V, c, s = oracle_mod.neuron_trace(p, 0, 15.0, 0.0, np.full(500, 6 * 65536, np.int32))
    idx = np.flatnonzero(s)
    assert np.all(np.diff(idx) == 21)      # n_arp = 20 held steps, then 0.995*15 + 6 > 20 in one step
    for k in idx[:-1]:
        assert np.all(V[k:k + 21] == 15.0)


# ---------------------------------------------------------------------------
# Eq. 1 and the synapse records
# ---------------------------------------------------------------------------
def _module_probs(gx, gy, lam, p_local, ms):
    sx, sy = ms % gx, ms // gx
    xs, ys = np.meshgrid(np.arange(gx), np.arange(gy))
    d = np.sqrt((xs - sx) ** 2 + (ys - sy) ** 2).ravel()
    e = np.exp(-d / lam)
    if p_local >= 0:
        e[ms] = 0.0
        pr = (1 - p_local) * e / e.sum()
        pr[ms] = p_local
    else:
        pr = e / e.sum()
    return pr


def _chi2_p(obs, exp, min_exp=5.0):
    obs = np.asarray(obs, float)
    exp = np.asarray(exp, float)
    order = np.argsort(exp)
    o, e = obs[order], exp[order]
    # merge the smallest-expectation bins until each has >= min_exp
    mo, me, acc_o, acc_e = [], [], 0.0, 0.0
    for a, b in zip(o, e):
        acc_o += a
        acc_e += b
        if acc_e >= min_exp:
            mo.append(acc_o)
            me.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0:
        if me:
            mo[-1] += acc_o
            me[-1] += acc_e
        else:
            mo.append(acc_o)
            me.append(acc_e)
    mo, me = np.array(mo), np.array(me)
    stat = ((mo - me) ** 2 / me).sum()
    return scipy.stats.chi2.sf(stat, max(len(me) - 1, 1))


@pytest.mark.parametrize("ms", [12, 0, 4])
def test_target_module_law(oracle_mod, ms):
    gx = gy = 5
    p = W.base_params(gx, gy, 1.0)
    net = oracle_mod.OracleNet(p, 3)
    src = ms * W.K + np.arange(0, 1000, 2)          # excitatory sources (F and B)
    keys, _ = net.rows(src)
    tgt = (keys & 0xFFFFFF).ravel()
    mods = tgt // W.K
    obs = np.bincount(mods, minlength=gx * gy)
    exp = _module_probs(gx, gy, 1.0, 0.8, ms) * mods.size
    assert _chi2_p(obs, exp) > 1e-3
    assert abs(obs[ms] / mods.size - 0.8) < 4 * math.sqrt(0.16 / mods.size)


def test_cdf_thresholds_follow_eq1(oracle_mod):
    gx, gy = 6, 4
    for lam, pl in ((0.4, 0.8), (1.0, 0.8), (0.6, -1.0)):
        p = W.base_params(gx, gy, lam, p_local=pl)
        net = oracle_mod.OracleNet(p, 1)
        for ms in (0, 7, 23):
            # lambda and p_local cross the ABI as binary32 values
            pr = _module_probs(gx, gy, float(np.float32(lam)), float(np.float32(pl)), ms)
            thr = net.cdf_row(ms).astype(np.float64) / 2.0 ** 32
            assert np.max(np.abs(thr - np.cumsum(pr)[:-1])) < 1e-9


def test_delay_target_weight_laws(oracle_mod):
    p = W.base_params(3, 3, 1.0)
    net = oracle_mod.OracleNet(p, 5)
    m = 4
    exc = m * W.K + np.arange(0, 1000, 4)
    inh = m * W.K + np.arange(1000, 1250)
    ke, we = net.rows(exc)
    ki, wi = net.rows(inh)
    d = (ke >> 24).ravel()
    assert d.min() == 1 and d.max() == 20
    assert _chi2_p(np.bincount(d, minlength=21)[1:], np.full(20, d.size / 20)) > 1e-3
    lt = ((ke & 0xFFFFFF) % W.K).ravel()
    assert _chi2_p(np.bincount(lt, minlength=W.K), np.full(W.K, lt.size / W.K)) > 1e-3
    # inhibitory projections stay in the source module (Sec. 2.2)
    assert np.all((ki & 0xFFFFFF) // W.K == m)
    zsd = net.ztab().astype(np.float64).std()
    for w, J in ((we.ravel().astype(np.float64), 0.5), (wi.ravel().astype(np.float64), -2.0)):
        se = 0.25 * abs(J) / math.sqrt(w.size)
        assert abs(w.mean() - J) < 4 * se
        assert abs(w.std() / (0.25 * abs(J) * zsd) - 1) < 0.02
        assert np.all(np.sign(w[w != 0]) == np.sign(J))


@pytest.mark.parametrize("min_delay,n_delay", [(10, 20), (20, 20), (3, 254)])
def test_min_delay_law(oracle_mod, min_delay, n_delay):
    """Delays uniform on min_delay..n_delay (the paper's 1 ms minimum delay,
    Sec. 2.1.1, is 10 steps of 0.1 ms); min_delay 0 and 1 give the same rows."""
    p = W.base_params(3, 3, 1.0)
    p["n_delay"], p["min_delay"] = n_delay, min_delay
    net = oracle_mod.OracleNet(p, 5)
    keys, _ = net.rows(range(4 * W.K, 4 * W.K + 1250, 5))
    d = (keys >> 24).ravel()
    span = n_delay - min_delay + 1
    assert d.min() >= min_delay and d.max() <= n_delay
    if span > 1:
        assert d.min() == min_delay and d.max() == n_delay
        counts = np.bincount(d - min_delay, minlength=span)
        assert _chi2_p(counts, np.full(span, d.size / span)) > 1e-3
    p0, p1 = dict(p), dict(p)
    p0["min_delay"], p1["min_delay"] = 0, 1
    a, b = oracle_mod.OracleNet(p0, 5), oracle_mod.OracleNet(p1, 5)
    assert np.array_equal(a.row(7000)[0], b.row(7000)[0])


def test_rows_are_stable_sorted_by_delay_then_target(oracle_mod):
    """Rows hold the individually drawn synapses ordered by delay, then target,
    then draw index (NumPy's lexicographic sort of the drawn records)."""
    p = W.base_params(2, 2, 0.4)
    net = oracle_mod.OracleNet(p, 9)
    for s in (0, 777, 1249, 2600, 4999):
        keys, w = net.row(s)
        raw = [net.synapse(s, j) for j in range(net.M)]
        rk = np.array([r[0] for r in raw], np.uint32)
        rw = np.array([r[1] for r in raw], np.float32)
        order = np.lexsort((np.arange(len(rk)), rk & 0xFFFFFF, rk >> 24))
        assert np.array_equal(keys, rk[order])
        assert np.array_equal(w, rw[order])
        assert len(keys) == 1125
        assert np.all(np.diff((keys >> 24).astype(np.int64)) >= 0)


def test_pure_kernel_local_share(oracle_mod):
    """Pure Eq. 1 kernel: share of excitatory synapses kept in the source module."""
    gx = gy = 11
    paper = _golden("paper_local_share.json")["lambda_to_local_share"]
    for lam in (0.4, 0.6):
        p = W.base_params(gx, gy, lam, p_local=-1.0)
        net = oracle_mod.OracleNet(p, 2)
        ms = 60
        keys, _ = net.rows(ms * W.K + np.arange(0, 1000, 2))
        share = np.mean((keys & 0xFFFFFF) // W.K == ms)
        xs = np.arange(-30, 31)
        d = np.sqrt(xs[:, None] ** 2 + xs[None, :] ** 2)
        exact = 1.0 / np.exp(-d / lam).sum()
        assert abs(share - exact) < 4 * math.sqrt(exact * (1 - exact) / keys.size)
        assert abs(share - paper[str(lam)]) < 0.08


def test_single_module_grid(oracle_mod):
    net = oracle_mod.OracleNet(W.base_params(1, 1, 0.4), 4)
    keys, _ = net.rows(range(0, 1250, 25))
    assert np.all((keys & 0xFFFFFF) < 1250)


# ---------------------------------------------------------------------------
# Whole-network definitions
# ---------------------------------------------------------------------------
def _wfix(w, fmt):
    w = w.astype(np.float32)
    if fmt == W.REC_I16:
        q = np.clip(np.rint(w * np.float32(1024.0)), -32768, 32767).astype(np.int64)
        return q * 64
    return np.rint(w * np.float32(65536.0)).astype(np.int64)


@pytest.mark.parametrize("fmt,min_delay", [(W.REC_F32, 1), (W.REC_I16, 1), (W.REC_F32, 10)])
def test_recurrent_input_definition(oracle_mod, fmt, min_delay):
    """Input read at step t = sum over spikes (t', s) and records (d, tgt) of s
    with t' + d = t of the record's fixed-point weight."""
    p = W.base_params(2, 1, 1.0, "AW", record_format=fmt)
    p["min_delay"] = min_delay
    net = oracle_mod.OracleNet(p, 21)
    T = 400
    net.enable_trace(0, T)
    net.run(T)
    rec, ext = net.trace()
    ts, ids = net.raster()
    assert len(ts) > 200
    exp = np.zeros((T + 32, net.N), np.int64)
    for s in np.unique(ids):
        keys, w = net.row(int(s))
        d = (keys >> 24).astype(np.int64)
        tgt = (keys & 0xFFFFFF).astype(np.int64)
        wf = _wfix(w, fmt)
        for t0 in ts[ids == s]:
            np.add.at(exp, (t0 + d, tgt), wf)
    assert np.array_equal(exp[:T], rec.astype(np.int64))
    # the external input is a Poisson count of Gaussian amplitudes: mean lambda*J_ext
    lam = 400 * 4.5 * 1e-4
    e = ext[:, :1000].astype(np.float64) / 65536.0
    assert abs(e.mean() - lam * 0.858) < 4 * math.sqrt(lam * 0.858 ** 2 * 1.07 / e.size)


def test_rates_refractory_and_counters(oracle_mod):
    p = W.base_params(2, 2, 0.4, "AW")
    net = oracle_mod.OracleNet(p, 8)
    net.run(1000)
    ts, ids = net.raster()
    assert np.all(np.diff(ts.astype(np.int64)) >= 0)
    # rates are the raster binned by (5 ms bin, module, population)
    pops = np.where(ids % W.K < 250, 0, np.where(ids % W.K < 1000, 1, 2))
    hist = np.zeros((20, 4, 3), np.uint32)
    np.add.at(hist, (ts // 50, ids // W.K, pops), 1)
    assert np.array_equal(hist, net.rates())
    # refractoriness: consecutive spikes of one neuron at least n_arp + 1 steps apart
    order = np.lexsort((ts, ids))
    same = ids[order][1:] == ids[order][:-1]
    gaps = np.diff(ts[order].astype(np.int64))[same]
    gap_min = np.where(ids[order][1:][same] % W.K < 1000, 21, 11)
    assert np.all(gaps >= gap_min)
    c = net.counters()
    assert c["spikes"] == len(ts) and c["rec_events"] == len(ts) * 1125
    lam = 400 * 4.5 * 1e-4
    n_draws = 1000 * net.N
    assert abs(c["ext_events"] / n_draws - lam) < 4 * math.sqrt(lam / n_draws)


def test_counter_based_construction_is_order_free(oracle_mod):
    """A row depends only on (seed, source): building it before or after running
    the network, or in a second instance, gives the same bytes."""
    p = W.base_params(2, 2, 0.4)
    a = oracle_mod.OracleNet(p, 77)
    k1, w1 = a.row(3000)
    a.run(200)
    k2, w2 = a.row(3000)
    b = oracle_mod.OracleNet(p, 77)
    k3, w3 = b.row(3000)
    c = oracle_mod.OracleNet(p, 78)
    k4, _ = c.row(3000)
    assert np.array_equal(k1, k2) and np.array_equal(k1, k3)
    assert np.array_equal(w1, w2) and np.array_equal(w1, w3)
    assert not np.array_equal(k1, k4)


def test_shot_noise_campbell(oracle_mod):
    """Threshold out of reach, no recurrent input: V is a linear filter of the
    external shot noise.  In discrete time with per-step input of mean lam*E[a] and
    variance lam*E[a^2] (compound Poisson), the stationary moments are
    E[V] = lam E[a] / (1 - P) and Var[V] = lam E[a^2] / (1 - P^2)  (Campbell)."""
    p = W.base_params(1, 1, 1.0, "AW")
    p["V_th"] = [1000.0, 1000.0, 1000.0]     # V stays near 31 +- 4 mV
    p["g_c"] = [0.0, 0.0, 0.0]
    net = oracle_mod.OracleNet(p, 31)
    net.run(3000)             # 15 tau_m: V0 <= 1000 mV has decayed below 1e-3 mV
    V, c, _ = net.state()
    assert net.counters()["spikes"] == 0
    lam = 400 * 4.5 * 1e-4
    z = scipy.special.ndtri((np.arange(4096) + 0.5) / 4096.0)
    for sl, tau, jext in ((slice(0, 1000), 20.0, 0.858), (slice(1000, 1250), 10.0, 1.120)):
        P = math.exp(-0.1 / tau)
        a = jext * (1 + 0.25 * z)
        m = lam * a.mean() / (1 - P)
        var = lam * (a ** 2).mean() / (1 - P * P)
        v = V[sl].astype(np.float64)
        assert abs(v.mean() - m) < 4 * math.sqrt(var / v.size), (v.mean(), m)
        assert abs(v.var() / var - 1) < 4 * math.sqrt(2.0 / v.size) + 0.02, (v.var(), var)


def test_external_drive_compound_poisson_cumulants(oracle_mod):
    """At a high external rate (lam = 3 events per step) the per-step external
    input is a compound Poisson sum of independent amplitudes drawn from the
    Gaussian quantile table (Sec. 2.1, Table S1): its cumulants are
    kappa_n = lam E[a^n], n = 1, 2, 3.  A wrong count law moves kappa_1, an
    amplitude index shared by two events of one step moves kappa_2 and kappa_3."""
    p = W.base_params(1, 1, 1.0, "AW")
    p["nu_ext"] = [75.0, 75.0, 75.0]          # 400 trains x 75 Hz x 0.1 ms = 3
    p["V_th"] = [1.0e6, 1.0e6, 1.0e6]
    p["g_c"] = [0.0, 0.0, 0.0]
    net = oracle_mod.OracleNet(p, 5)
    T = 2000
    net.enable_trace(0, T)
    net.run(T)
    _, ext = net.trace()
    assert net.counters()["spikes"] == 0
    lam = 3.0
    z = scipy.special.ndtri((np.arange(4096) + 0.5) / 4096.0)
    for sl, jext in ((slice(0, 1000), 0.858), (slice(1000, 1250), 1.120)):
        a = jext * (1.0 + 0.25 * z)
        k = [lam * (a ** n).mean() for n in range(1, 7)]
        x = ext[:, sl].astype(np.float64).ravel() / 65536.0
        n = x.size
        d = x - x.mean()
        m2, m3 = (d ** 2).mean(), (d ** 3).mean()
        se1 = math.sqrt(k[1] / n)
        se2 = math.sqrt((k[3] + 2 * k[1] ** 2) / n)
        se3 = math.sqrt((k[5] + 9 * k[1] * k[3] + 9 * k[2] ** 2 + 6 * k[1] ** 3) / n)
        assert abs(x.mean() - k[0]) < 5 * se1, (x.mean(), k[0])
        assert abs(m2 - k[1]) < 5 * se2, (m2, k[1])
        assert abs(m3 - k[2]) < 5 * se3, (m3, k[2])


# ---------------------------------------------------------------------------
# Initial state (the paper does not state one; read as V0 uniform on [0, V_th))
# ---------------------------------------------------------------------------
def test_initial_state_uniform_per_population(oracle_mod):
    """V0 of every neuron is uniform on [0, V_th) of its own population, on a
    grid of 2^-24 V_th (a 24-bit uniform), independent from neuron to neuron
    and independent of the draws the other random streams make (construction,
    external drive, extra external events); c0 = 0 and no neuron starts
    refractory.  Distinct thresholds per population catch a wrong population
    lookup, the 24-bit grid and the range catch a wrong shift, neighbour
    correlations and repeated values catch a counter shared by several neurons,
    and the cross-stream correlations catch V0 taken from another stream's
    draw.  Which of the unused streams V0 takes is a contract detail that only
    the GPU parity tests check."""
    p = W.base_params(4, 4, 1.0, "AW")
    p["V_th"] = [20.0, 17.0, 13.0]
    seed = 0x5EED0000ABCD
    net = oracle_mod.OracleNet(p, seed)
    V, c, ref = net.state()
    assert np.all(c == 0.0) and np.all(ref == 0)
    local = np.arange(net.N) % W.K
    pop = np.where(local < 250, 0, np.where(local < 1000, 1, 2))
    vth = np.array(p["V_th"], np.float32)[pop]
    assert np.all(V >= 0.0) and np.all(V < vth)
    # the 24-bit grid: V0 = fl(V_th * k * 2^-24) for an integer k < 2^24
    k = np.rint(V.astype(np.float64) / vth.astype(np.float64) * 2.0 ** 24).astype(np.int64)
    assert np.all((k >= 0) & (k < 2 ** 24))
    assert np.array_equal((vth * (k.astype(np.float32) * np.float32(2.0 ** -24))).astype(np.float32), V)
    assert k.max() > 0.999 * 2 ** 24 and k.min() < 0.001 * 2 ** 24
    u = k / 2.0 ** 24
    for q in range(3):
        assert scipy.stats.kstest(u[pop == q], "uniform").pvalue > 1e-3, q
    # independence across neurons
    n = u.size
    for lag in (1, 2, 3, 4, 1250):
        r = np.corrcoef(u[:-lag], u[lag:])[0, 1]
        assert abs(r) < 4.5 / math.sqrt(n), (lag, r)
    assert np.unique(k).size > n - 60      # ~N^2 / 2^25 = 12 coincidences expected
    # independent of the other streams' draws at the same counters
    k0, k1 = seed & 0xFFFFFFFF, seed >> 32
    idx = np.arange(0, n, 7)
    others = {
        "construction": [oracle_mod.philox([i, 0, 0, 0], k0, k1)[0] for i in idx],
        "drive": [oracle_mod.philox([i // 4, 0, 1, 0], k0, k1)[i % 4] for i in idx],
        "extra events": [oracle_mod.philox([i, 0, 3, 0], k0, k1)[0] for i in idx],
    }
    for name, words in others.items():
        w = (np.array(words, np.uint64) >> 8).astype(np.float64) / 2.0 ** 24
        r = np.corrcoef(w, u[idx])[0, 1]
        assert abs(r) < 4.5 / math.sqrt(idx.size), (name, r)
