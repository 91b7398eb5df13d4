"""Mean-field description of a module (Eq. 3; host FP64): the
first-passage-time gain function against its deterministic limit and against
the oracle's simulation of unconnected neurons under Poisson drive (a pin
independent of the gain's formula), and the fixed points and nullclines of
Eq. 3."""
import math

import numpy as np
import pytest

import workloads as W
from paper_1902_08410_gb300 import meanfield as M


def test_gain_deterministic_limit():
    """sigma -> 0 above threshold: 1 / (tau_arp + tau_m ln((mu - V_r) / (mu - V_th)))."""
    for mu in (20.5, 22.0, 30.0):
        exact = 1.0 / (2.0 + 20.0 * math.log((mu - 15.0) / (mu - 20.0)))
        assert M.gain(mu, 0.0, 20.0, 2.0, 20.0, 15.0) == pytest.approx(exact, rel=1e-12)
        assert M.gain(mu, 1e-3, 20.0, 2.0, 20.0, 15.0) == pytest.approx(exact, rel=2e-3)
    assert M.gain(19.0, 0.0, 20.0, 2.0, 20.0, 15.0) == 0.0
    assert M.gain(10.0, 0.05, 20.0, 2.0, 20.0, 15.0) < 1e-12


def _unconnected(mu_e, mu_i, jext=0.1):
    p = W.base_params(1, 1, 1.0, "AW")
    p["J"] = [[0.0] * 3 for _ in range(3)]
    p["g_c"] = [0.0] * 3
    p["J_ext"] = [jext] * 3
    tau = p["tau_m"]
    p["nu_ext"] = [1e3 * mu_e / (400 * jext * tau[0]), 1e3 * mu_e / (400 * jext * tau[1]),
                   1e3 * mu_i / (400 * jext * tau[2])]
    return p


@pytest.mark.parametrize("mu_e,mu_i", [(22.0, 22.0), (18.5, 18.5), (25.0, 30.0)])
def test_gain_matches_simulated_unconnected_neurons(oracle_mod, mu_e, mu_i):
    """1250 neurons without recurrent synapses, driven by 400 Poisson trains of
    0.1 mV (+-25%) events, simulated by the oracle for 1.8 s after a 0.2 s
    transient: the excitatory (inhibitory) rate agrees with the diffusion
    gain within 3% (6%); the rest is the time step and the finite jumps."""
    p = _unconnected(mu_e, mu_i)
    mu, sigma = M.moments(p, [0, 0, 0], [0, 0, 0])
    assert np.allclose(mu, [mu_e, mu_e, mu_i])
    o = oracle_mod.OracleNet(p, 3)
    o.run(20000)
    t, i = o.raster()
    loc, keep = i % 1250, t >= 2000
    sim_e = np.count_nonzero((loc < 1000) & keep) / (1000 * 1.8)
    sim_i = np.count_nonzero((loc >= 1000) & keep) / (250 * 1.8)
    th = M.phi(p, [0, 0, 0], [0, 0, 0])
    assert sim_e == pytest.approx(th[0], rel=0.03), (sim_e, th)
    assert sim_i == pytest.approx(th[2], rel=0.06), (sim_i, th)


def test_moments_of_the_recurrent_input():
    """mu and sigma^2 are linear in the rates with the in-degree split by
    population sizes (1125 synapses: 225 F, 675 B, 225 I)."""
    p = W.base_params(4, 4, 0.4, "AW")
    mu0, s0 = M.moments(p, [0, 0, 0], [0, 0, 0])
    mu1, s1 = M.moments(p, [10.0, 0, 0], [0, 0, 0])
    assert mu1[0] - mu0[0] == pytest.approx(20.0 * 225 * 0.5 * 10e-3)
    assert s1[0] ** 2 - s0[0] ** 2 == pytest.approx(20.0 * 225 * 0.25 * 1.0625 * 10e-3)
    mu2, _ = M.moments(p, [0, 0, 0], [2.0, 2.0, 0.0])
    assert mu0[0] - mu2[0] == pytest.approx(20.0 * 0.005 * 2.0)


@pytest.mark.parametrize("regime", ["AW", "SWA"])
def test_fixed_point_and_nullclines(regime):
    """Relaxing Eq. 3 reaches a stable fixed point: nu = phi(nu, c) with
    c = alpha tau_c nu, every Jacobian eigenvalue negative, and the rate
    nullcline at that fatigue passes through it."""
    p = W.base_params(4, 4, 0.4, regime)
    fp = M.fixed_point(p, (5.0, 5.0, 20.0), relax_ms=3000.0)
    assert fp["converged"] and fp["residual_hz"] < 1e-6
    nu, c = fp["nu_hz"], fp["c_mv"]
    assert c[0] == pytest.approx(1.0 * 1000.0 * nu[0] * 1e-3) and c[2] == 0.0
    assert np.all(fp["eigenvalues"].real < 0.0)
    roots = M.rate_nullcline(p, c[0], np.geomspace(1e-3, 300.0, 300))
    assert np.min(np.abs(roots - nu[0])) < 1e-6
    _, traj, _ = M.integrate(p, nu, c, 200.0)
    assert np.allclose(traj[-1], nu, rtol=1e-6, atol=1e-9)
