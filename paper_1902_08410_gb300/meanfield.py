"""Mean-field description of one module (host, FP64, off the per-step path).

Sec. 2.2 and Eq. 3 of the paper: every population p of a module (F, B, I)
receives independent inputs with a common mean and variance; its stationary
rate is the first-passage-time gain function of a leaky integrate-and-fire
neuron driven by white noise in the diffusion approximation (Ricciardi),

    1 / phi = tau_arp + tau_m sqrt(pi) * integral from (V_r - mu)/sigma
              to (V_th - mu)/sigma of exp(u^2) (1 + erf u) du,

and Eq. 3 lets the excitatory rates relax to phi with time constant tau_E,
the inhibitory rate with tau_I, while the fatigue variable c of the
excitatory populations follows dc/dt = -c / tau_c + alpha_c nu.

Input moments for population t (rates in 1/ms, J in mV, tau in ms), from
Eq. 2 with delta-shaped synaptic input and the adaptation current -g_c c / C_m:

    mu_t      = E_t + tau_m,t (sum_s K_ts J_ts nu_s + N_ext J_ext,t nu_ext,t - (g_c / C_m)_t c_t)
    sigma_t^2 = tau_m,t (sum_s K_ts J_ts^2 (1 + dJ^2) nu_s + N_ext J_ext,t^2 (1 + dJ_ext^2) nu_ext,t)

(dJ = relative spread of the efficacies).  K_ts is the mean number of
synapses a neuron of population t receives from population s: with a fixed
out-degree M and targets uniform within a module, every neuron receives M
synapses on average, split by the sources' population sizes (250, 750, 250
of 1250), so K_ts = M N_s / 1250.  In a grid whose modules share the same
rates the inter-module synapses carry the same rates, so the module's
mean field uses the whole in-degree.

The integrand exp(u^2)(1 + erf u) equals erfcx(-u), which stays finite for
any u.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import quad
from scipy.special import erfcx

POP_SIZES = (250, 750, 250)   # F, B, I neurons of a 1250-neuron module (Sec. 2.1)
K = 1250


def gain(mu: float, sigma: float, tau_m: float, tau_arp: float, v_th: float, v_r: float) -> float:
    """Ricciardi's first-passage-time rate (1/ms) of a LIF neuron whose free
    membrane potential has mean mu and diffusion amplitude sigma (mV); sigma = 0
    gives the deterministic rate."""
    if sigma <= 0.0:
        if mu <= v_th:
            return 0.0
        return 1.0 / (tau_arp + tau_m * math.log((mu - v_r) / (mu - v_th)))
    lo, hi = (v_r - mu) / sigma, (v_th - mu) / sigma
    if lo > 30.0:
        return 0.0                # the integrand exceeds e^900 over the whole range
    integral, _ = quad(lambda u: erfcx(-u), lo, hi, limit=200)
    return 1.0 / (tau_arp + tau_m * math.sqrt(math.pi) * integral)


def _pop(p: dict, key: str) -> np.ndarray:
    return np.asarray(p[key], dtype=np.float64)


def in_degree(p: dict) -> np.ndarray:
    """K[t][s]: mean synapses a neuron of population t receives from population s."""
    frac = np.asarray(POP_SIZES, np.float64) / K
    return np.tile(float(p["out_degree"]) * frac, (3, 1))


def moments(p: dict, nu_hz, c) -> tuple[np.ndarray, np.ndarray]:
    """(mu, sigma) in mV of the three populations for rates nu (Hz) and fatigue c (mV)."""
    nu = np.asarray(nu_hz, np.float64) * 1e-3          # 1/ms
    c = np.asarray(c, np.float64)
    tau = _pop(p, "tau_m")
    J = np.asarray(p["J"], np.float64)
    Kts = in_degree(p)
    dj, dje = float(p["dJ_frac"]), float(p["dJ_ext_frac"])
    jext, next_, nuext = _pop(p, "J_ext"), _pop(p, "N_ext"), _pop(p, "nu_ext") * 1e-3
    g_over_c = _pop(p, "g_c") / _pop(p, "C_m")
    drift = (Kts * J) @ nu + next_ * jext * nuext - g_over_c * c
    diff = (Kts * J * J * (1.0 + dj * dj)) @ nu + next_ * jext * jext * (1.0 + dje * dje) * nuext
    mu = _pop(p, "E_L") + tau * drift
    sigma = np.sqrt(np.maximum(tau * diff, 0.0))
    return mu, sigma


def phi(p: dict, nu_hz, c) -> np.ndarray:
    """Gain functions of the three populations (Hz)."""
    mu, sigma = moments(p, nu_hz, c)
    tau, arp, vth, vr = _pop(p, "tau_m"), _pop(p, "tau_arp"), _pop(p, "V_th"), _pop(p, "V_r")
    return np.array([1e3 * gain(mu[i], sigma[i], tau[i], arp[i], vth[i], vr[i]) for i in range(3)])


def eq3_rhs(p: dict, nu_hz, c, tau_e: float = 20.0, tau_i: float = 10.0) -> tuple[np.ndarray, np.ndarray]:
    """Eq. 3: (d nu / dt in Hz/ms, dc / dt in mV/ms); tau_E and tau_I in ms.
    Populations with alpha_c = 0 (the inhibitory one) carry no fatigue."""
    nu = np.asarray(nu_hz, np.float64)
    c = np.asarray(c, np.float64)
    alpha, tau_c = _pop(p, "alpha_c"), _pop(p, "tau_c")
    exc = alpha > 0.0
    tau_pop = np.where(exc, tau_e, tau_i)
    dnu = (phi(p, nu, c) - nu) / tau_pop
    dc = np.where(exc, -c / tau_c + alpha * nu * 1e-3, 0.0)
    return dnu, dc


def integrate(p: dict, nu0_hz, c0, t_ms: float, dt_ms: float = 0.5, tau_e: float = 20.0,
              tau_i: float = 10.0) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Euler integration of Eq. 3: returns (t [ms], nu [step][pop] in Hz, c [step][pop])."""
    n = int(round(t_ms / dt_ms))
    nu = np.asarray(nu0_hz, np.float64).copy()
    c = np.asarray(c0, np.float64).copy()
    tt = np.arange(n + 1) * dt_ms
    out_nu = np.empty((n + 1, 3))
    out_c = np.empty((n + 1, 3))
    out_nu[0], out_c[0] = nu, c
    for k in range(n):
        dnu, dc = eq3_rhs(p, nu, c, tau_e, tau_i)
        nu = np.maximum(nu + dt_ms * dnu, 0.0)
        c = c + dt_ms * dc
        out_nu[k + 1], out_c[k + 1] = nu, c
    return tt, out_nu, out_c


def adapted_fatigue(p: dict, nu_hz) -> np.ndarray:
    """Stationary fatigue c = alpha_c tau_c nu (mV) of the c-nullcline."""
    return _pop(p, "alpha_c") * _pop(p, "tau_c") * np.asarray(nu_hz, np.float64) * 1e-3


def fixed_point(p: dict, nu0_hz=(5.0, 5.0, 10.0), tau_e: float = 20.0, tau_i: float = 10.0,
                relax_ms: float = 0.0) -> dict:
    """Fixed point of Eq. 3: nu = phi(nu, c) with c on its nullcline
    (c = alpha_c tau_c nu), by root finding from nu0, after relaxing Eq. 3 from
    nu0 (with c on its nullcline) for `relax_ms` when given.  Returns the rates
    (Hz), fatigue (mV), the residual (Hz), whether the root finder converged,
    and the eigenvalues (1/ms) of Eq. 3's Jacobian there, over the rates and
    the fatigue of the adapting populations (stable when every real part is
    negative)."""
    from scipy.optimize import root

    def resid(x):
        nu = np.maximum(x, 0.0)
        return phi(p, nu, adapted_fatigue(p, nu)) - nu

    start = np.asarray(nu0_hz, np.float64)
    if relax_ms > 0.0:
        _, traj, _ = integrate(p, start, adapted_fatigue(p, start), relax_ms, 0.5, tau_e, tau_i)
        start = traj[-1]
    sol = root(resid, start, method="hybr")
    nu = np.maximum(sol.x, 0.0)
    c = adapted_fatigue(p, nu)
    exc = np.flatnonzero(_pop(p, "alpha_c") > 0.0)

    def rhs(state):
        nu_s = state[:3]
        c_s = np.zeros(3)
        c_s[exc] = state[3:]
        dnu, dc = eq3_rhs(p, nu_s, c_s, tau_e, tau_i)
        return np.concatenate([dnu, dc[exc]])

    x0 = np.concatenate([nu, c[exc]])
    n = x0.size
    jac = np.empty((n, n))
    for k in range(n):
        h = 1e-4 * max(1.0, abs(x0[k]))
        xp, xm = x0.copy(), x0.copy()
        xp[k] += h
        xm[k] -= h
        jac[:, k] = (rhs(xp) - rhs(xm)) / (2.0 * h)
    return {"nu_hz": nu, "c_mv": c, "residual_hz": float(np.max(np.abs(resid(nu)))),
            "eigenvalues": np.linalg.eigvals(jac), "converged": bool(sol.success)}


def rate_nullcline(p: dict, c_e: float, nu_e_grid) -> np.ndarray:
    """Points of the rate nullcline at fatigue c_e of the excitatory
    populations: the excitatory rates nu_E (Hz, applied to F and B alike) on
    the grid's sign changes of phi_E - nu_E, with the inhibitory rate solved
    self-consistently at each grid point (exact for networks whose F and B
    populations share their parameters, as the benchmark networks do)."""
    from scipy.optimize import brentq
    c = np.array([c_e, c_e, 0.0])

    def nu_i_of(nu_e):
        f = lambda x: phi(p, [nu_e, nu_e, x], c)[2] - x
        hi = 10.0
        while f(hi) > 0.0 and hi < 1e4:
            hi *= 2.0
        return brentq(f, 0.0, hi, xtol=1e-9) if f(0.0) > 0.0 else 0.0

    grid = np.asarray(nu_e_grid, np.float64)
    r = np.array([phi(p, [v, v, nu_i_of(v)], c)[0] - v for v in grid])
    out = []
    for k in np.flatnonzero(np.sign(r[:-1]) * np.sign(r[1:]) < 0):
        out.append(brentq(lambda v: phi(p, [v, v, nu_i_of(v)], c)[0] - v, grid[k], grid[k + 1], xtol=1e-9))
    return np.asarray(out)
