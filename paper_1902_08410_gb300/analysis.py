"""Activity analysis of recorded networks (host, FP64, off the per-step path).

Sec. 2.3 of the paper: module firing rates are sampled in 5 ms bins; power
spectra use Welch's method; a module's multi-unit activity (MUA) is its mean
firing rate, analysed as log(MUA / MUA_down) plus zero-mean white noise of
variance 0.5; for slow-wave activity the Down-to-Up transition time T(x, y) of
every module defines the wavefront, whose local speed is Eq. 4,
V = 1 / |grad T|, averaged over all positions.

Readings where the paper leaves the procedure open:
  * log of a rate that can be zero: the rates are offset by one spike per bin
    (1 / (K * bin) Hz) before the logarithm, in numerator and denominator.
  * MUA_down and the threshold: per module, a two-cluster split (k-means on
    log rate, started at the 10th and 90th percentiles); MUA_down is the mean
    rate of the lower cluster and the threshold sits midway between the two
    cluster centres, in log(MUA / MUA_down) units.  A module whose cluster
    centres lie less than `min_sep` (1.0, a factor e in rate) apart is not
    bistable: it has no Up states.
  * Up and Down states are the threshold crossings of the noisy log-MUA,
    cleaned in three passes: single-bin Up flickers are dropped, then Down
    runs shorter than `min_down_bins` (dips inside an Up state) and Up runs
    shorter than `min_up_bins` (both 20 ms) are merged into the surrounding
    state.
  * A wave is a collective Down-to-Up transition: the transitions of all
    modules, in time order, are cut into waves wherever consecutive ones are
    more than `gap_s` apart or a module would take part twice (each module
    transits at most once per wave); waves that reach fewer than half of the
    modules are dropped.
  * grad T by central differences in the interior and one-sided differences
    at the open boundary (numpy.gradient), in units of the inter-module
    distance; positions where the gradient vanishes or T is missing are left
    out of the average.
"""
from __future__ import annotations

import numpy as np

K = 1250                 # neurons per module (Sec. 2.1)


def module_mua(counts: np.ndarray, bin_s: float) -> np.ndarray:
    """Mean firing rate (Hz) of each module per bin from the integer counters
    [bin][module][population]: returns [bin][module]."""
    c = np.asarray(counts, dtype=np.float64)
    return c.sum(axis=2) / (K * bin_s)


def dominant_frequency(counts: np.ndarray, bin_s: float, f_lo: float = 0.2, f_hi: float = 10.0,
                       skip_frac: float = 0.1) -> float | None:
    """Peak of the Welch power spectrum of the whole-network rate in [f_lo, f_hi]
    Hz, after dropping the first `skip_frac` of the record (initial transient)."""
    from scipy.signal import welch
    x = np.asarray(counts, dtype=np.float64).sum(axis=(1, 2))
    x = x[int(len(x) * skip_frac):]
    if len(x) < 8:
        return None
    x = x - x.mean()
    f, pxx = welch(x, fs=1.0 / bin_s, nperseg=min(len(x), 512))
    band = (f >= f_lo) & (f <= f_hi)
    return float(f[band][np.argmax(pxx[band])]) if band.any() else None


def _two_means(y: np.ndarray, iters: int = 50) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Two-cluster split (k-means, k = 2) of every column of y [sample][column]:
    (low centres, high centres, is_high)."""
    lo, hi = np.percentile(np.ascontiguousarray(y.T), [10.0, 90.0], axis=1)
    flat = hi <= lo
    is_hi = (y > 0.5 * (lo + hi)) & ~flat
    for _ in range(iters):
        n_hi = is_hi.sum(axis=0)
        n_lo = y.shape[0] - n_hi
        ok = (n_hi > 0) & (n_lo > 0)
        s_hi = np.where(is_hi, y, 0.0).sum(axis=0)
        s_all = y.sum(axis=0)
        lo = np.where(ok, (s_all - s_hi) / np.maximum(n_lo, 1), lo)
        hi = np.where(ok, s_hi / np.maximum(n_hi, 1), hi)
        nxt = (y > 0.5 * (lo + hi)) & ~flat & ok
        if np.array_equal(nxt, is_hi & ok):
            is_hi = nxt
            break
        is_hi = nxt
    return lo, hi, is_hi


def log_mua(mua: np.ndarray, bin_s: float, noise_var: float = 0.5, seed: int | None = 0,
            min_sep: float = 1.0):
    """log(MUA / MUA_down) per module with white noise of variance `noise_var`
    added (None seed or zero variance: no noise).  Returns (log_mua [bin][module],
    threshold [module], inf where the module is not bistable, mua_down [module])."""
    mua = np.asarray(mua, dtype=np.float64)
    eps = 1.0 / (K * bin_s)
    nm = mua.shape[1]
    out = np.empty_like(mua)
    thr = np.empty(nm)
    down = np.empty(nm)
    rng = np.random.default_rng(seed) if (seed is not None and noise_var > 0) else None
    lo, hi, is_hi = _two_means(np.log(mua + eps))
    n_lo = (~is_hi).sum(axis=0)
    down[:] = np.where(n_lo > 0, np.where(is_hi, 0.0, mua).sum(axis=0) / np.maximum(n_lo, 1), mua.mean(axis=0))
    out[:] = np.log((mua + eps) / (down + eps))
    thr[:] = np.where(hi - lo >= min_sep, 0.5 * (hi - lo), np.inf)
    if rng is not None:
        out += rng.normal(0.0, np.sqrt(noise_var), size=out.shape)
    return out, thr, down


def up_states(lmua: np.ndarray, thr: np.ndarray, min_up_bins: int = 4, min_down_bins: int = 4) -> np.ndarray:
    """Boolean Up state per bin and module: log-MUA above the module's
    threshold; interior single-bin Up runs, then Down runs shorter than
    `min_down_bins`, then Up runs shorter than `min_up_bins`, are merged into
    their neighbours."""
    up = np.asarray(lmua) > np.asarray(thr)[None, :]
    up = up.copy()
    for m in np.flatnonzero(up.any(axis=0)):
        u = up[:, m]
        for state, min_len in ((True, 2), (False, min_down_bins), (True, min_up_bins)):
            edges = np.flatnonzero(np.diff(u.astype(np.int8))) + 1
            starts = np.concatenate(([0], edges))
            ends = np.concatenate((edges, [len(u)]))
            for s, e in zip(starts, ends):
                if u[s] == state and e - s < min_len and s > 0 and e < len(u):
                    u[s:e] = not state
        up[:, m] = u
    return up


def down_to_up_times(up: np.ndarray, bin_s: float) -> list[np.ndarray]:
    """Per module, the times (s, start of the first Up bin) of its Down-to-Up
    transitions."""
    up = np.asarray(up)
    return [(np.flatnonzero(~up[:-1, m] & up[1:, m]) + 1) * bin_s for m in range(up.shape[1])]


def waves(times: list[np.ndarray], gx: int, gy: int, gap_s: float = 0.05,
          min_frac: float = 0.5) -> list[np.ndarray]:
    """Collective Down-to-Up transitions: list of T[y][x] (s, NaN where a module
    took no part), one per wave reaching at least `min_frac` of the modules."""
    ev_t = np.concatenate([np.asarray(t, np.float64) for t in times]) if times else np.zeros(0)
    ev_m = np.concatenate([np.full(len(t), m) for m, t in enumerate(times)]) if times else np.zeros(0, int)
    if ev_t.size == 0:
        return []
    order = np.argsort(ev_t, kind="stable")
    ev_t, ev_m = ev_t[order], ev_m[order]
    out = []
    T = np.full(gx * gy, np.nan)

    def close(T):
        if np.count_nonzero(~np.isnan(T)) >= min_frac * gx * gy:
            out.append(T.reshape(gy, gx))

    for i in range(ev_t.size):
        if i > 0 and (ev_t[i] - ev_t[i - 1] > gap_s or not np.isnan(T[ev_m[i]])):
            close(T)
            T = np.full(gx * gy, np.nan)
        T[ev_m[i]] = ev_t[i]
    close(T)
    return out


def wave_speed(T: np.ndarray, imd: float = 1.0) -> float:
    """Eq. 4: mean over positions of V = 1 / |grad T| for one wavefront T[y][x]
    (s), in units of `imd` per second (imd = inter-module distance)."""
    T = np.asarray(T, dtype=np.float64)
    if T.shape[0] < 2 or T.shape[1] < 2:
        return float("nan")
    gy_, gx_ = np.gradient(T)                 # per inter-module distance
    g = np.hypot(gx_, gy_)
    ok = np.isfinite(g) & (g > 0)
    if not ok.any():
        return float("nan")
    return float(np.mean(imd / g[ok]))


def slow_wave_speeds(counts: np.ndarray, gx: int, gy: int, bin_s: float, imd: float = 1.0,
                     noise_var: float = 0.5, seed: int | None = 0, skip_s: float = 0.0) -> dict:
    """Whole analysis of Sec. 2.3 on a recorded network: log-MUA, Up/Down
    states, wavefronts and their mean speeds (Eq. 4).  `counts` are the
    network's rate counters [bin][module][population].  `waves` counts the
    collective transitions found, `timed_waves` those with a finite speed (a
    wavefront that reaches every module within one bin has none)."""
    c = np.asarray(counts)[int(round(skip_s / bin_s)):]
    mua = module_mua(c, bin_s)
    lm, thr, down = log_mua(mua, bin_s, noise_var, seed)
    up = up_states(lm, thr)
    times = down_to_up_times(up, bin_s)
    ws = waves(times, gx, gy)
    speeds = [wave_speed(T, imd) for T in ws]
    speeds = [s for s in speeds if np.isfinite(s)]
    return {"waves": len(ws), "timed_waves": len(speeds),
            "mean_speed": float(np.mean(speeds)) if speeds else None,
            "sd_speed": float(np.std(speeds)) if speeds else None,
            "transitions_per_module_s": float(sum(len(t) for t in times)) / (up.shape[1] * up.shape[0] * bin_s)
            if up.size else 0.0,
            "up_fraction": float(up.mean()) if up.size else 0.0, "mua_down_hz": float(np.mean(down))}
