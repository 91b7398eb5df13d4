"""Activity analysis of Sec. 2.3 (host, FP64): Eq. 4 wavefront speed against
closed forms, and the log-MUA / Up-Down / wave pipeline on synthetic rasters
with a known planar wave."""
import math

import numpy as np
import pytest

from paper_1902_08410_gb300 import analysis as A


@pytest.mark.parametrize("theta", [0.0, 0.3, math.pi / 4, 2.0])
def test_planar_wavefront_speed_exact(theta):
    """T = (x cos th + y sin th) / v has |grad T| = 1 / v everywhere (central
    and one-sided differences are exact on a linear field)."""
    v = 37.5
    y, x = np.mgrid[0:9, 0:13].astype(np.float64)
    T = (x * math.cos(theta) + y * math.sin(theta)) / v
    assert A.wave_speed(T) == pytest.approx(v, rel=1e-12)
    assert A.wave_speed(T, imd=0.4) == pytest.approx(0.4 * v, rel=1e-12)


def test_radial_wavefront_speed():
    """T = r / v from a point source: |grad r| = 1 away from the source, so the
    mean of Eq. 4 over the grid is v up to the few positions next to it."""
    v = 20.0
    y, x = np.mgrid[0:41, 0:41].astype(np.float64)
    T = np.hypot(x - 20.0, y - 20.0) / v
    assert A.wave_speed(T) == pytest.approx(v, rel=0.03)


def test_missing_positions_are_left_out():
    v = 10.0
    y, x = np.mgrid[0:8, 0:8].astype(np.float64)
    T = x / v
    T[3, 4] = np.nan
    s = A.wave_speed(T)
    assert np.isfinite(s) and s == pytest.approx(v, rel=1e-12)


def _planar_wave_counts(gx, gy, v, period_s, up_s, n_waves, bin_s, up_hz, down_hz, seed):
    rng = np.random.default_rng(seed)
    nb = int(round((n_waves + 1) * period_s / bin_s))
    t = (np.arange(nb) + 0.5) * bin_s
    y, x = np.mgrid[0:gy, 0:gx]
    rate = np.full((nb, gy * gx), down_hz)
    onsets = []
    for w in range(n_waves):
        t0 = (w + 0.5) * period_s
        T = t0 + x.ravel() / v
        onsets.append(T.reshape(gy, gx))
        on = (t[:, None] >= T[None, :]) & (t[:, None] < T[None, :] + up_s)
        rate[on] = up_hz
    lam = rate * A.K * bin_s
    counts = np.zeros((nb, gy * gx, 3), np.uint32)
    counts[:, :, 1] = rng.poisson(lam)
    return counts, onsets


def test_slow_wave_pipeline_recovers_planar_wave():
    """Poisson spike counts of Up states (20 Hz) sweeping a 16 x 10 grid at 40
    modules/s over a 0.3 Hz Down background: every wave is found, each module's
    Down-to-Up time is, for 99% of the modules, within three 5 ms bins of the
    true onset, and the mean Eq. 4 speed is within 5% of 40."""
    bin_s, v = 0.005, 40.0
    counts, onsets = _planar_wave_counts(16, 10, v, 2.0, 0.3, 4, bin_s, 20.0, 0.3, seed=3)
    mua = A.module_mua(counts, bin_s)
    lm, thr, down = A.log_mua(mua, bin_s, noise_var=0.5, seed=1)
    assert np.all(np.abs(down - 0.3) < 0.1)
    up = A.up_states(lm, thr)
    ws = A.waves(A.down_to_up_times(up, bin_s), 16, 10)
    assert len(ws) == 4
    for T, T0 in zip(ws, onsets):
        assert np.all(np.isfinite(T))
        err = np.abs(T - T0)
        assert np.median(err) <= bin_s + 1e-12
        assert np.mean(err <= 3 * bin_s + 1e-12) >= 0.99
    out = A.slow_wave_speeds(counts, 16, 10, bin_s)
    assert out["waves"] == 4
    assert out["mean_speed"] == pytest.approx(v, rel=0.05)
    assert out["up_fraction"] == pytest.approx(4 * 0.3 / (5 * 2.0), abs=0.01)


def test_back_to_back_waves_are_separated():
    """Waves every 0.4 s that each take 0.375 s to cross the grid leave no
    quiet gap between them; each module transits once per wave, so every wave
    is still found on its own, with its speed."""
    bin_s, v = 0.005, 40.0
    counts, onsets = _planar_wave_counts(16, 10, v, 0.4, 0.15, 10, bin_s, 20.0, 0.3, seed=4)
    mua = A.module_mua(counts, bin_s)
    lm, thr, _ = A.log_mua(mua, bin_s, noise_var=0.5, seed=2)
    ws = A.waves(A.down_to_up_times(A.up_states(lm, thr), bin_s), 16, 10)
    assert len(ws) == 10
    for T, T0 in zip(ws, onsets):
        assert np.median(np.abs(T - T0)) <= bin_s + 1e-12
    assert A.slow_wave_speeds(counts, 16, 10, bin_s)["mean_speed"] == pytest.approx(v, rel=0.05)


def test_asynchronous_activity_has_no_collective_waves():
    """Stationary Poisson firing (no Up/Down alternation) yields no wave that
    reaches half the modules."""
    rng = np.random.default_rng(5)
    counts = np.zeros((2000, 64, 3), np.uint32)
    counts[:, :, 1] = rng.poisson(8.0 * A.K * 0.005, size=(2000, 64))
    out = A.slow_wave_speeds(counts, 8, 8, 0.005)
    assert out["waves"] == 0 and out["mean_speed"] is None


def test_dominant_frequency_of_modulated_rate():
    """Welch PSD peak of a rate modulated at 1.5 Hz, sampled in 5 ms bins."""
    rng = np.random.default_rng(2)
    bin_s = 0.005
    t = np.arange(20000) * bin_s
    lam = 400.0 * (1.0 + 0.8 * np.sin(2 * np.pi * 1.5 * t))
    counts = np.zeros((t.size, 4, 3), np.uint32)
    counts[:, 0, 0] = rng.poisson(lam)
    f = A.dominant_frequency(counts, bin_s)
    assert abs(f - 1.5) <= 1.0 / (512 * bin_s)
