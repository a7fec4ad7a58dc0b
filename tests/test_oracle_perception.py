"""Pins of the oracle's per-step perception of the TTC trigger (extension:
noise, dropout and latency of the readings): each reading against numpy's
independent Philox-4x64-10, the noise against the exact Irwin-Hall CDF, the
dropout frequency, the trigger step of a coasting car against a brute-force
search over numpy-drawn readings, and the latency shift."""
import math

import numpy as np
import pytest
from scipy import stats

import aeb_inputs as ai
from test_oracle_rng import numpy_philox_block

PERC_KEY1 = 0x5045524345505431  # "PERCEPT1"
TWO_M32 = 2.0 ** -32


def numpy_reading(m, row, k):
    """(present, noise) of the reading of step k from numpy's Philox: block
    (row, k // 2, 0, 0); even k takes the words' high 32-bit halves, odd k
    the low halves."""
    w = numpy_philox_block([row, k // 2, 0, 0], [m.perc_seed, PERC_KEY1])
    h = [(int(x) >> 32) if k % 2 == 0 else (int(x) & 0xFFFFFFFF) for x in w]
    u = [float(x) * TWO_M32 for x in h]
    if u[3] < m.perc_drop:
        return False, 0.0
    return True, m.perc_sigma * (2.0 * (((u[0] + u[1]) + u[2]) - 1.5))


def irwin_hall3_cdf(s):
    s = np.clip(s, 0.0, 3.0)
    return np.where(s <= 1, s ** 3 / 6,
                    np.where(s <= 2, (-2 * s ** 3 + 9 * s ** 2 - 9 * s + 3) / 6,
                             1 - (3 - s) ** 3 / 6))


def test_readings_match_numpy_philox(oracle_mod):
    m = ai.Model(trigger=ai.TRIGGER_TTC, perc_sigma=0.7, perc_drop=0.25, perc_seed=991)
    rng = np.random.default_rng(5)
    for row, k in [(0, 0), (0, 1), (0, 2), (0, 3), (1, 0), (2 ** 40, 17), (5, 2 ** 33 + 1)] + [
            (int(r), int(k)) for r, k in zip(rng.integers(0, 2 ** 40, 60), rng.integers(0, 10 ** 6, 60))]:
        assert oracle_mod.perception(m, row, k) == numpy_reading(m, row, k), (row, k)


def test_paired_readings_are_independent(oracle_mod):
    """Readings 2j and 2j + 1 share a block but not its bits: across many
    pairs their noises are uncorrelated and each pair differs."""
    m = ai.Model(trigger=ai.TRIGGER_TTC, perc_sigma=1.0, perc_drop=0.0, perc_seed=12)
    a = np.array([oracle_mod.perception(m, 3, 2 * j)[1] for j in range(4000)])
    b = np.array([oracle_mod.perception(m, 3, 2 * j + 1)[1] for j in range(4000)])
    assert np.all(a != b)
    assert abs(np.corrcoef(a, b)[0, 1]) < 4.5 / math.sqrt(len(a))


def test_noise_distribution_and_dropout(oracle_mod):
    m = ai.Model(trigger=ai.TRIGGER_TTC, perc_sigma=1.0, perc_drop=0.2, perc_seed=3)
    draws = [oracle_mod.perception(m, row, k) for row in range(40) for k in range(500)]
    present = np.array([p for p, _ in draws])
    noise = np.array([x for p, x in draws if p])
    n = len(draws)
    # dropout: binomial(n, 0.2) within 4.5 standard deviations
    assert abs((~present).sum() - 0.2 * n) < 4.5 * math.sqrt(n * 0.2 * 0.8)
    # noise: zero mean, unit variance, bounded by 3, Irwin-Hall(3) shape
    assert np.all(np.abs(noise) <= 3.0)
    assert abs(noise.mean()) < 4.5 / math.sqrt(len(noise))
    assert abs(noise.var() - 1.0) < 0.05
    ks = stats.kstest(noise / 2.0 + 1.5, irwin_hall3_cdf)
    assert ks.pvalue > 1e-3, ks


def coasting(v0, d0, bias):
    """Coasting ego cars (no drag, flat road, no reaction delay)."""
    g = 9.81
    n = len(v0)
    return {"v0": np.asarray(v0, float), "d0": np.asarray(d0, float), "mu": np.full(n, 0.8),
            "gs": np.zeros(n), "gc": np.full(n, g), "mass": np.full(n, 1500.0),
            "cd": np.zeros(n), "tau": np.zeros(n), "t_delay": np.zeros(n),
            "noise": np.asarray(bias, float)}


def brute_force_trigger(m, row, v0, d0, bias, lat):
    """First step n whose reading (taken at step n + lat) is present and gives
    ((d0 - x_n) + bias) + noise <= thr v0, with x_n the constant-speed RK4
    positions (exact kinematics of a coasting car)."""
    dt = m.dt
    h6 = dt / 6.0
    x = 0.0
    for n in range(int(round(m.t_max / dt))):
        present, noise = numpy_reading(m, row, n + lat)
        if present and ((d0 - x) + bias) + noise <= m.ttc_thr * v0:
            return n
        x = x + h6 * (((v0 + 2.0 * v0) + 2.0 * v0) + v0)
    return None


@pytest.mark.parametrize("latency", [0.0, 0.0304])
def test_trigger_step_against_numpy(oracle_mod, latency):
    m = ai.Model(trigger=ai.TRIGGER_TTC, ttc_thr=2.0, perc_sigma=1.5, perc_drop=0.35,
                 perc_latency=latency, perc_seed=4242, t_max=6.0)
    rng = np.random.default_rng(7)
    n = 12
    v0, d0, bias = rng.uniform(15, 30, n), rng.uniform(60, 120, n), rng.normal(0, 0.5, n)
    p = coasting(v0, d0, bias)
    o = oracle_mod.rollout(m, p)
    lat = math.ceil(latency / m.dt - 1e-12)
    for i in range(n):
        nt = brute_force_trigger(m, i, v0[i], d0[i], bias[i], lat)
        assert nt is not None
        assert o["n_onset"][i] == nt + lat, (i, o["n_onset"][i], nt, lat)


def test_latency_shifts_the_onset(oracle_mod):
    """Without noise or dropout a latency of L steps delays the onset by L."""
    base = ai.Model(trigger=ai.TRIGGER_TTC, ttc_thr=1.5, t_max=8.0)
    p = ai.draw_params(base, ai.single_scenario(seed=71), 200)
    o0 = oracle_mod.rollout(base, p)
    o1 = oracle_mod.rollout(ai.replace(base, perc_latency=0.0371), p)
    fired = o0["n_onset"] >= 0
    assert fired.sum() > 150
    assert np.array_equal(o1["n_onset"][fired], o0["n_onset"][fired] + 38)


def test_no_perception_is_the_plain_trigger(oracle_mod):
    """All perception settings at zero (any seed): the plain TTC trigger, bit for bit."""
    m = ai.ttc_model(thr=2.0)
    p = ai.draw_params(m, ai.single_scenario(seed=72), 300)
    a = oracle_mod.rollout(m, p)
    b = oracle_mod.rollout(ai.replace(m, perc_seed=12345), p)
    for k in a:
        assert np.array_equal(np.asarray(a[k]).view(np.uint8), np.asarray(b[k]).view(np.uint8)), k


def test_readings_follow_the_row_not_the_thread_split(oracle_mod):
    """A sample's readings are keyed by its parameter row, so splitting the
    rows over threads changes nothing."""
    m = ai.replace(ai.ttc_model(thr=2.0), perc_sigma=0.8, perc_drop=0.2, perc_latency=0.05,
                   perc_seed=11)
    p = ai.draw_params(m, ai.single_scenario(seed=21), 999)
    a = oracle_mod.rollout(m, p, threads=1)
    b = oracle_mod.rollout(m, p, threads=7)
    for k in a:
        assert np.array_equal(np.asarray(a[k]).view(np.uint8), np.asarray(b[k]).view(np.uint8)), k
