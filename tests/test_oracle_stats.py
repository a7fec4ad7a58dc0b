"""Pins of the oracle's reductions (Sec. VI-B, VI-C) and of the model as a whole
against the statistics the paper prints (Table I, Sec. VI-B, VI-C)."""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

import aeb_inputs as ai

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_statistics.json")


@pytest.fixture(scope="module")
def paper_run(oracle_mod):
    m, sc = ai.paper_model(), ai.paper_scenario(seed=0)
    n = 200_000
    p = oracle_mod.sample(m, sc, 0, n)
    return oracle_mod.rollout(m, p, threads=os.cpu_count() or 1)


def test_paper_statistics(paper_run, oracle_mod):
    """Eq. 11-15 with the Sec. IV-B constants must land on the printed
    convergence values.  Bands are the printed range widened by sampling error;
    the alternative readings of Eq. 5 (sign flipped, mu g cap, no cap) give
    means near 78.6-78.7 m and fail the mean band."""
    gold = json.load(open(GOLDEN))
    d = paper_run["x_ref"][paper_run["status"] != 255]
    n = len(d)
    mean, sd = d.mean(), d.std(ddof=1)
    se_mean = sd / math.sqrt(n)
    lo, hi = gold["mean_range_m"]
    assert lo - 4 * se_mean <= mean <= hi + 4 * se_mean, mean
    se_sd = sd / math.sqrt(2 * n) * 2.0  # skewed: widened
    lo, hi = gold["std_range_m"]
    assert lo - 4 * se_sd <= sd <= hi + 4 * se_sd, sd
    # safe headways at 5 % and 1 % risk (Sec. VI-C), against the N = 12,000
    # sampling error of the printed values
    for key, q in (("headway_5pct_m", 0.95), ("headway_1pct_m", 0.99)):
        x = oracle_mod.quantile(d, q)
        dens = stats.gaussian_kde(d[::20])(x)[0]
        se = math.sqrt(q * (1 - q) / gold["n_distribution"]) / dens
        assert abs(x - gold[key]) <= 3 * se, (key, x, se)
    # printed range of the N = 12,000 run lies inside ours at N = 200,000
    assert d.min() <= gold["range_m"][0] + 2 and d.max() >= gold["range_m"][1] - 2


def test_paper_mode_raw_equals_refined_to_step(paper_run):
    """The paper's D_stop = x(t_stop) on the grid (Eq. 3) is within one step of
    travel of the refined stopping point.  In the last step the speed is below
    one step's change of speed (<= 10 m/s^2 * dt), so |x_{n+1} - x_n| <= 1e-5 m
    and the refined point lies on that chord."""
    s = paper_run["status"] == 0
    diff = paper_run["x_ref"][s] - paper_run["x_raw"][s]
    assert np.all(np.abs(diff) <= 1e-5)


def _brute(out, lo_d, w_d, lo_v, w_v, nb):
    st = out["status"]
    d = out["x_ref"][st == 0]
    v = out["v_imp"][st == 1]
    hd = np.bincount(np.clip(np.floor((d - lo_d) / w_d), 0, nb - 1).astype(np.int64), minlength=nb)
    hv = np.bincount(np.clip(np.floor((v - lo_v) / w_v), 0, nb - 1).astype(np.int64), minlength=nb)
    return d, v, hd, hv


def test_reduce_against_brute_force(oracle_mod):
    m, sc = ai.single_model(), ai.single_scenario(seed=11)
    p = ai.concat_params([ai.draw_params(m, sc, 3000, seed=1), ai.edge_params(m)])
    out = oracle_mod.rollout(m, p)
    nb = 4096
    st = oracle_mod.reduce(out, 0.0, 0.125, 0.0, 1 / 64, nb)
    d, v, hd, hv = _brute(out, 0.0, 0.125, 0.0, 1 / 64, nb)
    s = out["status"]
    assert st.n == len(s)
    assert (st.n_stop, st.n_contact, st.n_horizon, st.n_invalid) == (
        int(np.sum(s == 0)), int(np.sum(s == 1)), int(np.sum(s == 2)), int(np.sum(s == 255)))
    assert st.steps == int(out["n_steps"].astype(np.int64).sum())
    for got, vals in ((st.sum_d, d), (st.sum_v, v)):
        exact = math.fsum(vals)
        assert abs(got - exact) <= len(vals) * 2.3e-16 * math.fsum(np.abs(vals))
    assert abs(st.sumsq_d - math.fsum(d * d)) <= len(d) * 2.3e-16 * math.fsum(d * d)
    assert (st.min_d, st.max_d) == (d.min(), d.max())
    assert (st.min_v, st.max_v) == (v.min(), v.max())
    assert np.array_equal(st.hist_d, hd) and np.array_equal(st.hist_v, hv)
    assert st.hist_d.sum() == st.n_stop and st.hist_v.sum() == st.n_contact


def test_reduce_with_shifted_origins(oracle_mod):
    m, sc = ai.single_model(), ai.single_scenario(seed=12)
    out = oracle_mod.rollout(m, ai.draw_params(m, sc, 2000, seed=3))
    for lo_d, w_d, lo_v, w_v in ((20.0, 0.0625, -1.0, 0.25), (-3.5, 1.0, 2.0, 0.125)):
        st = oracle_mod.reduce(out, lo_d, w_d, lo_v, w_v, 512)
        _, _, hd, hv = _brute(out, lo_d, w_d, lo_v, w_v, 512)
        assert np.array_equal(st.hist_d, hd) and np.array_equal(st.hist_v, hv)


def test_histogram_clamps_end_bins(oracle_mod):
    out = {"status": np.zeros(4, np.uint8), "x_ref": np.array([-1.0, 0.0, 511.9, 10_000.0]),
           "v_imp": np.zeros(4), "n_steps": np.ones(4, np.int32)}
    st = oracle_mod.reduce(out, 0.0, 0.125, 0.0, 1 / 64, 4096)
    assert st.hist_d[0] == 2 and st.hist_d[4095] == 2 and st.hist_d.sum() == 4


def test_quantile_definition(oracle_mod):
    rng = np.random.default_rng(2)
    for n in (1, 2, 7, 100, 1001):
        x = rng.normal(size=n)
        for q in (0.0, 0.05, 0.5, 0.95, 0.99, 0.999, 1.0):
            assert oracle_mod.quantile(x, q) == np.quantile(x, q, method="inverted_cdf")


def test_moments_closed_forms(oracle_mod):
    """The arithmetic sequence a + d j, j = 0 .. n-1 (every value and the
    sums exact in binary64) has mean a + d (n - 1) / 2 and unbiased variance
    d^2 n (n + 1) / 12; an offset far above the spread must not disturb the
    spread (two passes)."""
    for a, d, n in ((0.0, 1.0, 2), (3.0, 0.5, 7), (-40.0, 0.25, 1000), (1e8, 1.0, 101)):
        x = a + d * np.arange(n, dtype=np.float64)
        m, sd = oracle_mod.moments(x)
        assert m == a + d * (n - 1) / 2
        assert math.isclose(sd, math.sqrt(d * d * n * (n + 1) / 12.0), rel_tol=1e-14)
    m, sd = oracle_mod.moments([5.0])
    assert m == 5.0 and math.isnan(sd)
    m, sd = oracle_mod.moments([])
    assert math.isnan(m) and math.isnan(sd)


def test_exceedance(oracle_mod):
    x = np.array([1.0, 2.0, 3.0, 4.0])
    assert oracle_mod.exceedance(x, 2.0, 4) == 0.5
    assert oracle_mod.exceedance(x, 0.0, 8) == 0.5


@pytest.mark.parametrize("k,n", [(0, 10), (3, 10), (10, 10), (37, 1000), (5000, 100000), (1, 1)])
def test_wilson_matches_scipy(oracle_mod, k, n):
    lo, hi = oracle_mod.wilson(k, n)
    ci = stats.binomtest(k, n).proportion_ci(confidence_level=0.95, method="wilson")
    assert abs(lo - ci.low) < 1e-12 and abs(hi - ci.high) < 1e-12
