"""The library's statistics calls (host code, no GPU needed) against the oracle's
plain definitions, on statistics the oracle's own reduction produced:

  * aeb_stats_summary / aeb_job_stats_summary: counts exact; mean and unbiased
    standard deviation of the stopping distance and the impact speed (Sec. VI-B,
    Table I) within the rounding bound of forming them from sums; the collision
    probability exact and its Wilson interval equal to the oracle's;
  * aeb_hist_quantile: the returned bin holds the oracle's order statistic
    x_(ceil(q N)) (the safe headways of Sec. VI-C at q = 0.95, 0.99, 0.999);
  * aeb_hist_exceedance: at inner bin edges, equal to the oracle's
    P(D_stop > H0) of Eq. 19 times the valid count, exactly;
  * aeb_is_estimate: equal to the oracle's estimator on the same weights and
    events to 1e-12 relative, fed the exactly rounded sums.
"""
import math

import numpy as np
import pytest

import aeb_inputs as ai
from stat_bounds import check_summary, to_stats


@pytest.fixture(scope="module")
def aeb():
    import paper_2604_27193_gb300 as aeb
    aeb.build()
    aeb.lib()
    return aeb


WORKLOADS = {
    "single_scenario": (ai.single_model(), ai.single_scenario(seed=50), 20_000),
    "paper_preset": (ai.paper_model(), ai.paper_scenario(seed=51), 20_000),
}
SPEC = (0.0, 0.125, 0.0, 1.0 / 64.0)


@pytest.fixture(scope="module")
def runs(oracle_mod):
    res = {}
    for name, (m, sc, n) in WORKLOADS.items():
        p = oracle_mod.sample(m, sc, 0, n)
        out = oracle_mod.rollout(m, p, threads=8)
        res[name] = out
    return res


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_summary_against_oracle(aeb, oracle_mod, runs, name):
    out = runs[name]
    st = to_stats(aeb, oracle_mod.reduce(out, *SPEC), SPEC)
    check_summary(aeb, oracle_mod, out, aeb.aeb_stats_summary(st))
    js = aeb.JobStats()
    for f, _ in aeb.JobStats._fields_:
        setattr(js, f, getattr(st, f))
    a, b = aeb.aeb_stats_summary(st), aeb.aeb_job_stats_summary(js)
    assert bytes(a) == bytes(b)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_hist_quantile_holds_order_statistic(aeb, oracle_mod, runs, name):
    out = runs[name]
    st = to_stats(aeb, oracle_mod.reduce(out, *SPEC), SPEC)
    d = out["x_ref"][out["status"] == 0]
    v = out["v_imp"][out["status"] == 1]
    for which, vals in ((aeb.HIST_D, d), (aeb.HIST_V, v)):
        if len(vals) == 0:
            continue
        for q in (0.0, 0.05, 0.5, 0.95, 0.99, 0.999, 1.0):
            lo, hi = aeb.aeb_hist_quantile(st, q, which)
            x = oracle_mod.quantile(vals, q)
            assert lo <= x < hi, (which, q, lo, x, hi)
            w = st.w_d if which == aeb.HIST_D else st.w_v
            assert hi - lo == w or math.isinf(lo) or math.isinf(hi)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_hist_exceedance_equals_eq19(aeb, oracle_mod, runs, name):
    out = runs[name]
    st = to_stats(aeb, oracle_mod.reduce(out, *SPEC), SPEC)
    d = out["x_ref"][out["status"] == 0]
    v = out["v_imp"][out["status"] == 1]
    n_valid = int(np.count_nonzero(out["status"] != 255))
    for h in (0.125, 40.0, 60.0, 79.25, 100.625, 111.125, 122.75, 135.0, 511.875):
        r = aeb.aeb_hist_exceedance(st, h, aeb.HIST_D)
        assert r.n == n_valid
        assert r.k == int(np.count_nonzero(d > h))
        assert r.p == oracle_mod.exceedance(d, h, n_valid)
        lo, hi = oracle_mod.wilson(r.k, n_valid)
        assert abs(r.ci_lo - lo) <= 1e-15 and abs(r.ci_hi - hi) <= 1e-15
    for h in (1.0, 5.0, 10.0 + 1.0 / 64.0, 20.0):
        r = aeb.aeb_hist_exceedance(st, h, aeb.HIST_V)
        assert r.k == int(np.count_nonzero(v > h))
        assert r.p == oracle_mod.exceedance(v, h, n_valid)


def test_hist_calls_reject_bad_arguments(aeb, oracle_mod, runs):
    out = runs["single_scenario"]
    st = to_stats(aeb, oracle_mod.reduce(out, *SPEC), SPEC)
    for h in (0.0, 0.1, 512.0, -3.0, float("nan"), float("inf")):  # not an inner edge
        with pytest.raises(aeb.AebError) as e:
            aeb.aeb_hist_exceedance(st, h, aeb.HIST_D)
        assert e.value.code == aeb.EINVAL
    for q in (-0.01, 1.01, float("nan")):
        with pytest.raises(aeb.AebError):
            aeb.aeb_hist_quantile(st, q)
    with pytest.raises(aeb.AebError):
        aeb.aeb_hist_quantile(st, 0.5, 7)
    empty = aeb.empty_stats(aeb.hist_spec())
    with pytest.raises(aeb.AebError):
        aeb.aeb_hist_quantile(empty, 0.5)
    bad = to_stats(aeb, oracle_mod.reduce(out, *SPEC), SPEC)
    bad.hist_d[7] += 1  # bins no longer add up to n_stop
    with pytest.raises(aeb.AebError):
        aeb.aeb_hist_quantile(bad, 0.5)
    bad = to_stats(aeb, oracle_mod.reduce(out, *SPEC), SPEC)
    bad.n += 1  # counts no longer add up to n
    with pytest.raises(aeb.AebError):
        aeb.aeb_stats_summary(bad)


def test_quantile_end_bins_are_open(aeb, oracle_mod):
    """Values beyond the histogram's range sit in its end bins, so a quantile
    found there is bounded by +-inf on that side."""
    out = {"status": np.zeros(5, np.uint8), "x_ref": np.array([-5.0, -1.0, 3.0, 600.0, 700.0]),
           "v_imp": np.zeros(5), "n_steps": np.ones(5, np.int32)}
    st = to_stats(aeb, oracle_mod.reduce(out, *SPEC), SPEC)
    assert aeb.aeb_hist_quantile(st, 0.2) == (-math.inf, 0.125)
    assert aeb.aeb_hist_quantile(st, 0.5) == (3.0, 3.125)
    assert aeb.aeb_hist_quantile(st, 1.0) == (511.875, math.inf)


def test_summary_small_sets(aeb, oracle_mod):
    out = {"status": np.array([0, 1, 2, 255], np.uint8), "x_ref": np.array([10.0, 60.0, 5.0, np.nan]),
           "v_imp": np.array([0.0, 3.5, 0.0, np.nan]), "n_steps": np.array([4, 5, 6, 0], np.int32)}
    st = to_stats(aeb, oracle_mod.reduce(out, *SPEC), SPEC)
    sm = aeb.aeb_stats_summary(st)
    assert sm.mean_d == 10.0 and math.isnan(sm.std_d) and sm.mean_v == 3.5
    assert sm.n_valid == 3 and sm.p_contact == 1 / 3 and sm.steps == 15
    sm = aeb.aeb_stats_summary(aeb.empty_stats())
    assert sm.n == 0 and math.isnan(sm.mean_d) and math.isnan(sm.p_contact)
    assert (sm.p_contact_lo, sm.p_contact_hi) == (0.0, 1.0)


def test_is_estimate_against_oracle(aeb, oracle_mod):
    """The library's estimator on the exactly rounded weighted sums equals the
    oracle's on the weights and events, to 1e-12 relative (the only
    difference is the order of the final operations)."""
    m = ai.paper_model()
    nominal = ai.paper_scenario(seed=60)
    proposal = ai.rare_event_proposal(nominal)
    cols, w = oracle_mod.sample_is(m, nominal, proposal, 0, 20_000)
    out = oracle_mod.rollout(m, cols, threads=8)
    valid = out["status"] != 255
    for thr in (100.0, 120.0, 135.0):
        ev = valid & ((out["status"] == 1) | (out["x_ref"] > thr))
        p, se, (lo, hi) = oracle_mod.is_estimate(w, ev)
        y = np.where(ev, w, 0.0)
        ws = aeb.WStats(len(w), int(valid.sum()), int(ev.sum()), math.fsum(w[valid]),
                        math.fsum(w[valid] ** 2), math.fsum(y), math.fsum(y * y))
        r = aeb.aeb_is_estimate(ws)
        assert r.n == len(w) and r.n_event == int(ev.sum())
        for a, b in ((r.p, p), (r.se, se), (r.ci_lo, lo), (r.ci_hi, hi)):
            assert abs(a - b) <= 1e-12 * abs(b), (thr, a, b)
    one = aeb.aeb_is_estimate(aeb.WStats(1, 1, 1, 2.0, 4.0, 2.0, 4.0))
    assert one.p == 2.0 and math.isnan(one.se)
    with pytest.raises(aeb.AebError):
        aeb.aeb_is_estimate(aeb.WStats(10, 5, 6, 1.0, 1.0, 1.0, 1.0))
