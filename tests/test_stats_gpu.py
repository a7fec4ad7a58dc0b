"""Statistics of device reductions through the C ABI against the oracle
(Sec. VI-B Table I, Sec. VI-C Eq. 19 and the safe headways, rare events):

  * binary64 rollouts and the device reduction, then aeb_hist_quantile at
    q = 0.95, 0.99, 0.999: the returned bin holds the oracle's order statistic
    (so the library's safe headway is within one bin width of it);
    aeb_hist_exceedance at bin edges equal to the oracle's P(D_stop > H0);
    aeb_stats_summary within the rounding bounds of its sums; on the
    single-scenario workload and the paper preset;
  * aeb_reduce_weighted + aeb_is_estimate on importance-sampled binary64
    rollouts: the estimate and its standard error equal the oracle's
    is_estimate on the same weights and events to 1e-12 relative (the
    device sums run at most chunk/256 + 8 + 1 + 8 additions deep, so their
    error is below 1e-14 relative; the terms are non-negative);
  * the FP32-compensated moments against the binary64 ones on the same
    samples, within the bounds the per-sample tolerances imply.
"""
import math

import numpy as np
import pytest

import aeb_inputs as ai
from stat_bounds import check_summary, moment_bounds

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def aeb():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2604_27193_gb300 as aeb
    aeb.build()
    aeb.lib()
    return aeb


def device_stats(aeb, m, cols, n, precision, spec=(0.0, 0.125, 0.0, 1.0 / 64.0)):
    P = {f: torch.from_numpy(np.ascontiguousarray(cols[f])).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(n)
    aeb.aeb_rollout(m, P, n, precision, O)
    S = aeb.alloc_stats()
    aeb.aeb_reduce(O, n, aeb.hist_spec(*spec), S)
    return {k: v.cpu().numpy() for k, v in O.items()}, aeb.stats_from_buffer(S)


WORKLOADS = {
    "single_scenario": (ai.single_model(), ai.single_scenario(seed=70), 100_000),
    "paper_preset": (ai.paper_model(), ai.paper_scenario(seed=71), 100_000),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_headways_exceedance_summary_fp64(aeb, oracle_mod, name):
    m, sc, n = WORKLOADS[name]
    cols = aeb.aeb_sample_params(m, sc, 0, n)
    exp = oracle_mod.rollout(m, cols, threads=16)
    got, st = device_stats(aeb, m, cols, n, aeb.FP64_PLAIN)
    d = exp["x_ref"][exp["status"] == 0]
    n_valid = int(np.count_nonzero(exp["status"] != 255))
    rep = {}
    for q in (0.95, 0.99, 0.999):
        lo, hi = aeb.aeb_hist_quantile(st, q)
        x = oracle_mod.quantile(d, q)
        assert lo <= x < hi and hi - lo == st.w_d, (q, lo, x, hi)
        rep[q] = (x, hi)
    for h in (60.0, 79.25, 100.625, 111.125, 122.75):
        r = aeb.aeb_hist_exceedance(st, h)
        assert r.k == int(np.count_nonzero(d > h)) and r.n == n_valid
        assert r.p == oracle_mod.exceedance(d, h, n_valid)
    check_summary(aeb, oracle_mod, exp, aeb.aeb_stats_summary(st))
    print(name, "safe headways (oracle order statistic, library bin edge):", rep)


def test_is_estimate_fp64_against_oracle(aeb, oracle_mod):
    m = ai.paper_model()
    nominal = ai.paper_scenario(seed=72)
    n = 200_000
    cols, w = aeb.aeb_sample_params_is(m, nominal, ai.rare_event_proposal(nominal), 0, n)
    exp = oracle_mod.rollout(m, cols, threads=16)
    P = {f: torch.from_numpy(cols[f]).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(n, which=("status", "x_ref"))
    aeb.aeb_rollout(m, P, n, aeb.FP64_PLAIN, O)
    W = torch.from_numpy(w).cuda()
    valid = exp["status"] != 255
    for thr in (110.0, 125.0, 135.0):
        S = torch.zeros(aeb.WSTATS_BYTES, dtype=torch.uint8, device="cuda")
        aeb.aeb_reduce_weighted(O, W, n, thr, S)
        r = aeb.aeb_is_estimate(aeb.wstats_from_buffer(S))
        ev = valid & ((exp["status"] == 1) | (exp["x_ref"] > thr))
        p, se, (lo, hi) = oracle_mod.is_estimate(w, ev)
        assert r.n_event == int(ev.sum()) and r.n_event > 50
        for a, b in ((r.p, p), (r.se, se), (r.ci_lo, lo), (r.ci_hi, hi)):
            assert abs(a - b) <= 1e-12 * abs(b), (thr, a, b)


def fp32_moment_errors(aeb, st32, st64, out32, out64, d0):
    """FP32 against binary64 moments on the same samples, with the bounds that
    follow from the per-sample tolerances: over the samples that stopped in
    both, |x32 - x64| <= 1e-5 x64, so |d mean_d| <= 1e-5 mean(x64) and
    |d std_d| <= 1e-5 rms(x64) sqrt(k / (k - 1)) (the spread of the
    perturbation); per contact, |d v_imp| v_imp <= 1e-4 d0, so
    |d mean_v| <= mean(1e-4 d0 / v_imp).  Samples whose flag differs (counted)
    move the means by at most their share times the range.  Rounding of the
    sums (moment_bounds) is added."""
    a, b = aeb.aeb_stats_summary(st32), aeb.aeb_stats_summary(st64)
    s32, s64 = out32["status"], out64["status"]
    flag = int(np.count_nonzero(s32 != s64))
    x64 = out64["x_ref"][s64 == 0]
    v64 = out64["v_imp"][s64 == 1]
    k, kv = len(x64), len(v64)
    dm, dsd = moment_bounds(x64)
    share = flag / max(k, 1)
    rng_d = float(x64.max() - x64.min()) if k else 0.0
    bound_mean_d = 1e-5 * float(x64.mean()) + share * rng_d + 2 * dm
    bound_std_d = 1e-5 * math.sqrt(float(np.mean(x64 * x64)) * k / (k - 1)) + share * rng_d + 2 * dsd
    dmv, _ = moment_bounds(v64) if kv > 1 else (0.0, 0.0)
    d0c = d0[s64 == 1]
    bound_mean_v = float(np.mean(1e-4 * d0c / np.maximum(v64, 1e-12))) + flag / max(kv, 1) * (
        float(v64.max()) if kv else 0.0) + 2 * dmv
    rep = {"flag_disagree": flag,
           "sum_d_rel": abs(st32.sum_d - st64.sum_d) / abs(st64.sum_d),
           "mean_d_rel": abs(a.mean_d - b.mean_d) / b.mean_d,
           "std_d_rel": abs(a.std_d - b.std_d) / b.std_d,
           "mean_v_rel": abs(a.mean_v - b.mean_v) / b.mean_v if kv else 0.0,
           "p_contact_abs": abs(a.p_contact - b.p_contact)}
    assert abs(a.mean_d - b.mean_d) <= bound_mean_d, (rep, bound_mean_d)
    assert abs(a.std_d - b.std_d) <= bound_std_d, (rep, bound_std_d)
    if kv:
        assert abs(a.mean_v - b.mean_v) <= bound_mean_v, (rep, bound_mean_v)
    assert abs(a.p_contact - b.p_contact) * a.n_valid <= flag
    return rep


@pytest.mark.parametrize("name,n", [("single_scenario", 200_000), ("paper_preset", 200_000)])
def test_fp32_moments_against_fp64(aeb, name, n):
    m, sc, _ = WORKLOADS[name]
    cols = aeb.aeb_sample_params(m, sc, 0, n)
    out64, st64 = device_stats(aeb, m, cols, n, aeb.FP64_PLAIN)
    out32, st32 = device_stats(aeb, m, cols, n, aeb.FP32_COMP)
    rep = fp32_moment_errors(aeb, st32, st64, out32, out64, cols["d0"])
    print(name, rep)
