"""The FP32 parity checker itself, on the CPU: planted disagreements made with
the oracle stand in for the binary32 kernel's outputs.

  * the oracle run with its TTC threshold scaled by 1 -+ 1e-6 moves the
    trigger margin by ~6e-5 m, inside the tie band eps (~1e-4 m here), so
    every onset disagreement it causes is proven a tie and, forced to the
    planted trigger step, the oracle reproduces the planted outputs exactly;
  * scaled by 1 -+ 1e-3 (~0.06 m, far outside eps) the checker must reject;
  * an x_raw error of 2e-5 relative and a step count two steps off must be
    rejected by the FP32 report.
"""
import numpy as np
import pytest

import aeb_inputs as ai
from fp32_bounds import fp32_report, resolve_onset_ties, with_gap

CASES = {
    "ttc_2s": (ai.ttc_model(thr=2.0), ai.single_scenario(seed=90), 20_000),
    "ttc_perception": (ai.replace(ai.ttc_model(thr=2.0), perc_sigma=0.8, perc_drop=0.2,
                                  perc_latency=0.05, perc_seed=4),
                       ai.single_scenario(seed=91), 20_000),
    "moving_lead_ttc": (ai.replace(ai.lead_braking_model(lead_decel=4.0), trigger=ai.TRIGGER_TTC,
                                   ttc_thr=3.0), ai.lead_braking_scenario(seed=92), 20_000),
}


@pytest.fixture(scope="module")
def runs(oracle_mod):
    res = {}
    for name, (m, sc, n) in CASES.items():
        p = ai.draw_params(m, sc, n)
        res[name] = (p, oracle_mod.rollout(m, p, threads=8))
    return res


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("scale", [1 + 1e-6, 1 - 1e-6])
def test_rounding_sized_trigger_shift_is_a_proven_tie(oracle_mod, runs, name, scale):
    m, _, n = CASES[name]
    p, exp = runs[name]
    planted = oracle_mod.rollout(ai.replace(m, ttc_thr=m.ttc_thr * scale), p, threads=8)
    res, (ties, worst) = resolve_onset_ties(oracle_mod, m, p, np.arange(n), planted, exp)
    assert ties > 0 and worst <= 1.0
    for k in planted:
        a, b = planted[k], res[k]
        if a.dtype == np.float64:
            a, b = a.view(np.uint64), b.view(np.uint64)
        assert np.array_equal(a, b), k
    fp32_report(m, with_gap(planted, p, m), with_gap(res, p, m), (ties, worst))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("scale", [1 + 1e-3, 1 - 1e-3])
def test_clear_trigger_shift_is_rejected(oracle_mod, runs, name, scale):
    m, _, n = CASES[name]
    p, exp = runs[name]
    planted = oracle_mod.rollout(ai.replace(m, ttc_thr=m.ttc_thr * scale), p, threads=8)
    assert np.any(planted["n_onset"] != exp["n_onset"])
    with pytest.raises(AssertionError, match="not a tie"):
        resolve_onset_ties(oracle_mod, m, p, np.arange(n), planted, exp)


def test_x_raw_and_step_errors_are_rejected(oracle_mod, runs):
    m = ai.single_model()
    p = ai.draw_params(m, ai.single_scenario(seed=93), 5_000)
    exp = with_gap(oracle_mod.rollout(m, p, threads=8), p, m)
    fp32_report(m, exp, exp)
    bad = {k: v.copy() for k, v in exp.items()}
    bad["x_raw"][17] *= 1 + 2e-5
    with pytest.raises(AssertionError):
        fp32_report(m, bad, exp)
    bad = {k: v.copy() for k, v in exp.items()}
    bad["n_steps"][23] += 2
    with pytest.raises(AssertionError):
        fp32_report(m, bad, exp)
    bad = {k: v.copy() for k, v in exp.items()}
    i = int(np.nonzero(exp["status"] == 0)[0][0])
    bad["n_steps"][i] += 1  # one step later, but the stop is not on a step boundary
    with pytest.raises(AssertionError):
        fp32_report(m, bad, exp)
