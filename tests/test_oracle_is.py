"""Pins of the oracle's importance sampling (extension: rare-event estimation):
draws identical to plain sampling from the proposal, likelihood ratios against
scipy's densities and tail masses (clamp atoms included), unbiasedness, and a
rare event with an exact probability."""
import math

import numpy as np
import pytest
from scipy import stats

import aeb_inputs as ai

QFIELD = {"v0": "v0", "d0": "d0", "mu": "mu", "mass": "mass", "cd": "cd", "tau": "tau",
          "t_delay": "t_delay", "noise": "noise"}


def scipy_ratio(dp, dq, x):
    """p(x) / q(x) of one quantity with scipy's distributions."""
    if dq.kind == ai.CONST:
        return np.ones_like(x)
    if dq.kind == ai.UNIFORM:
        P = stats.uniform(dp.p0, dp.p1 - dp.p0)
        Q = stats.uniform(dq.p0, dq.p1 - dq.p0)
    else:
        P, Q = stats.norm(dp.p0, dp.p1), stats.norm(dq.p0, dq.p1)
    r = P.pdf(x) / Q.pdf(x)
    if np.isfinite(dq.lo) and Q.cdf(dq.lo) > 0:
        r = np.where(x <= dq.lo, P.cdf(dp.lo) / Q.cdf(dq.lo), r)
    if np.isfinite(dq.hi) and Q.sf(dq.hi) > 0:
        r = np.where(x >= dq.hi, P.sf(dp.hi) / Q.sf(dq.hi), r)
    return r


def nominal_and_proposal():
    p = ai.Scenario(v0=ai.normal(30.0, 2.0, 20.0, 38.0), d0=ai.const(0.0),
                    mu=ai.normal(0.8, 0.1, 0.3, 1.1), grade=ai.normal(0.0, 0.05),
                    mass=ai.uniform(1300.0, 1700.0), cd=ai.normal(0.3, 0.05),
                    tau=ai.uniform(0.1, 0.2), t_delay=ai.const(0.0), noise=ai.const(0.0), seed=9)
    q = ai.replace(p, v0=ai.normal(34.0, 2.5, 20.0, 38.0), mu=ai.normal(0.65, 0.12, 0.3, 1.1),
                   mass=ai.uniform(1250.0, 1750.0), scenario_id=4)
    return p, q


def test_draws_are_the_proposal_draws(oracle_mod):
    p, q = nominal_and_proposal()
    m = ai.paper_model()
    cols, w = oracle_mod.sample_is(m, p, q, 100, 2_000)
    plain = oracle_mod.sample(m, q, 100, 2_000)
    for f in ai.FIELDS:
        assert np.array_equal(cols[f].view(np.uint64), plain[f].view(np.uint64)), f
    assert np.all(w >= 0) and np.all(np.isfinite(w))


def test_weights_against_scipy(oracle_mod):
    p, q = nominal_and_proposal()
    m = ai.paper_model()
    cols, w = oracle_mod.sample_is(m, p, q, 0, 20_000)
    exp = np.ones(len(w))
    for name in ("v0", "d0", "mu", "mass", "cd", "tau", "t_delay", "noise"):
        exp *= scipy_ratio(getattr(p, name), getattr(q, name), cols[name])
    theta = np.arctan2(cols["gs"], cols["gc"])
    exp *= scipy_ratio(p.grade, q.grade, theta)
    assert np.allclose(w, exp, rtol=1e-9, atol=0), np.max(np.abs(w / exp - 1))
    # the clamp atoms of v0 at 38 m/s carry probability mass under both laws
    assert np.any(cols["v0"] == 38.0)


def test_unbiased(oracle_mod):
    """E_q[w] = 1 and E_q[w v0] = E_p[v0] for the clamped nominal law."""
    p, q = nominal_and_proposal()
    cols, w = oracle_mod.sample_is(ai.paper_model(), p, q, 0, 200_000)
    n = len(w)
    assert abs(w.mean() - 1.0) < 5 * w.std() / math.sqrt(n)
    # mean of N(30, 2^2) clamped to [20, 38]
    P = stats.norm(30.0, 2.0)
    a, b = 20.0, 38.0
    za, zb = (a - 30) / 2, (b - 30) / 2
    mean_clamped = (a * P.cdf(a) + b * P.sf(b)
                    + 30 * (P.cdf(b) - P.cdf(a)) - 2 * (stats.norm.pdf(zb) - stats.norm.pdf(za)))
    y = w * cols["v0"]
    assert abs(y.mean() - mean_clamped) < 5 * y.std() / math.sqrt(n)


def test_rare_event_exact(oracle_mod):
    """P_p(v0 > 36) = P(Z > 3) for v0 ~ N(30, 2^2): the weighted estimate from
    2e4 proposal draws centred at 36 lands within 4 standard errors, with a
    standard error well below plain Monte Carlo's at the same size."""
    p = ai.Scenario(v0=ai.normal(30.0, 2.0), seed=3)
    q = ai.replace(p, v0=ai.normal(36.0, 2.0), scenario_id=1)
    cols, w = oracle_mod.sample_is(ai.paper_model(), p, q, 0, 20_000)
    est, se, (lo, hi) = oracle_mod.is_estimate(w, cols["v0"] > 36.0)
    exact = stats.norm.sf(3.0)
    assert abs(est - exact) < 4 * se
    assert lo < exact < hi or abs(est - exact) < 4 * se
    se_plain = math.sqrt(exact * (1 - exact) / 20_000)
    assert se < se_plain / 10


def test_incompatible_proposal_rejected(oracle_mod):
    p, q = nominal_and_proposal()
    with pytest.raises(ValueError):
        oracle_mod.sample_is(ai.paper_model(), p, ai.replace(q, mass=ai.uniform(1400.0, 1700.0)), 0, 10)
    with pytest.raises(ValueError):
        oracle_mod.sample_is(ai.paper_model(), p, ai.replace(q, v0=ai.normal(34.0, 2.5, 21.0, 38.0)), 0, 10)


def test_is_standard_error(oracle_mod):
    """The reported standard error is that of the mean of y = w 1[E]: equal to
    numpy's sample variance (ddof = 1) over n, and calibrated: over 200
    independent batches of the rare event above, the spread of the estimates
    matches the mean reported standard error, and the 95 % intervals cover the
    exact probability about 95 % of the time."""
    p = ai.Scenario(v0=ai.normal(30.0, 2.0), seed=3)
    q = ai.replace(p, v0=ai.normal(36.0, 2.0), scenario_id=1)
    n, batches = 2_000, 200
    exact = stats.norm.sf(3.0)
    est, ses, cover = [], [], 0
    for b in range(batches):
        cols, w = oracle_mod.sample_is(ai.paper_model(), p, q, b * n, n)
        e, se, (lo, hi) = oracle_mod.is_estimate(w, cols["v0"] > 36.0)
        y = np.where(cols["v0"] > 36.0, w, 0.0)
        assert abs(se - math.sqrt(np.var(y, ddof=1) / n)) <= 1e-12 * se
        est.append(e)
        ses.append(se)
        cover += lo <= exact <= hi
    spread = np.std(est, ddof=1)
    assert abs(spread / np.mean(ses) - 1.0) < 0.2, (spread, np.mean(ses))
    assert 0.88 * batches <= cover <= 0.995 * batches, cover
