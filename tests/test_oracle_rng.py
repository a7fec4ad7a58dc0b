"""Pins of the oracle's sampler (Sec. IV-A, IV-C): the Philox-4x64-10 block
function against numpy's independent implementation, the counter layout, and
the distribution transforms against scipy's distributions."""
import numpy as np
import pytest
from scipy import stats

import aeb_inputs as ai

M64 = (1 << 64) - 1


def numpy_philox_block(ctr, key):
    """numpy's Philox advances its 256-bit counter before producing a block, so
    the block for counter c is the first output of a generator started at c-1."""
    c = [int(x) for x in ctr]
    # 256-bit decrement with borrow
    for j in range(4):
        if c[j] > 0:
            c[j] -= 1
            break
        c[j] = M64
    bg = np.random.Philox(counter=np.array(c, dtype=np.uint64),
                          key=np.array([int(k) for k in key], dtype=np.uint64))
    return bg.random_raw(4).astype(np.uint64)


def test_philox_matches_numpy(oracle_mod):
    rng = np.random.default_rng(123)
    cases = [([0, 0, 0, 0], [0, 0]), ([M64] * 4, [M64, M64]), ([5, 0, 0, 0], [0, 0])]
    for _ in range(200):
        cases.append((rng.integers(0, 2**63, 4, dtype=np.uint64).tolist(),
                      rng.integers(0, 2**63, 2, dtype=np.uint64).tolist()))
    for ctr, key in cases:
        got = oracle_mod.philox4x64_10(ctr, key)
        exp = numpy_philox_block(ctr, key)
        assert np.array_equal(got, exp), (ctr, key)


def test_uniform_extraction_and_counter_layout(oracle_mod):
    """A U[0,1) quantity takes word 0 (even quantity) or word 2 (odd quantity)
    of block (i, q // 2, 0, 0) under key (seed, scenario_id); checked against
    numpy's generator."""
    m = ai.single_model()
    sc = ai.Scenario(v0=ai.uniform(0.0, 1.0), d0=ai.uniform(0.0, 1.0), seed=77, scenario_id=5)
    p = oracle_mod.sample(m, sc, 1000, 16)
    for j in range(16):
        i = 1000 + j
        w = numpy_philox_block([i, 0, 0, 0], [77, 5])
        assert p["v0"][j] == float(int(w[0]) >> 11) * 2.0**-53
        assert p["d0"][j] == float(int(w[2]) >> 11) * 2.0**-53


def test_sample_offsets_are_consistent(oracle_mod):
    m = ai.single_model()
    sc = ai.single_scenario(seed=9)
    a = oracle_mod.sample(m, sc, 0, 500)
    b = oracle_mod.sample(m, sc, 123, 200)
    for f in ai.FIELDS:
        assert np.array_equal(a[f][123:323], b[f]), f


def test_quantities_are_independent_streams(oracle_mod):
    m = ai.single_model()
    sc1 = ai.single_scenario(seed=1)
    sc2 = ai.replace(sc1, v0=ai.normal(20.0, 3.0), tau=ai.const(0.2))
    a = oracle_mod.sample(m, sc1, 0, 300)
    b = oracle_mod.sample(m, sc2, 0, 300)
    for f in ("d0", "mu", "gs", "gc", "mass", "cd", "t_delay", "noise"):
        assert np.array_equal(a[f], b[f]), f
    assert not np.array_equal(a["v0"], b["v0"])
    assert np.all(b["tau"] == 0.2)
    c = oracle_mod.sample(m, ai.replace(sc1, scenario_id=1), 0, 300)
    assert not np.array_equal(a["v0"], c["v0"])


@pytest.mark.parametrize("lo,hi", [(15.0, 35.0), (0.4, 0.9), (-2.0, 7.5)])
def test_uniform_distribution(oracle_mod, lo, hi):
    m = ai.single_model()
    sc = ai.Scenario(v0=ai.uniform(lo, hi), seed=3)
    x = oracle_mod.sample(m, sc, 0, 20000)["v0"]
    assert x.min() >= lo and x.max() < hi
    assert stats.kstest(x, stats.uniform(loc=lo, scale=hi - lo).cdf).pvalue > 1e-3


@pytest.mark.parametrize("mean,sd", [(30.0, 2.0), (0.0, 0.05), (1500.0, 100.0)])
def test_normal_distribution(oracle_mod, mean, sd):
    m = ai.single_model()
    sc = ai.Scenario(mass=ai.normal(mean, sd), seed=4)
    x = oracle_mod.sample(m, sc, 0, 20000)["mass"]
    assert stats.kstest(x, stats.norm(loc=mean, scale=sd).cdf).pvalue > 1e-3
    assert abs(x.mean() - mean) < 5 * sd / np.sqrt(len(x))


def test_clamped_normal(oracle_mod):
    m = ai.single_model()
    sc = ai.Scenario(d0=ai.normal(60.0, 5.0, 55.0, 62.0), seed=5)
    x = oracle_mod.sample(m, sc, 0, 40000)["d0"]
    assert x.min() == 55.0 and x.max() == 62.0
    n = len(x)
    p_lo, p_hi = stats.norm.cdf(-1.0), stats.norm.sf(0.4)
    assert abs(np.mean(x == 55.0) - p_lo) < 5 * np.sqrt(p_lo * (1 - p_lo) / n)
    assert abs(np.mean(x == 62.0) - p_hi) < 5 * np.sqrt(p_hi * (1 - p_hi) / n)


def test_grade_columns(oracle_mod):
    m = ai.single_model()
    sc = ai.Scenario(grade=ai.normal(0.0, 0.05), seed=6)
    p = oracle_mod.sample(m, sc, 0, 20000)
    assert np.allclose(p["gs"] ** 2 + p["gc"] ** 2, m.g ** 2, rtol=1e-14, atol=0)
    theta = np.arctan2(p["gs"], p["gc"])
    assert stats.kstest(theta, stats.norm(scale=0.05).cdf).pvalue > 1e-3
    assert np.all(p["gc"] > 0)


def test_const_distribution(oracle_mod):
    p = oracle_mod.sample(ai.paper_model(), ai.paper_scenario(), 0, 100)
    assert np.all(p["tau"] == 0.15) and np.all(p["t_delay"] == 0.0) and np.all(p["noise"] == 0.0)
