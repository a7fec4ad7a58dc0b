"""aeb_evaluate_scenario: the whole path from the seed, host sampling of each
chunk of 2^20 samples overlapped with the upload and rollout of the one before.

  * small FP64 case against the oracle drawing, rolling out and reducing the
    same samples (Sec. IV-C sampling, Sec. IV-D rollouts, Sec. VI-B/C
    statistics): counts and histograms exact;
  * several chunks (a ragged last one), both precisions, a non-zero first
    sample, per-step perception (readings keyed by the sample's index in the
    call): byte-identical statistics to aeb_sample_params + aeb_evaluate;
  * repeated calls (the staging buffers reused) and n = 0;
  * a bad scenario, precision or NULL stats is rejected before any work.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import aeb_inputs as ai

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def aeb():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2604_27193_gb300 as aeb
    aeb.build()
    aeb.lib()
    return aeb


def two_calls(aeb, m, sc, first, n, precision):
    p = aeb.aeb_sample_params(m, sc, first, n)
    return aeb.aeb_evaluate(m, p, n, precision, aeb.hist_spec())


def test_small_fp64_against_oracle(aeb, oracle_mod):
    m, sc = ai.single_model(), ai.single_scenario(seed=60)
    n, first = 5_000, 123
    st = aeb.aeb_evaluate_scenario(m, sc, first, n, aeb.FP64_PLAIN, aeb.hist_spec())
    p = oracle_mod.sample(m, sc, first, n)
    ex = oracle_mod.reduce(oracle_mod.rollout(m, p, threads=8))
    for k in ("n", "n_stop", "n_contact", "n_horizon", "n_invalid", "steps", "min_d", "max_d"):
        assert getattr(st, k) == getattr(ex, k), k
    assert np.array_equal(np.frombuffer(bytes(st.hist_d), np.uint64), ex.hist_d)
    assert np.array_equal(np.frombuffer(bytes(st.hist_v), np.uint64), ex.hist_v)


CASES = {
    "fp32_three_chunks": (ai.single_model(), ai.single_scenario(seed=61), 0, 2_500_003, 1),
    "fp32_first_offset": (ai.single_model(), ai.single_scenario(seed=62), 1_000_001, 1_048_577, 1),
    "fp64_two_chunks": (ai.single_model(), ai.single_scenario(seed=63), 5, 1_100_000, 0),
    "fp32_perception": (ai.replace(ai.ttc_model(thr=2.0), perc_sigma=1.0, perc_drop=0.2,
                                   perc_latency=0.05, perc_seed=9),
                        ai.single_scenario(seed=64), 17, 2_200_000, 1),
}


@pytest.mark.parametrize("name", list(CASES))
def test_same_bits_as_sampling_then_evaluate(aeb, name):
    m, sc, first, n, prec = CASES[name]
    if prec == 0 and n > 200_000:
        # the binary64 kernel at 1e6 samples takes ~0.5 s per call; keep it
        m = ai.replace(m, t_max=2.0)
    precision = aeb.FP32_COMP if prec else aeb.FP64_PLAIN
    st = aeb.aeb_evaluate_scenario(m, sc, first, n, precision, aeb.hist_spec())
    ref = two_calls(aeb, m, sc, first, n, precision)
    assert bytes(st) == bytes(ref)
    assert st.n == n


def test_repeated_calls_and_empty(aeb):
    m, sc = ai.single_model(), ai.single_scenario(seed=65)
    a = aeb.aeb_evaluate_scenario(m, sc, 0, 3_300_000, aeb.FP32_COMP, aeb.hist_spec())
    b = aeb.aeb_evaluate_scenario(m, sc, 0, 3_300_000, aeb.FP32_COMP, aeb.hist_spec(), n_threads=3)
    assert bytes(a) == bytes(b)
    z = aeb.aeb_evaluate_scenario(m, sc, 0, 0, aeb.FP32_COMP, aeb.hist_spec())
    assert z.n == 0 and z.n_stop == 0 and z.steps == 0


def test_bad_arguments_rejected(aeb):
    m, sc = ai.single_model(), ai.single_scenario(seed=66)
    bad = ai.replace(sc, mass=ai.Dist(7, 0.0, 0.0))  # unknown distribution kind
    with pytest.raises(aeb.AebError) as e:
        aeb.aeb_evaluate_scenario(m, bad, 0, 1000, aeb.FP32_COMP, aeb.hist_spec())
    assert e.value.code == aeb.EINVAL
    with pytest.raises(aeb.AebError) as e:
        aeb.aeb_evaluate_scenario(m, sc, 0, 1000, 5, aeb.hist_spec())
    assert e.value.code == aeb.EINVAL
