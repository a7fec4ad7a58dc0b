"""TTC-threshold sweep (collision probability against the trigger threshold,
TTC = H0 / v, Sec. VI-C): pooled counts and Wilson intervals from batched
launches over a shared parameter block."""
import numpy as np
import pytest

import aeb_inputs as ai

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def aeb():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2604_27193_gb300 as aeb
    aeb.build()
    aeb.lib()
    return aeb


def test_small_sweep_fp64_against_oracle(aeb, oracle_mod):
    m = ai.ttc_model()
    scen = ai.ttc_scenarios(8, seed=4)
    thr = np.linspace(0.5, 4.0, 16)
    n = 2000
    res, jobs = aeb.aeb_ttc_sweep(m, scen, n, thr, aeb.FP64_PLAIN, per_job=True)
    for t, s in ((0, 0), (5, 3), (15, 7), (9, 1)):
        p = oracle_mod.sample(m, scen[s], 0, n)
        ex = oracle_mod.reduce(oracle_mod.rollout(ai.replace(m, ttc_thr=float(thr[t])), p, threads=8))
        j = jobs[t * len(scen) + s]
        assert (j.n_contact, j.n_stop, j.n_horizon, j.steps) == (ex.n_contact, ex.n_stop, ex.n_horizon, ex.steps)
    for r in res:
        assert r.n == len(scen) * n and r.n_invalid == 0
        assert r.ci_lo <= r.p_contact <= r.ci_hi
        lo, hi = oracle_mod.wilson(r.n_contact, r.n)
        assert abs(lo - r.ci_lo) < 1e-15 and abs(hi - r.ci_hi) < 1e-15
    p = [r.p_contact for r in res]
    assert all(p[i] >= p[i + 1] for i in range(len(p) - 1)), p


def test_full_size_sweep(aeb, oracle_mod):
    """256 thresholds x 64 scenarios x 1e5 samples (FP32-compensated), then the
    same sweep in binary64 on a 1e6-sample subset (the first 61 samples of each
    scenario at every threshold): the subset's binary64 counts equal the CPU
    oracle's, and the FP32 counts on the subset differ from them by at most a
    few tolerated trigger/flag flips per threshold."""
    m = ai.ttc_model()
    scen = ai.ttc_scenarios(64, seed=4)
    thr = ai.ttc_thresholds(256)
    res = aeb.aeb_ttc_sweep(m, scen, 100_000, thr, aeb.FP32_COMP)
    assert len(res) == 256 and all(r.n == 6_400_000 for r in res)
    p = np.array([r.p_contact for r in res])
    assert np.all(np.diff(p) <= 1e-3)  # non-increasing up to sampling-free flips
    assert p[0] > p[-1]
    sub = 61
    r64, j64 = aeb.aeb_ttc_sweep(m, scen, sub, thr, aeb.FP64_PLAIN, per_job=True)
    r32 = aeb.aeb_ttc_sweep(m, scen, sub, thr, aeb.FP32_COMP)
    flips = [abs(a.n_contact - b.n_contact) for a, b in zip(r64, r32)]
    assert max(flips) <= 3, flips
    # binary64 subset against the oracle: 64 scenarios x 61 samples at 16 thresholds
    for t in range(0, 256, 16):
        mt = ai.replace(m, ttc_thr=float(thr[t]))
        for s in range(0, 64, 7):
            pp = oracle_mod.sample(m, scen[s], 0, sub)
            ex = oracle_mod.reduce(oracle_mod.rollout(mt, pp))
            assert j64[t * 64 + s].n_contact == ex.n_contact and j64[t * 64 + s].steps == ex.steps


def test_sweep_with_perception_fp64_against_oracle(aeb, oracle_mod):
    """Per-step perception inside the batched sweep: a job's readings are keyed
    by its parameter rows (scenario s occupies rows s n .. (s+1) n - 1 of the
    shared block), so the binary64 counts equal the oracle's run on the same
    rows."""
    m = ai.replace(ai.ttc_model(), perc_sigma=0.6, perc_drop=0.15, perc_latency=0.02,
                   perc_seed=5)
    scen = ai.ttc_scenarios(4, seed=9)
    thr = np.array([0.8, 1.6, 2.4])
    n = 1500
    res, jobs = aeb.aeb_ttc_sweep(m, scen, n, thr, aeb.FP64_PLAIN, per_job=True)
    for t in range(len(thr)):
        for s in range(len(scen)):
            p = oracle_mod.sample(m, scen[s], 0, n)
            ex = oracle_mod.reduce(oracle_mod.rollout(ai.replace(m, ttc_thr=float(thr[t])), p,
                                                      threads=8, row0=s * n))
            j = jobs[t * len(scen) + s]
            assert (j.n_contact, j.n_stop, j.n_horizon, j.steps) == \
                (ex.n_contact, ex.n_stop, ex.n_horizon, ex.steps), (t, s)
