"""GPU parity: the CUDA path through the C ABI against the oracle on the same
seeded inputs.

  * AEB_FP64_PLAIN must equal the oracle in every bit of every output
    (Sec. V-D / VI-A: maximum deviation 0.000000 m between CPU and GPU).
  * AEB_FP32_COMP must stay within the stated tolerances, for every output:
      - stopped in both: |x_ref - x_ref64| <= 1e-5 x_ref64 (relative);
      - stop/contact flag may differ only where the path that stopped has
        |final gap| < 1e-3 m; such samples are counted;
      - stopped: t_end within 1e-6 s + 1e-6 relative;
      - contact: the contact instant and speed are as well conditioned as the
        position allows, so the bound is the position bound carried through
        the kinematics: |dt_end| v_imp <= 1e-5 d0 and
        |dv_imp| v_imp <= r_max 1e-5 d0 (r_max = 10 m/s^2 bounds |dv/dt|);
      - horizon: t_end identical;
      - n_steps equal, or one apart where the end falls on a step boundary
        (stop: t_end within the stop bound of the boundary; contact: within
        the contact bound); x_raw (the paper's D_stop = x(t_stop), Eq. 3)
        within 1e-5 relative, plus where n_steps is one apart the travel of
        that step (stop: <= r_max dt^2, the speed there is below r_max dt;
        contact: <= dt (v_imp + v_lead + r_max dt));
      - brake onset identical in immediate mode (an integer computed in
        binary64 from the same rule).  Under the TTC trigger the onset may
        differ only where the trigger decision is a rounding tie, proven per
        sample: at the step where the binary32 kernel fired and the oracle did
        not, the oracle's binary64 margin (gap + noise) - thr closing speed is
        <= eps; at every step where the oracle fired and the kernel did not,
        the margin is >= -eps (a reading's dropout decision is the oracle's
        exactly: an integer comparison of its word with ceil(perc_drop 2^32)).
        eps = 2^-21 (|gap + noise| + thr |closing| + x_n + d0 + x_L + thr v_L)
        + 18 2^-24 perc_sigma: eight binary32 ulps of every quantity the kernel
        rounds on the way to the margin (the compensated state carries <= ~6
        ulps of position through the approach, each operand of the margin one
        rounding, the lead's closed form in binary32 about three), and for the
        reading's noise 6 2^-24 sigma from the 24-bit uniforms (the oracle's
        have 32 bits), 6 from the two roundings of their sum, 6 from the two
        products that scale it.  Such a sample is then compared, with every
        bound above, against the oracle run with its trigger forced to the
        kernel's step: no sample escapes the bounds.
  * aeb_reduce: integer counts and histograms exact, extremes exact, sums
    within n * 2^-52 * sum|x| of the exactly rounded sum.
"""
import math

import numpy as np
import pytest

import aeb_inputs as ai
from fp32_bounds import fp32_report, resolve_onset_ties, with_gap

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def aeb():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2604_27193_gb300 as aeb
    aeb.build()
    aeb.lib()
    return aeb


def gpu_rollout(aeb, m, params, precision):
    n = len(params["v0"])
    P = {f: torch.from_numpy(np.ascontiguousarray(params[f])).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(max(n, 1))
    aeb.aeb_rollout(m, P, n, precision, O)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy()[:n] for k, v in O.items()}


def bits_equal(a, b):
    a, b = np.asarray(a), np.asarray(b)
    if a.dtype == np.float64:
        return np.array_equal(a.view(np.uint64), b.view(np.uint64))
    return np.array_equal(a, b)


def assert_bit_exact(got, exp):
    for k in ("status", "x_raw", "x_ref", "v_imp", "t_end", "n_steps", "n_onset"):
        if not bits_equal(got[k], exp[k]):
            bad = np.nonzero(got[k].view(np.uint64) != exp[k].view(np.uint64)
                             if got[k].dtype == np.float64 else got[k] != exp[k])[0]
            i = bad[0]
            raise AssertionError(f"{k}: {len(bad)} mismatches, first at {i}: "
                                 f"gpu {got[k][i]!r} oracle {exp[k][i]!r}")


FP64_CASES = {
    "single_scenario": (ai.single_model(), ai.single_scenario(seed=0), 10_000),
    "paper_preset": (ai.paper_model(), ai.paper_scenario(seed=1), 4_000),
    "ttc_1s": (ai.ttc_model(thr=1.0), ai.single_scenario(seed=2), 3_000),
    "ttc_2.5s": (ai.ttc_model(thr=2.5), ai.single_scenario(seed=3), 3_000),
    "lumped_lead": (ai.replace(ai.single_model(), cap_mode=ai.CAP_LUMPED),
                    ai.single_scenario(seed=4), 3_000),
    "per_axle_no_lead": (ai.replace(ai.single_model(), lead=0), ai.single_scenario(seed=5), 3_000),
    "coarse_dt_20ms": (ai.single_model(dt=0.02), ai.single_scenario(seed=6), 3_000),
    "fine_dt_0.1ms": (ai.single_model(dt=1e-4), ai.single_scenario(seed=7), 300),
    "short_horizon": (ai.replace(ai.single_model(), t_max=1.5), ai.single_scenario(seed=8), 2_000),
    "moving_lead_braking": (ai.lead_braking_model(), ai.lead_braking_scenario(seed=9), 5_000),
    "moving_lead_constant": (ai.lead_braking_model(lead_v0=10.0, lead_decel=0.0),
                             ai.lead_braking_scenario(seed=15), 3_000),
    "moving_lead_ttc": (ai.replace(ai.lead_braking_model(lead_decel=4.0), trigger=ai.TRIGGER_TTC,
                                   ttc_thr=3.0), ai.lead_braking_scenario(seed=16), 3_000),
    "moving_lead_lumped_20ms": (ai.replace(ai.lead_braking_model(dt=0.02), cap_mode=ai.CAP_LUMPED),
                                ai.lead_braking_scenario(seed=17), 3_000),
    "ttc_perception": (ai.replace(ai.ttc_model(thr=2.0), perc_sigma=0.8, perc_drop=0.2,
                                  perc_latency=0.05, perc_seed=11), ai.single_scenario(seed=21), 3_000),
    "moving_lead_ttc_perception": (ai.replace(ai.lead_braking_model(lead_decel=4.0),
                                              trigger=ai.TRIGGER_TTC, ttc_thr=3.0, perc_sigma=1.5,
                                              perc_drop=0.4, perc_latency=0.0123, perc_seed=12),
                                   ai.lead_braking_scenario(seed=22), 3_000),
    # feature combinations at coarse steps
    "ttc_perception_10ms": (ai.replace(ai.ttc_model(thr=2.0, dt=0.01), perc_sigma=0.8,
                                       perc_drop=0.2, perc_latency=0.05, perc_seed=31),
                            ai.single_scenario(seed=33), 3_000),
    "moving_lead_ttc_5ms": (ai.replace(ai.lead_braking_model(dt=5e-3, lead_decel=4.0),
                                       trigger=ai.TRIGGER_TTC, ttc_thr=3.0),
                            ai.lead_braking_scenario(seed=34), 3_000),
    # a wide noise band (many lanes in it at once) at an odd latency; every
    # reading missing (the trigger never fires)
    "ttc_perception_wide": (ai.replace(ai.ttc_model(thr=2.0), perc_sigma=4.0, perc_drop=0.5,
                                       perc_latency=0.021, perc_seed=41),
                            ai.single_scenario(seed=41), 3_000),
    "ttc_perception_all_missing": (ai.replace(ai.ttc_model(thr=2.0), perc_sigma=1.0, perc_drop=1.0,
                                              perc_seed=42), ai.single_scenario(seed=42), 2_000),
    # the serving stream's icy road class (the friction cap binds from onset),
    # the TTC trigger at a fine step, and the TTC trigger with Eq. 5's cap
    "icy_road": (ai.single_model(), ai.replace(ai.single_scenario(seed=45),
                                               mu=ai.uniform(*ai.ROAD_CLASSES["icy"])), 3_000),
    "ttc_fine_dt_0.1ms": (ai.ttc_model(thr=2.0, dt=1e-4), ai.single_scenario(seed=46), 300),
    "ttc_lumped": (ai.replace(ai.ttc_model(thr=1.5), cap_mode=ai.CAP_LUMPED),
                   ai.single_scenario(seed=47), 3_000),
}


@pytest.mark.parametrize("name", list(FP64_CASES))
def test_fp64_bit_exact(aeb, oracle_mod, name):
    m, sc, n = FP64_CASES[name]
    p = ai.draw_params(m, sc, n)
    exp = oracle_mod.rollout(m, p, threads=8)
    got = gpu_rollout(aeb, m, p, aeb.FP64_PLAIN)
    assert_bit_exact(got, exp)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 255, 257, 1031, 4099])
def test_fp64_ragged_sizes(aeb, oracle_mod, n):
    m = ai.single_model()
    p = ai.draw_params(m, ai.single_scenario(seed=n), n)
    assert_bit_exact(gpu_rollout(aeb, m, p, aeb.FP64_PLAIN), oracle_mod.rollout(m, p))


@pytest.mark.parametrize("lead,trigger", [(1, 0), (0, 0), (1, 1)])
def test_edge_cases_both_precisions(aeb, oracle_mod, lead, trigger):
    m = ai.replace(ai.single_model(), lead=lead, trigger=trigger, ttc_thr=2.0)
    p = ai.edge_params(m)
    exp = oracle_mod.rollout(m, p)
    assert_bit_exact(gpu_rollout(aeb, m, p, aeb.FP64_PLAIN), exp)
    got = gpu_rollout(aeb, m, p, aeb.FP32_COMP)
    assert np.array_equal(got["status"], exp["status"])
    inv = exp["status"] == 255
    assert np.all(np.isnan(got["x_ref"][inv])) and np.all(got["n_steps"][inv] == 0)
    ok = ~inv
    assert np.allclose(got["x_ref"][ok], exp["x_ref"][ok], rtol=1e-5, atol=1e-7)


def test_zero_samples_and_tiny_horizon(aeb, oracle_mod):
    m = ai.replace(ai.single_model(), t_max=0.0)
    p = ai.draw_params(m, ai.single_scenario(), 50)
    exp = oracle_mod.rollout(m, p)
    assert np.all(exp["status"] == 2)
    assert_bit_exact(gpu_rollout(aeb, m, p, aeb.FP64_PLAIN), exp)
    P = {f: torch.zeros(1, dtype=torch.float64, device="cuda") for f in ai.FIELDS}
    aeb.aeb_rollout(ai.single_model(), P, 0, aeb.FP64_PLAIN, aeb.alloc_outputs(1))


FP32_CASES = {
    "single_scenario": (ai.single_model(), ai.single_scenario(seed=10), 20_000),
    "paper_preset": (ai.paper_model(), ai.paper_scenario(seed=11), 10_000),
    "single_scenario_dt_0.1ms": (ai.single_model(dt=1e-4), ai.single_scenario(seed=12), 400),
    "ttc_2s": (ai.ttc_model(thr=2.0), ai.single_scenario(seed=13), 10_000),
    "grid_scenario": (ai.single_model(), ai.grid_scenarios()[1234][0], 5_000),
    "moving_lead_braking": (ai.lead_braking_model(), ai.lead_braking_scenario(seed=18), 20_000),
    "moving_lead_constant": (ai.lead_braking_model(lead_v0=10.0, lead_decel=0.0),
                             ai.lead_braking_scenario(seed=19), 10_000),
    "moving_lead_ttc": (ai.replace(ai.lead_braking_model(lead_decel=4.0), trigger=ai.TRIGGER_TTC,
                                   ttc_thr=3.0), ai.lead_braking_scenario(seed=20), 10_000),
    "ttc_perception": (ai.replace(ai.ttc_model(thr=2.0), perc_sigma=0.8, perc_drop=0.2,
                                  perc_latency=0.05, perc_seed=13), ai.single_scenario(seed=23), 10_000),
    # long approaches to the breakpoints of r(D): windows cut to the exact safe length
    "per_axle_no_lead_slow_actuator": (ai.replace(ai.single_model(), lead=0),
                                       ai.replace(ai.single_scenario(seed=24),
                                                  tau=ai.uniform(0.3, 0.8)), 10_000),
    "lumped_lead": (ai.replace(ai.single_model(), cap_mode=ai.CAP_LUMPED),
                    ai.single_scenario(seed=25), 10_000),
    # per-step actuator decay dt/tau up to 0.2
    "coarse_dt_20ms": (ai.single_model(dt=0.02), ai.single_scenario(seed=26), 10_000),
    # feature combinations at coarse steps
    "ttc_perception_10ms": (ai.replace(ai.ttc_model(thr=2.0, dt=0.01), perc_sigma=0.8,
                                       perc_drop=0.2, perc_latency=0.05, perc_seed=32),
                            ai.single_scenario(seed=35), 10_000),
    "moving_lead_ttc_5ms": (ai.replace(ai.lead_braking_model(dt=5e-3, lead_decel=4.0),
                                       trigger=ai.TRIGGER_TTC, ttc_thr=3.0),
                            ai.lead_braking_scenario(seed=36), 10_000),
    # per-step perception: the band windows' trigger tests with a moving lead's
    # terms (odd latency: 31-step band windows from odd reading indices), a
    # wide band (more band lanes than slots: waits, shared reading batches),
    # every reading missing
    "moving_lead_ttc_perception": (ai.replace(ai.lead_braking_model(lead_decel=4.0),
                                              trigger=ai.TRIGGER_TTC, ttc_thr=3.0, perc_sigma=1.5,
                                              perc_drop=0.4, perc_latency=0.0123, perc_seed=14),
                                   ai.lead_braking_scenario(seed=37), 10_000),
    "ttc_perception_wide": (ai.replace(ai.ttc_model(thr=2.0), perc_sigma=4.0, perc_drop=0.5,
                                       perc_latency=0.021, perc_seed=43),
                            ai.single_scenario(seed=43), 10_000),
    "ttc_perception_all_missing": (ai.replace(ai.ttc_model(thr=2.0), perc_sigma=1.0, perc_drop=1.0,
                                              perc_seed=44), ai.single_scenario(seed=44), 5_000),
    # the serving stream's icy road class (the friction cap binds from onset,
    # long stops and many contacts), the TTC trigger at a fine step (trigger
    # tests bounded over many short steps), the TTC trigger with Eq. 5's cap
    "icy_road": (ai.single_model(), ai.replace(ai.single_scenario(seed=48),
                                               mu=ai.uniform(*ai.ROAD_CLASSES["icy"])), 10_000),
    "ttc_fine_dt_0.1ms": (ai.ttc_model(thr=2.0, dt=1e-4), ai.single_scenario(seed=49), 400),
    "ttc_lumped": (ai.replace(ai.ttc_model(thr=1.5), cap_mode=ai.CAP_LUMPED),
                   ai.single_scenario(seed=50), 10_000),
}


@pytest.mark.parametrize("name", list(FP32_CASES))
def test_fp32_comp_within_tolerance(aeb, oracle_mod, name):
    m, sc, n = FP32_CASES[name]
    p = ai.draw_params(m, sc, n)
    exp = oracle_mod.rollout(m, p, threads=8)
    got = gpu_rollout(aeb, m, p, aeb.FP32_COMP)
    exp, ties = resolve_onset_ties(oracle_mod, m, p, np.arange(n), got, exp)
    rep = fp32_report(m, with_gap(got, p, m), with_gap(exp, p, m), ties)
    print(name, rep)
    # every tie is proven above; many of them would point at a drift of the
    # kernel's margin, not at rounding
    assert rep["onset_ties"] <= max(3, 1e-3 * n), rep


@pytest.mark.parametrize("n", [1, 2, 31, 33, 257, 1031, 4099])
def test_fp32_ragged_sizes(aeb, oracle_mod, n):
    """Sizes that leave the last warp tile partial, with the edge samples
    (invalid, already stopped or in contact, no drag, tau = 0) placed at the
    end, so that samples that end at once sit inside partial tiles; the TTC
    trigger variant too."""
    for m in (ai.single_model(), ai.ttc_model(thr=2.0)):
        p = ai.concat_params([ai.draw_params(m, ai.single_scenario(seed=30 + n), n),
                              ai.edge_params(m)])
        k = len(p["v0"])
        exp = oracle_mod.rollout(m, p, threads=8)
        got = gpu_rollout(aeb, m, p, aeb.FP32_COMP)
        exp, ties = resolve_onset_ties(oracle_mod, m, p, np.arange(k), got, exp)
        inv = exp["status"] == 255
        assert np.array_equal(got["status"][inv], exp["status"][inv])
        assert np.all(np.isnan(got["x_ref"][inv])) and np.all(got["n_steps"][inv] == 0)
        ok = ~inv
        g, e = with_gap(got, p, m), with_gap(exp, p, m)
        fp32_report(m, {c: v[ok] for c, v in g.items()}, {c: v[ok] for c, v in e.items()}, ties)


def test_fp32_every_tile_size_same_results(aeb):
    """Per-sample results do not depend on the tile a warp prepares (32 ... 256
    samples, the largest allowed) nor on the resident blocks per SM: a lane's
    windows depend on its own state only."""
    m = ai.single_model()
    p = ai.concat_params([ai.draw_params(m, ai.single_scenario(seed=31), 70_001),
                          ai.edge_params(m)])
    old = aeb.aeb_get_launch_config(aeb.FP32_COMP)
    try:
        aeb.aeb_set_launch_config(aeb.FP32_COMP, 32, 6)
        ref = gpu_rollout(aeb, m, p, aeb.FP32_COMP)
        for tile, bps in ((64, 6), (128, 4), (256, 2), (32, 3)):
            aeb.aeb_set_launch_config(aeb.FP32_COMP, tile, bps)
            got = gpu_rollout(aeb, m, p, aeb.FP32_COMP)
            for k in ref:
                assert bits_equal(got[k], ref[k]), (tile, bps, k)
    finally:
        aeb.aeb_set_launch_config(aeb.FP32_COMP, old.tile, old.blocks_per_sm)


def test_reduce_against_oracle(aeb, oracle_mod):
    m = ai.single_model()
    p = ai.concat_params([ai.draw_params(m, ai.single_scenario(seed=20), 12_345),
                          ai.edge_params(m)])
    n = len(p["v0"])
    exp_out = oracle_mod.rollout(m, p, threads=8)
    P = {f: torch.from_numpy(p[f]).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(n)
    aeb.aeb_rollout(m, P, n, aeb.FP64_PLAIN, O)
    for spec in ((0.0, 0.125, 0.0, 1 / 64), (20.0, 0.0625, -1.0, 0.25)):
        S = aeb.alloc_stats()
        aeb.aeb_reduce(O, n, aeb.hist_spec(*spec), S)
        st = aeb.stats_from_buffer(S)
        ex = oracle_mod.reduce(exp_out, spec[0], spec[1], spec[2], spec[3], 4096)
        for k in ("n", "n_stop", "n_contact", "n_horizon", "n_invalid", "steps",
                  "min_d", "max_d", "min_v", "max_v"):
            assert getattr(st, k) == getattr(ex, k), k
        assert np.array_equal(np.frombuffer(bytes(st.hist_d), np.uint64), ex.hist_d)
        assert np.array_equal(np.frombuffer(bytes(st.hist_v), np.uint64), ex.hist_v)
        d = exp_out["x_ref"][exp_out["status"] == 0]
        v = exp_out["v_imp"][exp_out["status"] == 1]
        for got, vals in ((st.sum_d, d), (st.sumsq_d, d * d), (st.sum_v, v), (st.sumsq_v, v * v)):
            assert abs(got - math.fsum(vals)) <= len(vals) * 2.3e-16 * math.fsum(np.abs(vals))


def test_reduce_empty(aeb):
    O = aeb.alloc_outputs(1)
    S = aeb.alloc_stats()
    aeb.aeb_reduce(O, 0, aeb.hist_spec(), S)
    st = aeb.stats_from_buffer(S)
    assert st.n == 0 and st.n_stop == 0 and st.min_d == math.inf and st.max_d == -math.inf
    assert sum(st.hist_d) == 0


def test_deterministic_repeats(aeb):
    m = ai.single_model()
    n = 50_000
    p = ai.draw_params(m, ai.single_scenario(seed=30), n)
    P = {f: torch.from_numpy(p[f]).cuda() for f in ai.FIELDS}
    res = []
    for _ in range(2):
        O = aeb.alloc_outputs(n)
        aeb.aeb_rollout(m, P, n, aeb.FP32_COMP, O)
        S = aeb.alloc_stats()
        aeb.aeb_reduce(O, n, aeb.hist_spec(), S)
        res.append((O, bytes(S.cpu().numpy())))
    for k in res[0][0]:
        assert torch.equal(res[0][0][k], res[1][0][k]), k
    assert res[0][1] == res[1][1]


def test_evaluate_host_path(aeb, oracle_mod):
    """aeb_evaluate (host buffers in, host stats out) equals the device calls."""
    m = ai.single_model()
    n = 7_777
    p = aeb.aeb_sample_params(m, ai.single_scenario(seed=40), 0, n)
    host_out = {k: np.empty(n, dtype=aeb.OUT_DTYPES[k]) for k in aeb.OUTPUTS}
    st = aeb.aeb_evaluate(m, p, n, aeb.FP64_PLAIN, aeb.hist_spec(), host_out=host_out)
    exp = oracle_mod.rollout(m, p, threads=8)
    assert_bit_exact(host_out, exp)
    ex = oracle_mod.reduce(exp)
    assert (st.n_stop, st.n_contact, st.n_horizon) == (ex.n_stop, ex.n_contact, ex.n_horizon)
    assert np.array_equal(np.frombuffer(bytes(st.hist_d), np.uint64), ex.hist_d)
    st2 = aeb.aeb_evaluate(m, p, n, aeb.FP64_PLAIN, aeb.hist_spec())
    assert bytes(st2) == bytes(st)


@pytest.mark.parametrize("n", [2_500_003, 10_000_000])
def test_evaluate_chunked_upload(aeb, n):
    """aeb_evaluate above 2^19 samples uploads and rolls out in chunks of
    growing length on internal streams (2.5e6: four chunks, the last shorter
    than the one before; 1e7: the benchmark's end-to-end call); its outputs and
    statistics are byte-identical to one device-resident rollout and reduction
    of the same parameters."""
    m = ai.single_model()
    p = aeb.aeb_sample_params(m, ai.single_scenario(seed=41), 0, n)
    which = ("status", "x_ref", "v_imp", "n_steps", "n_onset")
    host_out = {k: np.empty(n, dtype=aeb.OUT_DTYPES[k]) for k in which}
    st = aeb.aeb_evaluate(m, p, n, aeb.FP32_COMP, aeb.hist_spec(), host_out=host_out)
    P = {f: torch.from_numpy(p[f]).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(n, which=which)
    aeb.aeb_rollout(m, P, n, aeb.FP32_COMP, O)
    S = aeb.alloc_stats()
    aeb.aeb_reduce(O, n, aeb.hist_spec(), S)
    for k in which:
        assert np.array_equal(host_out[k].view(np.uint8), O[k].cpu().numpy().view(np.uint8)), k
    assert bytes(st) == bytes(S.cpu().numpy())


def test_evaluate_adaptive_chunks_same_bits(aeb):
    """From its second call on a stream, aeb_evaluate grows its chunks by a
    factor measured in the call before (upload against rollout time), so
    successive calls cut the same samples differently; a new stream starts
    over with doubling.  Every call's statistics and outputs are byte-identical
    to the first call's."""
    m = ai.single_model()
    n = 3_000_001
    p = aeb.aeb_sample_params(m, ai.single_scenario(seed=44), 0, n)
    which = ("status", "x_ref", "n_steps")
    ref_out = {k: np.empty(n, dtype=aeb.OUT_DTYPES[k]) for k in which}
    s1 = torch.cuda.Stream()
    ref = bytes(aeb.aeb_evaluate(m, p, n, aeb.FP32_COMP, aeb.hist_spec(), host_out=ref_out,
                                 stream=s1))
    for stream in (s1, s1, s1, torch.cuda.Stream()):
        out = {k: np.empty(n, dtype=aeb.OUT_DTYPES[k]) for k in which}
        st = aeb.aeb_evaluate(m, p, n, aeb.FP32_COMP, aeb.hist_spec(), host_out=out,
                              stream=stream)
        assert bytes(st) == ref
        for k in which:
            assert np.array_equal(out[k].view(np.uint8), ref_out[k].view(np.uint8)), k


@pytest.mark.parametrize("precision", [0, 1])
def test_evaluate_chunked_perception_keys(aeb, precision):
    """Per-step perception readings are keyed by the sample's row in the
    whole call: through aeb_evaluate's chunks (here two, the second starting at
    row 262,144) every output equals one flat aeb_rollout of the same rows."""
    m = ai.replace(ai.ttc_model(thr=2.0), perc_sigma=0.8, perc_drop=0.2, perc_latency=0.05,
                   perc_seed=13)
    n = 600_001
    p = aeb.aeb_sample_params(m, ai.single_scenario(seed=43), 0, n)
    which = ("status", "x_ref", "v_imp", "t_end", "n_steps", "n_onset")
    host_out = {k: np.empty(n, dtype=aeb.OUT_DTYPES[k]) for k in which}
    st = aeb.aeb_evaluate(m, p, n, precision, aeb.hist_spec(), host_out=host_out)
    P = {f: torch.from_numpy(p[f]).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(n, which=which)
    aeb.aeb_rollout(m, P, n, precision, O)
    S = aeb.alloc_stats()
    aeb.aeb_reduce(O, n, aeb.hist_spec(), S)
    for k in which:
        assert np.array_equal(host_out[k].view(np.uint8), O[k].cpu().numpy().view(np.uint8)), k
    assert bytes(st) == bytes(S.cpu().numpy())


def test_full_size_sampled(aeb, oracle_mod):
    """The single-scenario workload at N = 1e7 in the benchmark's launch
    configuration: sampled outputs against the oracle, and invariants over
    every sample."""
    m = ai.single_model()
    n = 10_000_000
    p = aeb.aeb_sample_params(m, ai.single_scenario(seed=0), 0, n)
    P = {f: torch.from_numpy(p[f]).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(n)
    aeb.aeb_rollout(m, P, n, aeb.FP32_COMP, O)
    S = aeb.alloc_stats()
    aeb.aeb_reduce(O, n, aeb.hist_spec(), S)
    st = aeb.stats_from_buffer(S)
    got = {k: v.cpu().numpy() for k, v in O.items()}
    assert st.n == n and st.n_stop + st.n_contact + st.n_horizon + st.n_invalid == n
    assert st.steps == int(got["n_steps"].astype(np.int64).sum())
    assert np.all(got["n_steps"] >= 1)
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([rng.integers(0, n, 3000), [0, 1, n - 2, n - 1]]))
    sub = {f: p[f][idx] for f in ai.FIELDS}
    exp = with_gap(oracle_mod.rollout(m, sub, threads=8), sub, m)
    g = with_gap({k: v[idx] for k, v in got.items()}, sub, m)
    fp32_report(m, g, exp)


def test_full_size_fp64_sampled(aeb, oracle_mod):
    """The binary64 kernel on the full N = 1e7 single-scenario launch (the
    bench's comparison arm): every output of 2,000 sampled samples, and the
    first and last ones, bit-identical to the oracle."""
    m = ai.single_model()
    n = 10_000_000
    p = aeb.aeb_sample_params(m, ai.single_scenario(seed=0), 0, n)
    P = {f: torch.from_numpy(p[f]).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(n)
    aeb.aeb_rollout(m, P, n, aeb.FP64_PLAIN, O)
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([rng.integers(0, n, 2000), [0, 1, n - 2, n - 1]]))
    got = {k: v.cpu().numpy()[idx] for k, v in O.items()}
    exp = oracle_mod.rollout(m, {f: p[f][idx] for f in ai.FIELDS}, threads=8)
    assert_bit_exact(got, exp)


def test_full_size_fine_step_sampled(aeb, oracle_mod):
    """The FP32-compensated kernel on N = 1e7 at dt = 0.1 ms (the largest cell of
    the N x dt sweep, ~3.2e11 RK4 steps): 1,000 sampled samples against the
    oracle within the FP32 bounds."""
    m = ai.single_model(dt=1e-4)
    n = 10_000_000
    p = aeb.aeb_sample_params(m, ai.single_scenario(seed=0), 0, n)
    P = {f: torch.from_numpy(p[f]).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(n)
    aeb.aeb_rollout(m, P, n, aeb.FP32_COMP, O)
    rng = np.random.default_rng(2)
    idx = np.unique(np.concatenate([rng.integers(0, n, 1000), [0, n - 1]]))
    sub = {f: p[f][idx] for f in ai.FIELDS}
    exp = with_gap(oracle_mod.rollout(m, sub, threads=8), sub, m)
    g = with_gap({k: v.cpu().numpy()[idx] for k, v in O.items()}, sub, m)
    print("fine step", fp32_report(m, g, exp))
