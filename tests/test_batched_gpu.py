"""Batched launches: many jobs with uneven sample counts in one persistent
launch over a (job, tile) table, per-job fixed-order reductions, a captured
CUDA graph, and the launch-shape autotuner.  Per-sample results must not depend
on what else shares the launch: each job's outputs are identical alone and in
the batch, and binary64 outputs equal the oracle bit for bit."""
import math

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


def grid_jobs(aeb, m, n_jobs=40, seed=7):
    """A subset of the scenario grid with uneven counts (0, 1, ragged, large);
    outputs laid out in reverse job order to decouple the two offsets."""
    sc_all = ai.grid_scenarios(seed=2)
    rng = np.random.default_rng(seed)
    picks = rng.choice(len(sc_all), n_jobs, replace=False)
    sizes = [0, 1, 33, 64, 65, 1000] + [int(sc_all[k][1] // 8) for k in picks[6:]]
    parts, jobs_p = [], []
    off = 0
    for k, nj in zip(picks, sizes):
        parts.append(aeb.aeb_sample_params(m, sc_all[k][0], 0, nj))
        jobs_p.append((off, nj))
        off += nj
    params = {f: np.concatenate([p[f] for p in parts]) for f in ai.FIELDS}
    total = off
    out_off, o = [0] * n_jobs, 0
    for j in reversed(range(n_jobs)):
        out_off[j] = o
        o += sizes[j]
    jobs = [(po, out_off[j], nj, m.ttc_thr) for j, (po, nj) in enumerate(jobs_p)]
    return params, jobs, total


def to_dev(p):
    return {f: torch.from_numpy(np.ascontiguousarray(p[f])).cuda() for f in ai.FIELDS}


def run_batched(aeb, m, jobs, P, total, precision):
    O = aeb.alloc_outputs(max(total, 1))
    S = torch.empty(aeb.JOB_STATS_BYTES * len(jobs), dtype=torch.uint8, device="cuda")
    aeb.aeb_rollout_batched(m, jobs, P, precision, O, S)
    out = {k: v.cpu().numpy() for k, v in O.items()}
    return out, aeb.job_stats_from_buffer(S, len(jobs))


def job_slice(out, job):
    _, oo, n, _ = job
    return {k: v[oo:oo + n] for k, v in out.items()}


def bits(a):
    return a.view(np.uint64) if a.dtype == np.float64 else a


@pytest.mark.parametrize("trigger", [0, 1])
def test_batched_fp64_matches_oracle(aeb, oracle_mod, trigger):
    m = ai.replace(ai.single_model(), trigger=trigger, ttc_thr=2.0)
    params, jobs, total = grid_jobs(aeb, m)
    if trigger:  # per-job thresholds
        jobs = [(po, oo, n, 0.5 + 0.1 * j) for j, (po, oo, n, _) in enumerate(jobs)]
    out, stats = run_batched(aeb, m, jobs, to_dev(params), total, aeb.FP64_PLAIN)
    for j, job in enumerate(jobs):
        po, oo, n, thr = job
        sub = {f: params[f][po:po + n] for f in ai.FIELDS}
        mj = ai.replace(m, ttc_thr=thr)
        exp = oracle_mod.rollout(mj, sub, threads=8)
        got = job_slice(out, job)
        for k in ("status", "x_ref", "v_imp", "t_end", "n_steps", "n_onset", "x_raw"):
            assert np.array_equal(bits(got[k]), bits(exp[k])), (j, k)
        ex = oracle_mod.reduce(exp)
        st = stats[j]
        assert st.n == n
        for k in ("n_stop", "n_contact", "n_horizon", "n_invalid", "steps"):
            assert getattr(st, k) == getattr(ex, k), (j, k)
        if ex.n_stop:
            assert (st.min_d, st.max_d) == (ex.min_d, ex.max_d)
            d = exp["x_ref"][exp["status"] == 0]
            assert abs(st.sum_d - math.fsum(d)) <= len(d) * 2.3e-16 * math.fsum(np.abs(d))
        if ex.n_contact:
            v = exp["v_imp"][exp["status"] == 1]
            assert abs(st.sum_v - math.fsum(v)) <= len(v) * 2.3e-16 * math.fsum(np.abs(v)) + 1e-300
        if n == 0:
            assert st.n_stop == 0 and st.min_d == math.inf


def test_batched_fp32_alone_equals_in_mix(aeb):
    """Each job's FP32 outputs are the same bits whether it runs alone (flat
    launch) or inside the batch."""
    m = ai.single_model()
    params, jobs, total = grid_jobs(aeb, m, seed=9)
    P = to_dev(params)
    out, stats = run_batched(aeb, m, jobs, P, total, aeb.FP32_COMP)
    for j, job in enumerate(jobs[:12]):
        po, oo, n, _ = job
        if n == 0:
            continue
        Pj = {f: P[f][po:po + n].contiguous() for f in ai.FIELDS}
        Oj = aeb.alloc_outputs(n)
        aeb.aeb_rollout(m, Pj, n, aeb.FP32_COMP, Oj)
        alone = {k: v.cpu().numpy() for k, v in Oj.items()}
        mix = job_slice(out, job)
        for k in alone:
            assert np.array_equal(bits(alone[k]), bits(mix[k])), (j, k)
    assert sum(s.n for s in stats) == total


PERC = dict(trigger=ai.TRIGGER_TTC, ttc_thr=2.0, perc_sigma=1.2, perc_drop=0.25,
            perc_latency=0.013, perc_seed=77)


def test_batched_perception_key_offsets(aeb, oracle_mod):
    """Per-step perception in a batch: job j's sample i draws its readings
    from row key_offset_j + i.  Binary64 outputs equal the oracle run with
    that row offset, bit for bit; FP32 outputs of each job are the same bits
    alone (a flat launch keyed from the same row) and in the batch."""
    m = ai.replace(ai.single_model(), **PERC)
    params, jobs, total = grid_jobs(aeb, m, n_jobs=24, seed=13)
    # keys: a row range of its own per job, not the parameter offset
    jobs = [(po, oo, n, thr, 1_000_000 + 10_000 * j) for j, (po, oo, n, thr) in enumerate(jobs)]
    P = to_dev(params)
    out, _ = run_batched(aeb, m, jobs, P, total, aeb.FP64_PLAIN)
    for j, job in enumerate(jobs[:10]):
        po, oo, n, _, ko = job
        sub = {f: params[f][po:po + n] for f in ai.FIELDS}
        exp = oracle_mod.rollout(m, sub, threads=8, row0=ko)
        got = job_slice(out, job[:4])
        for k in ("status", "x_ref", "v_imp", "t_end", "n_steps", "n_onset"):
            assert np.array_equal(bits(got[k]), bits(exp[k])), (j, k)
    out32, _ = run_batched(aeb, m, jobs, P, total, aeb.FP32_COMP)
    for j, job in enumerate(jobs[:10]):
        po, oo, n, thr, ko = job
        if n == 0:
            continue
        Pj = {f: P[f][po:po + n].contiguous() for f in ai.FIELDS}
        Oj = aeb.alloc_outputs(n)
        Sj = torch.empty(aeb.JOB_STATS_BYTES, dtype=torch.uint8, device="cuda")
        aeb.aeb_rollout_batched(m, [(0, 0, n, thr, ko)], Pj, aeb.FP32_COMP, Oj, Sj)
        alone = {k: v.cpu().numpy() for k, v in Oj.items()}
        mix = job_slice(out32, job[:4])
        for k in alone:
            assert np.array_equal(bits(alone[k]), bits(mix[k])), (j, k)


def test_batched_shared_params_ttc_sweep(aeb, oracle_mod):
    """Thresholds share one parameter block (the TTC sweep layout): every job
    reads the same rows, writes its own; FP64 is bit-exact per threshold and
    the contact count falls as the threshold grows."""
    m = ai.ttc_model()
    n = 2000
    p = aeb.aeb_sample_params(m, ai.single_scenario(seed=3), 0, n)
    thrs = np.linspace(0.5, 4.0, 8)
    jobs = [(0, j * n, n, float(t)) for j, t in enumerate(thrs)]
    out, stats = run_batched(aeb, m, jobs, to_dev(p), n * len(thrs), aeb.FP64_PLAIN)
    contacts = [s.n_contact for s in stats]
    assert all(contacts[i] >= contacts[i + 1] for i in range(len(contacts) - 1))
    for j in (0, 3, 7):
        exp = oracle_mod.rollout(ai.replace(m, ttc_thr=float(thrs[j])), p, threads=8)
        got = job_slice(out, jobs[j])
        for k in ("status", "x_ref", "v_imp", "n_onset"):
            assert np.array_equal(bits(got[k]), bits(exp[k])), (j, k)


def test_plan_reuse_is_deterministic(aeb):
    m = ai.single_model()
    params, jobs, total = grid_jobs(aeb, m, n_jobs=20, seed=11)
    P = to_dev(params)
    O = aeb.alloc_outputs(total)
    S = torch.empty(aeb.JOB_STATS_BYTES * len(jobs), dtype=torch.uint8, device="cuda")
    plan = aeb.BatchPlan(m, jobs, P, aeb.FP32_COMP, O, S)
    plan.run()
    torch.cuda.synchronize()
    first = bytes(S.cpu().numpy())
    o1 = O["x_ref"].clone()
    S.zero_()
    plan.run()
    torch.cuda.synchronize()
    assert bytes(S.cpu().numpy()) == first
    assert torch.equal(o1, O["x_ref"])
    plan.close()


def test_autotune_and_cache(aeb, tmp_path):
    m = ai.single_model()
    n = 200_000
    p = aeb.aeb_sample_params(m, ai.single_scenario(seed=4), 0, n)
    P = to_dev(p)
    O = aeb.alloc_outputs(n)
    old = aeb.aeb_get_launch_config(aeb.FP32_COMP)
    cache = str(tmp_path / "tune.txt")
    try:
        best = aeb.aeb_autotune(m, P, n, aeb.FP32_COMP, O, cache_path=cache)
        assert best.tile in (32, 64, 128) and 3 <= best.blocks_per_sm <= 8
        cur = aeb.aeb_get_launch_config(aeb.FP32_COMP)
        assert (cur.tile, cur.blocks_per_sm) == (best.tile, best.blocks_per_sm)
        assert open(cache).read().strip().endswith(f"{best.tile} {best.blocks_per_sm}")
        aeb.aeb_set_launch_config(aeb.FP32_COMP, 64, 6)
        again = aeb.aeb_autotune(m, P, n, aeb.FP32_COMP, O, cache_path=cache)
        assert (again.tile, again.blocks_per_sm) == (best.tile, best.blocks_per_sm)
        # any tuned shape gives the same per-sample results
        ref = {k: v.clone() for k, v in O.items()}
        aeb.aeb_set_launch_config(aeb.FP32_COMP, 32, 4)
        aeb.aeb_rollout(m, P, n, aeb.FP32_COMP, O)
        for k in ref:
            assert torch.equal(ref[k], O[k]), k
    finally:
        aeb.aeb_set_launch_config(aeb.FP32_COMP, old.tile, old.blocks_per_sm)


def test_full_grid_sampled(aeb, oracle_mod):
    """The full scenario grid in the benchmark's configuration (4,096 scenarios,
    N log-uniform in [1e3, 6.4e4], ~6.3e7 rollouts, one captured plan):
    every job's counts add up; sampled samples of 16 jobs against the binary64
    oracle within the FP32 tolerance; three whole jobs identical to flat
    launches of their rows."""
    m = ai.single_model()
    grid = ai.grid_scenarios(seed=2)
    total = sum(n for _, n in grid)
    host = {f: np.empty(total, dtype=np.float64) for f in ai.FIELDS}
    jobs, off = [], 0
    for sc, n in grid:
        aeb.aeb_sample_params(m, sc, 0, n, {f: host[f][off:off + n] for f in ai.FIELDS})
        jobs.append((off, off, n, 0.0))
        off += n
    P = to_dev(host)
    which = ("status", "x_ref", "v_imp", "t_end", "n_steps", "n_onset")
    O = aeb.alloc_outputs(total, which=which)
    S = torch.empty(aeb.JOB_STATS_BYTES * len(jobs), dtype=torch.uint8, device="cuda")
    plan = aeb.BatchPlan(m, jobs, P, aeb.FP32_COMP, O, S)
    plan.run()
    torch.cuda.synchronize()
    plan.close()
    st = aeb.job_stats_from_buffer(S, len(jobs))
    assert len(st) == 4096 and sum(s.n for s in st) == total
    for s, (_, _, n, _) in zip(st, jobs):
        assert s.n == n and s.n_stop + s.n_contact + s.n_horizon + s.n_invalid == n
    out = {k: v.cpu().numpy() for k, v in O.items()}
    rng = np.random.default_rng(11)
    for j in rng.choice(len(jobs), 16, replace=False):
        po, oo, n, _ = jobs[j]
        rows = np.sort(rng.choice(n, min(n, 48), replace=False))
        p = {f: host[f][po + rows] for f in ai.FIELDS}
        exp = oracle_mod.rollout(m, p)
        got = {k: out[k][oo + rows] for k in which}
        same = got["status"] == exp["status"]
        gap = p["d0"] - np.where(same, exp["x_ref"], np.minimum(exp["x_ref"], got["x_ref"]))
        assert np.all(same | (np.abs(gap) < 1e-3)), j
        stp = same & (exp["status"] == 0)
        rel = np.abs(got["x_ref"][stp] - exp["x_ref"][stp]) / exp["x_ref"][stp]
        assert rel.size == 0 or rel.max() <= 1e-5, (j, rel.max())
        assert np.array_equal(got["n_onset"], exp["n_onset"])
    for j in (0, 2047, 4095):
        po, oo, n, _ = jobs[j]
        Pj = {f: P[f][po:po + n].contiguous() for f in ai.FIELDS}
        Oj = aeb.alloc_outputs(n, which=which)
        aeb.aeb_rollout(m, Pj, n, aeb.FP32_COMP, Oj)
        for k in which:
            assert np.array_equal(bits(Oj[k].cpu().numpy()), bits(out[k][oo:oo + n])), (j, k)
