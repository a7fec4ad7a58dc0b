"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every function ``include/aeb.h`` declares, its ctypes
mirrors match the header's layouts, invalid arguments are rejected before any
device work, and the host sampler reproduces the oracle's sampler bit for bit
(Sec. IV-C: CPU and GPU runs consume identical parameter sets)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import aeb_inputs as ai

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aeb.h")


@pytest.fixture(scope="module")
def aeb():
    import paper_2604_27193_gb300 as aeb
    aeb.build()
    return aeb


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(aeb_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(aeb):
    names = declared_functions()
    assert {"aeb_sample_params", "aeb_rollout", "aeb_reduce", "aeb_evaluate"} <= set(names)
    L = C.CDLL(aeb._build.LIB)
    for n in names:
        assert hasattr(L, n), n
    assert aeb.lib().aeb_abi_version() == aeb.ABI_VERSION == 6


def test_struct_layouts_match_header(aeb, tmp_path):
    probe = tmp_path / "probe.c"
    structs = {"aeb_model": aeb.Model, "aeb_dist": aeb.Dist, "aeb_scenario": aeb.Scenario,
               "aeb_params": aeb.Params, "aeb_outputs": aeb.Outputs,
               "aeb_hist_spec": aeb.HistSpec, "aeb_stats": aeb.Stats, "aeb_job": aeb.Job,
               "aeb_job_stats": aeb.JobStats, "aeb_launch_config": aeb.LaunchConfig,
               "aeb_serve_cfg": aeb.ServeCfg, "aeb_latency": aeb.Latency,
               "aeb_serve_counters": aeb.ServeCounters, "aeb_sweep_result": aeb.SweepResult,
               "aeb_wstats": aeb.WStats, "aeb_summary": aeb.Summary, "aeb_prob": aeb.Prob,
               "aeb_is_result": aeb.IsResult, "aeb_serve_faults": aeb.ServeFaults}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"',
             "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(probe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


def test_launch_config_validation(aeb):
    old = aeb.aeb_get_launch_config(aeb.FP32_COMP)
    for tile, bps in ((16, 4), (48, 4), (512, 4), (64, -1), (64, 99)):
        with pytest.raises(aeb.AebError) as e:
            aeb.aeb_set_launch_config(aeb.FP32_COMP, tile, bps)
        assert e.value.code == aeb.EINVAL
    aeb.aeb_set_launch_config(aeb.FP32_COMP, 128, 5)
    c = aeb.aeb_get_launch_config(aeb.FP32_COMP)
    assert (c.tile, c.blocks_per_sm) == (128, 5)
    aeb.aeb_set_launch_config(aeb.FP32_COMP, old.tile, old.blocks_per_sm)
    with pytest.raises(aeb.AebError):
        aeb.aeb_get_launch_config(7)


def test_batch_rejects_bad_arguments_on_host(aeb):
    L = aeb.lib()
    m = aeb.model(ai.single_model())
    p = aeb.params_struct(_cols(4))
    o = aeb.outputs_struct(None)
    jobs = aeb.jobs_array([(0, 0, 4, 1.0)])
    h = C.c_void_p()
    # no output columns / no jobs / bad threshold: rejected before any device work
    assert L.aeb_batch_create(C.byref(m), jobs, 1, C.byref(p), 1, C.byref(o), 8, C.byref(h)) == aeb.EINVAL
    assert L.aeb_batch_create(C.byref(m), jobs, 0, C.byref(p), 1, C.byref(o), 8, C.byref(h)) == aeb.EINVAL
    assert L.aeb_batch_run(None, None) == aeb.EINVAL
    L.aeb_batch_destroy(None)


def test_serve_rejects_bad_config_on_host(aeb):
    L = aeb.lib()
    m = aeb.model(ai.single_model())
    h = C.c_void_p()
    good = dict(precision=1, device=0, arena_rows=1 << 20, chunk_samples=1 << 16,
                wave_samples=1 << 20, max_waves_in_flight=2, sampler_threads=1,
                max_request_samples=1 << 20)
    for k, v in (("chunk_samples", 100), ("chunk_samples", 0), ("max_waves_in_flight", 0),
                 ("max_waves_in_flight", 9), ("arena_rows", 0), ("precision", 5),
                 ("max_request_samples", 1 << 21), ("wave_samples", 1 << 10)):
        cfg = aeb.ServeCfg(**dict(good, **{k: v}))
        assert L.aeb_serve_create(C.byref(cfg), C.byref(m), C.byref(h)) == aeb.EINVAL, k
    assert L.aeb_serve_submit(None, None, 1, None) == aeb.EINVAL
    assert L.aeb_serve_poll(None, 1, 0, None, None) == aeb.EINVAL
    L.aeb_serve_destroy(None)


@pytest.mark.parametrize("k,n", [(0, 10), (3, 10), (10, 10), (37, 1000), (5000, 100000), (0, 0)])
def test_library_wilson_matches_oracle(aeb, oracle_mod, k, n):
    assert np.allclose(aeb.aeb_wilson(k, n), oracle_mod.wilson(k, n), rtol=0, atol=1e-15)


def _cols(n):
    return {f: np.zeros(n, dtype=np.float64) for f in ai.FIELDS}


def test_invalid_arguments_rejected_on_host(aeb):
    L = aeb.lib()
    m = aeb.model(ai.single_model())
    p = aeb.params_struct(_cols(4))
    o = aeb.outputs_struct(None)
    bad = []
    for field, val in (("dt", 0.0), ("dt", float("nan")), ("t_max", -1.0), ("wheelbase", 0.0),
                       ("cap_mode", 7), ("trigger", 3), ("lead", 2), ("reserved", 1),
                       ("g", float("inf")), ("lead_v0", -1.0), ("lead_decel", -0.5),
                       ("lead_v0", float("nan")), ("perc_sigma", -0.1), ("perc_drop", 1.5),
                       ("perc_latency", -1.0), ("perc_sigma", float("inf"))):
        mm = aeb.model(ai.single_model())
        setattr(mm, field, val)
        bad.append(mm)
    mm = aeb.model(ai.single_model())
    mm.dt, mm.t_max = 1e-9, 10.0  # 1e10 steps
    bad.append(mm)
    for mm in bad:
        assert L.aeb_rollout(C.byref(mm), C.byref(p), 4, 0, C.byref(o), None) == aeb.EINVAL
        assert L.aeb_last_error()
    assert L.aeb_rollout(C.byref(m), C.byref(p), 4, 5, C.byref(o), None) == aeb.EINVAL
    assert L.aeb_rollout(C.byref(m), None, 4, 0, C.byref(o), None) == aeb.EINVAL
    p2 = aeb.params_struct(_cols(4))
    p2.mu = 0
    assert L.aeb_rollout(C.byref(m), C.byref(p2), 4, 0, C.byref(o), None) == aeb.EINVAL
    p3 = aeb.params_struct(_cols(4))
    p3.v0 = p3.v0 + 4
    assert L.aeb_rollout(C.byref(m), C.byref(p3), 4, 0, C.byref(o), None) == aeb.EINVAL
    # n == 0 is a no-op that never touches a device
    assert L.aeb_rollout(C.byref(m), C.byref(p), 0, 0, C.byref(o), None) == aeb.OK
    h = aeb.hist_spec(w_d=0.1)
    assert L.aeb_reduce(C.byref(o), 0, C.byref(h), 8, None) == aeb.EINVAL
    h = aeb.hist_spec()
    assert L.aeb_reduce(C.byref(o), 5, C.byref(h), 8, None) == aeb.EINVAL  # NULL columns


def test_sampler_matches_oracle_bitwise(aeb, oracle_mod):
    """aeb_sample_params and the oracle's sampler are separate implementations
    of the same definition; on the same host they must agree in every bit."""
    cases = [(ai.single_model(), ai.single_scenario(seed=0), 0, 5000),
             (ai.paper_model(), ai.paper_scenario(seed=3), 123456789, 3000)]
    for sc, _n in ai.grid_scenarios()[:3]:
        cases.append((ai.single_model(), sc, 7, 1000))
    for m, sc, first, n in cases:
        got = aeb.aeb_sample_params(m, sc, first, n, n_threads=3)
        exp = oracle_mod.sample(m, sc, first, n)
        for f in ai.FIELDS:
            assert np.array_equal(got[f].view(np.uint64), exp[f].view(np.uint64)), f


def test_sampler_thread_count_invariance(aeb):
    m, sc = ai.single_model(), ai.single_scenario(seed=5)
    a = aeb.aeb_sample_params(m, sc, 0, 20000, n_threads=1)
    b = aeb.aeb_sample_params(m, sc, 0, 20000, n_threads=7)
    c = aeb.aeb_sample_params(m, sc, 0, 20000, n_threads=0)
    for f in ai.FIELDS:
        assert np.array_equal(a[f], b[f]) and np.array_equal(a[f], c[f])


def test_sampler_rejects_bad_distributions(aeb):
    m = ai.single_model()
    for bad in (ai.Dist(9, 0, 1), ai.Dist(ai.UNIFORM, float("nan"), 1.0),
                ai.Dist(ai.NORMAL, 0.0, 1.0, 2.0, 1.0)):
        sc = ai.replace(ai.single_scenario(), mu=bad)
        with pytest.raises(aeb.AebError) as e:
            aeb.aeb_sample_params(m, sc, 0, 10)
        assert e.value.code == aeb.EINVAL
    assert aeb.aeb_sample_params(m, ai.single_scenario(), 0, 0)["v0"].size == 0


def test_importance_sampler_matches_oracle(aeb, oracle_mod):
    """aeb_sample_params_is: the proposal draws bit for bit, the likelihood
    ratios within 1e-12 relative of the oracle's (both via the host libm; the
    expressions are ordered differently), independent of the thread count, and
    incompatible proposals rejected."""
    import numpy as np
    m = ai.paper_model()
    p = ai.paper_scenario(seed=5)
    q = ai.rare_event_proposal(p)
    cols, w = aeb.aeb_sample_params_is(m, p, q, 1000, 9_000, n_threads=3)
    ocols, ow = oracle_mod.sample_is(m, p, q, 1000, 9_000)
    for f in ai.FIELDS:
        assert np.array_equal(cols[f].view(np.uint64), ocols[f].view(np.uint64)), f
    assert np.all(np.abs(w - ow) <= 1e-12 * np.abs(ow))
    c1, w1 = aeb.aeb_sample_params_is(m, p, q, 1000, 9_000, n_threads=1)
    assert np.array_equal(w1.view(np.uint64), w.view(np.uint64))
    with pytest.raises(aeb.AebError) as e:
        aeb.aeb_sample_params_is(m, p, ai.replace(q, tau=ai.uniform(0.1, 0.2)), 0, 10)
    assert e.value.code == aeb.EINVAL


def test_readme_c_example_compiles_and_links(aeb, tmp_path):
    """The C example in the README builds against include/aeb.h and links
    against the library (it is not run: that needs a GPU)."""
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```c\n(.*?)```", text, flags=re.S)
    assert len(blocks) == 1
    src = tmp_path / "example.c"
    src.write_text(blocks[0])
    exe = tmp_path / "example"
    lib_dir = os.path.dirname(aeb._build.LIB)
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-o", str(exe), str(src), "-L", lib_dir, "-laeb", "-lm",
                    f"-Wl,-rpath,{lib_dir}"], check=True)
    assert exe.exists()
