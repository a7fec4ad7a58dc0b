"""The C ABI from a C caller on the GPU: the README's example program is built
against include/aeb.h, linked against the library and run, in both precisions,
on the paper's preset (Sec. IV-B, Eq. 11-15; 1e6 samples from seed 1).  Its
printed statistics are compared with the oracle's rollouts and reduction of the
same samples: binary64 counts and steps exact, sums within n 2^-52 sum|x|, mean
and standard deviation within the rounding bounds of their sums, each safe
headway bin (Sec. VI-C: 5, 1, 0.1 % risk) holding the oracle's order
statistic; FP32-compensated moments within the bounds its per-sample tolerance
implies."""
import math
import os
import re
import subprocess

import numpy as np
import pytest

import aeb_inputs as ai
from stat_bounds import moment_bounds

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = 1_000_000


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    import paper_2604_27193_gb300 as aeb
    aeb.build()
    text = open(os.path.join(ROOT, "README.md")).read()
    src_text = re.findall(r"```c\n(.*?)```", text, flags=re.S)[0]
    d = tmp_path_factory.mktemp("c_example")
    src, exe = d / "example.c", d / "example"
    src.write_text(src_text)
    lib_dir = os.path.dirname(aeb._build.LIB)
    subprocess.run(["gcc", "-std=c11", "-O2", "-Wall", "-Werror", "-I",
                    os.path.join(ROOT, "include"), "-o", str(exe), str(src), "-L", lib_dir,
                    "-laeb", "-lm", f"-Wl,-rpath,{lib_dir}"], check=True)
    return str(exe)


def run(program, *args):
    r = subprocess.run([program, *args], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    out = {}
    for line in r.stdout.splitlines():
        if line.startswith("quantile"):
            q, lo, hi = re.match(r"quantile (\S+) in \[(\S+), (\S+)\)", line).groups()
            out[float(q)] = (float(lo), float(hi))
        else:
            t = line.split()
            for k in range(0, len(t), 2):
                out[t[k]] = float(t[k + 1]) if "." in t[k + 1] or "e" in t[k + 1] else int(t[k + 1])
    return out


@pytest.fixture(scope="module")
def oracle_run(oracle_mod):
    m, sc = ai.paper_model(), ai.paper_scenario(seed=1)
    p = oracle_mod.sample(m, sc, 0, N)
    out = oracle_mod.rollout(m, p, threads=os.cpu_count() or 1)
    return out, oracle_mod.reduce(out)


def test_c_example_fp64_against_oracle(program, oracle_run, oracle_mod):
    out, ex = oracle_run
    got = run(program, "fp64")
    assert (got["n"], got["stop"], got["horizon"], got["invalid"], got["steps"]) == \
        (N, ex.n_stop, ex.n_horizon, ex.n_invalid, ex.steps)
    d = out["x_ref"][out["status"] == 0]
    for key, vals in (("sum_d", d), ("sumsq_d", d * d)):
        assert abs(got[key] - math.fsum(vals)) <= len(vals) * 2.0 ** -52 * math.fsum(np.abs(vals))
    m_o, sd_o = oracle_mod.moments(d)
    dm, dsd = moment_bounds(d)
    assert abs(got["mean_d"] - m_o) <= dm and abs(got["std_d"] - sd_o) <= dsd
    for q in (0.95, 0.99, 0.999):
        lo, hi = got[q]
        assert lo <= oracle_mod.quantile(d, q) < hi and hi - lo == 0.125, (q, lo, hi)
    print("C example, binary64:", got)


def test_c_example_fp32_against_oracle(program, oracle_run, oracle_mod):
    out, ex = oracle_run
    got = run(program)
    d = out["x_ref"][out["status"] == 0]
    # stop/horizon flags can differ only at a tie on the horizon step
    dn = abs(got["stop"] - ex.n_stop)
    assert dn <= 2 and got["n"] == N and got["invalid"] == ex.n_invalid
    m_o, sd_o = oracle_mod.moments(d)
    dm, dsd = moment_bounds(d)
    share = dn / len(d) * float(d.max() - d.min())
    assert abs(got["mean_d"] - m_o) <= 1e-5 * m_o + share + 2 * dm
    assert abs(got["std_d"] - sd_o) <= 1e-5 * math.sqrt(float(np.mean(d * d))) + share + 2 * dsd
    for q in (0.95, 0.99, 0.999):
        lo, hi = got[q]
        x = oracle_mod.quantile(d, q)
        # binary32 error moves a sample by <= 1e-5 x: the bin may be the
        # neighbour of the oracle's when the order statistic is that close
        assert lo - 1e-5 * x <= x < hi + 1e-5 * x, (q, lo, x, hi)
    print("C example, FP32-compensated:", got)
