"""The oracle's pins must catch plausible mistakes.  Each case plants one
mistake in a copy of the oracle source (on the CPU, in a temporary directory),
builds it, and runs the oracle pin tests against that build in a child
process: at least one pin has to fail.  The C cases mutate the C oracle; the
Python cases mutate the package's own statistics (interval, quantile,
exceedance, importance-sampling estimate, moments)."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "aeb_oracle.c")

MUTATIONS = [
    ("grade sign", "return ((-r) - (c->k * v) * v) - c->gs;",
     "return ((-r) - (c->k * v) * v) + c->gs;"),
    ("dropped drag", "return ((-r) - (c->k * v) * v) - c->gs;", "return (-r) - c->gs;"),
    ("RK4 stage 3 step", "double v3 = v + h2 * kv2;", "double v3 = v + dt * kv2;"),
    ("RK4 position weights", "double xn = x + h6 * (((v + 2.0 * v2) + 2.0 * v3) + v4);",
     "double xn = x + h6 * (((v + 2.0 * v2) + 2.0 * v2) + v4);"),
    ("front brake share", "c->f1 = (1.0 - m->beta) / (1.0 - mh);",
     "c->f1 = (m->beta) / (1.0 - mh);"),
    ("Eq. 5 sign", "c->cap = (mu * m->g) / (1.0 + mh);", "c->cap = (mu * m->g) / (1.0 - mh);"),
    ("no stop refinement", "double s = v / (v - vn);", "double s = 1.0;"),
    ("actuator stage", "ka2 = (u - a2) * c->it;", "ka2 = (u - a1) * c->it;"),
    ("TTC threshold", "int fire = reading && gap_meas <= m->ttc_thr * closing;",
     "int fire = reading && gap_meas < m->ttc_thr * closing - 0.01;"),
    ("onset rounding", "c->n_delay = om_steps_to_reach(td, m->dt);",
     "c->n_delay = (int64_t)(td / m->dt);"),
    ("impact speed", "*v_imp = v + s * (vn - v);", "*v_imp = vn;"),
    ("Box-Muller angle word", "double u2 = (double)(w1 >> 11) * two_m53;",
     "double u2 = (double)(w0 >> 11) * two_m53;"),
    ("contact test", "if (m->lead && xn >= c->d0) {", "if (m->lead && xn > c->d0 + 1e-3) {"),
    ("Philox key schedule", "if (round > 0) { k0 += W0; k1 += W1; }", "if (round > 0) { k0 += W0; }"),
    ("histogram origin", "double q = floor((x - lo) / w);", "double q = floor(x / w);"),
    ("lead displacement sign", "const double g1 = (c->d0 + lead_pos(m, t1)) - xn;",
     "const double g1 = (c->d0 - lead_pos(m, t1)) - xn;"),
    ("TTC ego speed for closing speed", "closing = v - lead_speed(m, t);", "closing = v;"),
    ("lead never stops", "if (t >= ts) return 0.5 * (vl * ts);",
     "if (t >= ts + 1e9) return 0.5 * (vl * ts);"),
    ("impact speed not relative", "c1 = vn - lead_speed(m, t1);", "c1 = vn;"),
    ("perception word", "double u3 = (double)((w[2] >> sh) & 0xffffffffULL) * two_m32;",
     "double u3 = (double)((w[1] >> sh) & 0xffffffffULL) * two_m32;"),
    ("perception half", "const int sh = (k & 1) ? 0 : 32;", "const int sh = (k & 1) ? 32 : 0;"),
    ("perception pair block", "uint64_t ctr[4] = {row, (uint64_t)k >> 1, 0, 0}",
     "uint64_t ctr[4] = {row, (uint64_t)k, 0, 0}"),
    ("dropout sense", "if (u4 < m->perc_drop) return 0;", "if (u4 > m->perc_drop) return 0;"),
    ("latency onset", "n_b = (n + lat) + c->n_delay;", "n_b = n + c->n_delay;"),
    ("reading index", "reading = perception(m, row, n + lat, &pn);",
     "reading = perception(m, row, n, &pn);"),
    ("IS normal ratio sign", "exp(0.5 * (zq * zq) - 0.5 * (zp * zp))",
     "exp(0.5 * (zp * zp) - 0.5 * (zq * zq))"),
    ("IS uniform ratio inverted", "return (q->p1 - q->p0) / (p->p1 - p->p0);",
     "return (p->p1 - p->p0) / (q->p1 - q->p0);"),
    ("IS atom ignored", "if (mq > 0.0) return cdf_dist(p, p->lo) / mq;", "if (mq < 0.0) return 1.0;"),
    ("rear axle static share", "c->r0 = (c->mg * (1.0 - m->phi_f)) / (1.0 + mh);",
     "c->r0 = (c->mg * m->phi_f) / (1.0 + mh);"),
    ("rear brake share", "c->r1 = m->beta / (1.0 + mh);", "c->r1 = (1.0 - m->beta) / (1.0 + mh);"),
    ("drag constant", "c->k = ((m->rho * cd) * m->area) / (2.0 * mass);",
     "c->k = ((m->rho * cd) * m->area) / mass;"),
    ("actuator rate", "c->it = (tau > 0.0) ? 1.0 / tau : 0.0;", "c->it = (tau > 0.0) ? tau : 0.0;"),
    ("horizon step", "if (n + 1 >= n_max) {", "if (n + 2 >= n_max) {"),
    ("second moment", "st->sumsq_d += d * d;", "st->sumsq_d += d;"),
    ("clamp upper bound", "if (x > d->hi) x = d->hi;", "if (x > d->hi) x = d->lo;"),
    ("normal scale", "x = d->p0 + d->p1 * z;", "x = d->p0 + z;"),
]


PY_MUTATIONS = [
    ("Wilson centre", "centre = (p + z * z / (2.0 * n)) / den", "centre = p / den"),
    ("quantile index", "k = int(np.ceil(q * len(s)))", "k = int(np.floor(q * len(s)))"),
    ("exceedance at the headway", "np.asarray(values) > h", "np.asarray(values) >= h"),
    ("IS variance centring", "var = (math.fsum(y * y) - n * p * p) / (n - 1)",
     "var = math.fsum(y * y) / (n - 1)"),
    ("biased standard deviation", "math.sqrt(math.fsum(r * r) / (k - 1))",
     "math.sqrt(math.fsum(r * r) / k)"),
]

PIN_TESTS = ("test_oracle_rng.py", "test_oracle_model.py", "test_oracle_stats.py",
             "test_oracle_perception.py", "test_oracle_is.py")


def run_pins(env):
    tests = [os.path.join(ROOT, "tests", f) for f in PIN_TESTS]
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           *tests], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=600)


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old}"
    mutated = tmp_path / "m.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "m.so"
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                    str(so), str(mutated), "-lm"], check=True)
    r = run_pins(dict(os.environ, AEB_ORACLE_SO=str(so)))
    assert r.returncode == 1, f"mutation '{name}' survived:\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name,old,new", PY_MUTATIONS, ids=[m[0] for m in PY_MUTATIONS])
def test_planted_python_mistake_is_caught(tmp_path, oracle_mod, name, old, new):
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    shutil.copy(SRC, pkg / "aeb_oracle.c")
    py = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert py.count(old) == 1, f"mutation anchor not unique: {old}"
    (pkg / "__init__.py").write_text(py.replace(old, new))
    env = dict(os.environ, AEB_ORACLE_PKG_ROOT=str(tmp_path), AEB_ORACLE_SO=oracle_mod.build())
    r = run_pins(env)
    assert r.returncode == 1, f"mutation '{name}' survived:\n{r.stdout[-2000:]}"
