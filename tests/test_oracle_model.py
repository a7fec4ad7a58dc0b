"""Pins of the oracle's rollout (Sec. III, IV-B, IV-D, V-D) against closed forms,
an independent high-order ODE solver, brute-force fixed points, invariants and
degenerate cases.  None of these re-runs the oracle's own formulas."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

import aeb_inputs as ai


def one(params_rows):
    """Build parameter columns from (v0, d0, mu, grade, mass, cd, tau, delay, noise) rows."""
    a = np.array(params_rows, dtype=np.float64).reshape(-1, 9)
    g = 9.81
    return {"v0": a[:, 0].copy(), "d0": a[:, 1].copy(), "mu": a[:, 2].copy(),
            "gs": g * np.sin(a[:, 3]), "gc": g * np.cos(a[:, 3]), "mass": a[:, 4].copy(),
            "cd": a[:, 5].copy(), "tau": a[:, 6].copy(), "t_delay": a[:, 7].copy(),
            "noise": a[:, 8].copy()}


# ---------------------------------------------------------------------------
# Constant deceleration: both axles at their limit (a_cmd = -15), no drag,
# flat road, instantaneous actuator.  D = v0 t_b + v0^2 / (2 mu g).
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("v0,mu,delay", [(15.0, 0.4, 0.1), (35.0, 0.9, 0.3), (27.3, 0.65, 0.0),
                                         (20.0, 0.5, 0.2137)])
def test_constant_deceleration_closed_form(oracle_mod, v0, mu, delay):
    m = ai.Model(a_cmd=-15.0, lead=0)
    p = one([(v0, 0.0, mu, 0.0, 1500.0, 0.0, 0.0, delay, 0.0)])
    o = oracle_mod.rollout(m, p)
    r = mu * m.g
    n_b = math.ceil(delay / m.dt - 1e-9)
    t_b = n_b * m.dt
    D = v0 * t_b + v0 * v0 / (2.0 * r)
    assert o["status"][0] == 0
    # linear refinement inside the last step misses the parabola by <= r dt^2 / 8
    assert abs(o["x_ref"][0] - D) <= r * m.dt ** 2 / 8 + 1e-9
    # the paper's raw D_stop = x(t_{n+1}) lies within r dt^2 / 2 below D
    assert -r * m.dt ** 2 / 2 - 1e-9 <= o["x_raw"][0] - D <= 1e-9
    assert abs(o["t_end"][0] - (t_b + v0 / r)) < 1e-9
    # the closed form with the continuous delay holds up to onset quantisation
    D_cont = v0 * delay + v0 * v0 / (2.0 * r)
    assert abs(o["x_ref"][0] - D_cont) <= v0 * m.dt + r * m.dt ** 2


def test_unsaturated_constant_deceleration(oracle_mod):
    """Demand below both axle limits: the realised deceleration is the demand."""
    m = ai.Model(a_cmd=-3.0, lead=0)
    p = one([(25.0, 0.0, 0.9, 0.0, 1500.0, 0.0, 0.0, 0.0, 0.0)])
    o = oracle_mod.rollout(m, p)
    assert abs(o["x_ref"][0] - 25.0 ** 2 / 6.0) <= 3.0 * m.dt ** 2 / 8 + 1e-9


def test_lumped_cap_closed_form(oracle_mod):
    """Eq. 5 as printed: r = min(|a_cmd|, mu g / (1 + mu h / L))."""
    m = ai.paper_model()
    for mu in (0.4, 0.6, 0.8, 1.0):
        p = one([(30.0, 0.0, mu, 0.0, 1500.0, 0.0, 0.0, 0.0, 0.0)])
        o = oracle_mod.rollout(m, p)
        r = min(6.0, mu * 9.81 / (1.0 + mu * 0.5 / 2.7))
        assert abs(o["x_ref"][0] - 900.0 / (2 * r)) <= r * m.dt ** 2 / 8 + 1e-9


@pytest.mark.parametrize("theta", [-0.08, -0.02, 0.03, 0.1])
def test_grade_closed_form(oracle_mod, theta):
    """Saturated axles on a grade: deceleration mu g cos(theta) + g sin(theta)."""
    m = ai.Model(a_cmd=-15.0, lead=0)
    p = one([(30.0, 0.0, 0.7, theta, 1500.0, 0.0, 0.0, 0.0, 0.0)])
    o = oracle_mod.rollout(m, p)
    c = 0.7 * 9.81 * math.cos(theta) + 9.81 * math.sin(theta)
    assert abs(o["x_ref"][0] - 900.0 / (2 * c)) <= c * m.dt ** 2 / 8 + 1e-9


@pytest.mark.parametrize("v0,mu,mass", [(35.0, 0.9, 200.0), (20.0, 0.4, 300.0), (30.0, 0.7, 1600.0)])
def test_quadratic_drag_closed_form(oracle_mod, v0, mu, mass):
    """dv/dt = -c - k v^2: t_s = atan(v0 sqrt(k/c)) / sqrt(k c),
    D = ln(1 + k v0^2 / c) / (2 k)."""
    m = ai.Model(a_cmd=-15.0, lead=0)
    cd = 0.35
    p = one([(v0, 0.0, mu, 0.0, mass, cd, 0.0, 0.0, 0.0)])
    o = oracle_mod.rollout(m, p)
    k = 1.225 * cd * 2.2 / (2 * mass)
    c = mu * 9.81
    D = math.log1p(k * v0 * v0 / c) / (2 * k)
    ts = math.atan(v0 * math.sqrt(k / c)) / math.sqrt(k * c)
    assert abs(o["x_ref"][0] - D) <= c * m.dt ** 2 / 8 + 1e-8
    assert abs(o["t_end"][0] - ts) <= 1e-8


@pytest.mark.parametrize("tau,delay", [(0.1, 0.0), (0.3, 0.0), (0.15, 0.2), (0.25, 0.123)])
def test_actuator_lag_closed_form(oracle_mod, tau, delay):
    """No drag, flat road, unsaturated demand a_c: after onset t_b,
    v = v0 + a_c (s - tau (1 - e^{-s/tau})), x = v0 t_b + v0 s
    + a_c (s^2/2 - tau s + tau^2 (1 - e^{-s/tau})), s = t - t_b."""
    ac = -3.0
    m = ai.Model(a_cmd=ac, lead=0)
    v0 = 22.0
    p = one([(v0, 0.0, 0.9, 0.0, 1500.0, 0.0, tau, delay, 0.0)])
    o = oracle_mod.rollout(m, p)
    tb = math.ceil(delay / m.dt - 1e-9) * m.dt
    v = lambda s: v0 + ac * (s - tau * (1 - math.exp(-s / tau)))
    x = lambda s: v0 * tb + v0 * s + ac * (s * s / 2 - tau * s + tau * tau * (1 - math.exp(-s / tau)))
    s_stop = brentq(v, 0.0, 60.0, xtol=1e-15)
    assert abs(o["x_ref"][0] - x(s_stop)) <= 3.0 * m.dt ** 2 / 8 + 1e-8
    assert abs(o["t_end"][0] - (tb + s_stop)) <= 1e-8


def _dop853_state(v0, tau, ac, k, gs, T):
    def f(t, y):
        x, v, a = y
        return [v, a - k * v * v - gs, (ac - a) / tau]
    sol = solve_ivp(f, (0.0, T), [0.0, v0, 0.0], method="DOP853", rtol=1e-13, atol=1e-13)
    return sol.y[0, -1], sol.y[1, -1]


def test_rk4_fourth_order_convergence(oracle_mod):
    """Smooth case (lag + drag + grade, demand below the axle limits, run to the
    horizon): the error against DOP853 falls by ~2^4 per halving of dt."""
    v0, tau, ac, mass, cd, theta, T = 30.0, 0.4, -2.0, 1500.0, 0.3, 0.02, 2.0
    k = 1.225 * cd * 2.2 / (2 * mass)
    gs = 9.81 * math.sin(theta)
    x_ref, _ = _dop853_state(v0, tau, ac, k, gs, T)
    errs = []
    for dt in (0.04, 0.02, 0.01):
        m = ai.Model(a_cmd=ac, lead=0, dt=dt, t_max=T)
        p = one([(v0, 0.0, 0.9, theta, mass, cd, tau, 0.0, 0.0)])
        o = oracle_mod.rollout(m, p)
        assert o["status"][0] == 2  # horizon
        errs.append(abs(o["x_ref"][0] - x_ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12.0 < r1 < 20.0 and 12.0 < r2 < 20.0, errs
    m = ai.Model(a_cmd=ac, lead=0, dt=1e-3, t_max=T)
    o = oracle_mod.rollout(m, one([(v0, 0.0, 0.9, theta, mass, cd, tau, 0.0, 0.0)]))
    assert abs(o["x_ref"][0] - x_ref) < 1e-9


# ---------------------------------------------------------------------------
# Contact with a stationary lead at d0
# ---------------------------------------------------------------------------

def _rk4_linear_step(M, c, z, h):
    """One classic RK4 step of z' = M z + c, written as what it is for a linear
    system: z + h sum_{j=0..3} (hM)^j / (j+1)! (M z + c), the degree-4 Taylor
    polynomial of the exact flow (the textbook stability function of RK4)."""
    def mv(A, x):
        return [sum(A[i][k] * x[k] for k in range(3)) for i in range(3)]
    f = [a + b for a, b in zip(mv(M, z), c)]
    term, acc = f, list(f)
    for j in range(1, 4):
        term = [h * t / (j + 1) for t in mv(M, term)]
        acc = [a + t for a, t in zip(acc, term)]
    return [zi + h * ai_ for zi, ai_ in zip(z, acc)]


@pytest.mark.parametrize("steps", [1, 2, 3])
def test_rk4_steps_against_exact_rationals(oracle_mod, steps):
    """Hand-stepped case: no drag, flat road, a cap far above the demand and an
    immediate command, so (x, v, a) follows the linear system x' = v, v' = a,
    a' = (a_cmd - a) / tau.  After 1, 2, 3 steps of dt = 20 ms at tau = 50 ms
    (dt / tau = 0.4, so every RK4 coefficient matters well above rounding) the
    oracle's position equals the exact rational RK4 iterate (Python fractions,
    from the binary64 inputs) to 1e-14 relative."""
    from fractions import Fraction as Fr
    dt, tau, acmd, v0 = 0.02, 0.05, -6.0, 20.0
    m = ai.replace(ai.paper_model(), dt=dt, t_max=steps * dt, a_cmd=acmd)
    p = one([v0, 100.0, 1.2, 0.0, 1500.0, 0.0, tau, 0.0, 0.0])
    out = oracle_mod.rollout(m, p)
    assert out["status"][0] == 2 and out["n_steps"][0] == steps
    it = Fr(1.0 / tau)  # the model's 1 / tau constant, as a binary64 value
    M = [[Fr(0), Fr(1), Fr(0)], [Fr(0), Fr(0), Fr(1)], [Fr(0), Fr(0), -it]]
    c = [Fr(0), Fr(0), it * Fr(acmd)]
    z = [Fr(0), Fr(v0), Fr(0)]
    for _ in range(steps):
        z = _rk4_linear_step(M, c, z, Fr(dt))
    x_exact = float(z[0])
    assert abs(out["x_raw"][0] - x_exact) <= 1e-14 * abs(x_exact), (out["x_raw"][0], x_exact)


@pytest.mark.parametrize("d0,delay", [(40.0, 0.2), (55.5, 0.05), (3.0, 0.3)])
def test_contact_kinematics(oracle_mod, d0, delay):
    v0, mu = 30.0, 0.6
    m = ai.Model(a_cmd=-15.0, lead=1)
    p = one([(v0, d0, mu, 0.0, 1500.0, 0.0, 0.0, delay, 0.0)])
    o = oracle_mod.rollout(m, p)
    r = mu * 9.81
    tb = math.ceil(delay / m.dt - 1e-9) * m.dt
    assert o["status"][0] == 1
    assert o["x_ref"][0] == d0
    if d0 <= v0 * tb:
        vi, tc = v0, d0 / v0
    else:
        rem = d0 - v0 * tb
        vi = math.sqrt(v0 * v0 - 2 * r * rem)
        tc = tb + (v0 - vi) / r
    assert abs(o["v_imp"][0] - vi) <= 1e-5
    assert abs(o["t_end"][0] - tc) <= 1e-6
    assert o["x_raw"][0] >= d0


def test_contact_wins_over_stop(oracle_mod):
    """A car that would stop exactly past the lead makes contact (contact is
    tested first), one that stops short does not."""
    v0, mu = 20.0, 0.5
    r = mu * 9.81
    D = v0 * v0 / (2 * r)
    m = ai.Model(a_cmd=-15.0, lead=1)
    o = oracle_mod.rollout(m, one([(v0, D - 0.01, mu, 0, 1500, 0, 0, 0, 0),
                                   (v0, D + 0.01, mu, 0, 1500, 0, 0, 0, 0),
                                   (v0, D - 0.0005, mu, 0, 1500, 0, 0, 0, 0),
                                   (v0, D + 0.0005, mu, 0, 1500, 0, 0, 0, 0)]))
    assert list(o["status"]) == [1, 0, 1, 0]
    assert o["v_imp"][0] > 0 and o["v_imp"][0] < math.sqrt(2 * r * 0.011)
    assert o["v_imp"][2] > 0 and o["v_imp"][2] < math.sqrt(2 * r * 0.0006)
    # contact is flagged in the step that first reaches the lead
    for i in (0, 2):
        assert 0.0 <= o["x_raw"][i] - o["x_ref"][i] <= o["v_imp"][i] * m.dt + 1e-9


def test_ttc_trigger_step(oracle_mod):
    """Coasting at constant speed (no drag, flat), the trigger fires at the first
    step n with d0 - n v0 dt + noise <= thr v0; braking starts n_delay later."""
    v0, mu, thr, noise, delay = 20.0, 0.8, 1.5, 0.37, 0.15
    dt = 1e-3
    d0 = 80.0
    m = ai.Model(a_cmd=-15.0, lead=1, trigger=1, ttc_thr=thr)
    o = oracle_mod.rollout(m, one([(v0, d0, mu, 0.0, 1500.0, 0.0, 0.0, delay, noise)]))
    q = (d0 + noise - thr * v0) / (v0 * dt)       # 2518.5: far from an integer
    assert abs(q - round(q)) > 0.1
    n_t = math.ceil(q)
    n_b = n_t + math.ceil(delay / dt - 1e-9)
    x_b = v0 * n_b * dt
    r = mu * 9.81
    D = x_b + v0 * v0 / (2 * r)
    assert D < d0
    assert o["status"][0] == 0
    assert abs(o["x_ref"][0] - D) <= r * dt * dt / 8 + 1e-8
    # a positive range bias makes the measured gap larger, so without it the
    # trigger fires earlier and the car stops shorter
    o2 = oracle_mod.rollout(m, one([(v0, d0, mu, 0.0, 1500.0, 0.0, 0.0, delay, 0.0)]))
    assert o2["x_ref"][0] < o["x_ref"][0]
    # a threshold that never fires: no braking, coast into the lead at v0
    m0 = ai.Model(a_cmd=-15.0, lead=1, trigger=1, ttc_thr=-1.0)
    o3 = oracle_mod.rollout(m0, one([(v0, d0, mu, 0.0, 1500.0, 0.0, 0.0, delay, 0.0)]))
    assert o3["status"][0] == 1 and abs(o3["v_imp"][0] - v0) < 1e-9
    assert o3["n_onset"][0] == -1


def test_ttc_probe_records_and_override(oracle_mod):
    """The TTC test hook (used to check the binary32 kernel's trigger ties):
    for a car at constant speed it records x_n = v0 n dt, the measured gap
    d0 - x_n + noise and thr v0 at every step before the trigger, with the
    margin positive before the trigger step and not positive at it; forcing
    the trigger k steps later shifts the stop by v0 k dt (constant
    deceleration after onset); forcing it never coasts into the lead."""
    v0, mu, thr, noise, delay = 20.0, 0.8, 1.5, 0.37, 0.15
    dt = 1e-3
    d0 = 80.0
    m = ai.Model(a_cmd=-15.0, lead=1, trigger=1, ttc_thr=thr)
    p = one([(v0, d0, mu, 0.0, 1500.0, 0.0, 0.0, delay, noise)])
    n_t = math.ceil((d0 + noise - thr * v0) / (v0 * dt))
    nd = math.ceil(delay / dt - 1e-9)
    out, rec = oracle_mod.rollout_probe(m, p, 0, force=-2, lo=0, hi=n_t + 50)
    ref = oracle_mod.rollout(m, p)
    for k in out:
        assert out[k] == ref[k][0] or (math.isnan(out[k]) and math.isnan(ref[k][0])), k
    assert out["n_onset"] == n_t + nd
    steps = np.arange(n_t + 1)
    assert np.allclose(rec["x"][:n_t + 1], v0 * steps * dt, rtol=0, atol=1e-9)
    assert np.allclose(rec["gap_meas"][:n_t + 1], d0 - v0 * steps * dt + noise, rtol=0, atol=1e-9)
    assert np.all(rec["thr_closing"][:n_t + 1] == thr * v0)
    assert np.all(rec["reading"][:n_t + 1] == 1)
    margin = rec["gap_meas"] - rec["thr_closing"]
    assert np.all(margin[:n_t] > 0) and margin[n_t] <= 0
    assert np.all(np.isnan(rec["gap_meas"][n_t + 1:])) and np.all(rec["reading"][n_t + 1:] == -1)
    same, _ = oracle_mod.rollout_probe(m, p, 0, force=n_t)
    assert same == out
    late, _ = oracle_mod.rollout_probe(m, p, 0, force=n_t + 7)
    assert late["n_onset"] == n_t + 7 + nd and late["status"] == 0
    r = mu * 9.81
    assert abs((late["x_ref"] - out["x_ref"]) - v0 * 7 * dt) <= r * dt * dt / 4 + 1e-9
    never, _ = oracle_mod.rollout_probe(m, p, 0, force=-1)
    assert never["n_onset"] == -1 and never["status"] == 1 and abs(never["v_imp"] - v0) < 1e-9


@pytest.mark.parametrize("case", ["plain", "perception", "moving_lead"])
def test_ttc_probe_without_override_is_the_rollout(oracle_mod, case):
    m = ai.ttc_model(thr=2.0)
    sc = ai.single_scenario(seed=77)
    if case == "perception":
        m = ai.replace(m, perc_sigma=0.8, perc_drop=0.2, perc_latency=0.05, perc_seed=5)
    elif case == "moving_lead":
        m = ai.replace(ai.lead_braking_model(lead_decel=4.0), trigger=1, ttc_thr=3.0)
        sc = ai.lead_braking_scenario(seed=78)
    n = 40
    p = oracle_mod.sample(m, sc, 0, n)
    ref = oracle_mod.rollout(m, p, row0=1000)
    for i in range(n):
        out, rec = oracle_mod.rollout_probe(m, p, i, row=1000 + i, lo=0, hi=20_000)
        for k in out:
            assert out[k] == ref[k][i], (i, k)
        tested = rec["reading"] >= 0
        margin = rec["gap_meas"] - rec["thr_closing"]
        fired = tested & (rec["reading"] == 1) & (margin <= 0)
        if ref["n_onset"][i] >= 0:
            # the first step whose present reading has a non-positive margin
            lat = oracle_mod.steps_to_reach(m.perc_latency, m.dt) if case == "perception" else 0
            n_t = int(np.argmax(fired))
            assert fired.any() and ref["n_onset"][i] == n_t + lat + \
                oracle_mod.steps_to_reach(p["t_delay"][i], m.dt)
            assert not tested[n_t + 1:].any()
        else:
            assert not fired.any()


# ---------------------------------------------------------------------------
# Realised deceleration: brute-force fixed point of the force balance
# ---------------------------------------------------------------------------

def brute_per_axle(D, mu, gc, beta, phi, hl):
    r = 0.0
    for _ in range(400):
        r_new = min(beta * D, mu * (gc * phi + r * hl)) + \
            min((1 - beta) * D, mu * (gc * (1 - phi) - r * hl))
        if abs(r_new - r) <= 1e-16 * max(1.0, abs(r)):
            r = r_new
            break
        r = r_new
    return r


def brute_lumped(D, mu, g, hl):
    r = 0.0
    for _ in range(400):
        r = min(D, mu * g - mu * hl * r)
    return r


def test_per_axle_cap_against_fixed_point(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(3000):
        mu = rng.uniform(0.0, 1.2)
        theta = rng.normal(0.0, 0.1)
        gc = 9.81 * math.cos(theta)
        beta = rng.uniform(0.3, 0.9)
        phi = rng.uniform(0.4, 0.7)
        h, L = rng.uniform(0.3, 0.8), rng.uniform(2.3, 3.2)
        D = rng.uniform(0.0, 20.0)
        m = ai.Model(beta=beta, phi_f=phi, h_cg=h, wheelbase=L)
        got = oracle_mod.axle_cap(m, mu, gc, D)
        exp = brute_per_axle(D, mu, gc, beta, phi, h / L)
        assert abs(got - exp) <= 1e-12 * max(1.0, exp), (mu, theta, beta, phi, h, L, D)


def test_per_axle_special_cases(oracle_mod):
    g = 9.81
    # no weight transfer and the brake split matching the load split: min(D, mu g)
    m = ai.Model(h_cg=0.0, beta=0.6, phi_f=0.6)
    for D in (1.0, 5.0, 7.0, 12.0):
        assert abs(oracle_mod.axle_cap(m, 0.7, g, D) - min(D, 0.7 * g)) < 1e-14
    # a large demand saturates both axles: mu g cos(theta)
    m = ai.Model()
    assert abs(oracle_mod.axle_cap(m, 0.8, g * math.cos(0.05), 100.0) - 0.8 * g * math.cos(0.05)) < 1e-13
    # a small demand is met in full
    assert oracle_mod.axle_cap(m, 0.8, g, 0.5) == 0.5


def test_lumped_cap_against_fixed_point(oracle_mod):
    rng = np.random.default_rng(8)
    for _ in range(500):
        mu, D = rng.uniform(0.0, 1.2), rng.uniform(0.0, 15.0)
        m = ai.Model(cap_mode=0, h_cg=0.5, wheelbase=2.7)
        got = oracle_mod.axle_cap(m, mu, 9.81, D)
        assert abs(got - brute_lumped(D, mu, 9.81, 0.5 / 2.7)) <= 1e-12 * max(1.0, got)


def _active_piece(D, mu, gc, beta, phi, hl):
    lines = [D, (mu * gc * phi + (1 - beta) * D) / (1 - mu * hl),
             (beta * D + mu * gc * (1 - phi)) / (1 + mu * hl), mu * gc]
    return int(np.argmin(lines))


@pytest.mark.parametrize("beta,mu,acmd", [
    (0.6, 0.9, -3.0),    # demand met
    (0.95, 0.6, -6.0),   # front axle at its limit
    (0.3, 0.6, -6.0),    # rear axle at its limit
    (0.7, 0.5, -15.0),   # both axles at their limits
])
def test_rollout_with_each_axle_piece_active(oracle_mod, beta, mu, acmd):
    """Instantaneous actuator, no drag, flat road: the realised deceleration is
    the brute-force fixed point r, so D = v0^2 / (2 r); each case makes a
    different piece of the force balance the active one."""
    g, v0 = 9.81, 28.0
    m = ai.Model(a_cmd=acmd, lead=0, beta=beta)
    hl = m.h_cg / m.wheelbase
    r = brute_per_axle(-acmd, mu, g, beta, m.phi_f, hl)
    assert abs(r - oracle_mod.axle_cap(m, mu, g, -acmd)) < 1e-12
    o = oracle_mod.rollout(m, one([(v0, 0.0, mu, 0.0, 1500.0, 0.0, 0.0, 0.0, 0.0)]))
    assert abs(o["x_ref"][0] - v0 * v0 / (2 * r)) <= r * m.dt ** 2 / 8 + 1e-9


def test_each_axle_piece_is_exercised():
    g, hl, phi = 9.81, 0.55 / 2.7, 0.6
    pieces = {_active_piece(-a, mu, g, b, phi, hl)
              for b, mu, a in ((0.6, 0.9, -3.0), (0.95, 0.6, -6.0), (0.3, 0.6, -6.0), (0.7, 0.5, -15.0))}
    assert pieces == {0, 1, 2, 3}


def test_ttc_trigger_step_random(oracle_mod):
    """Random thresholds, gaps and range biases: the oracle's trigger step must be
    the first n with d0 - n v0 dt + noise <= thr v0 (coasting at constant speed),
    which fixes the stopping point to D = v0 (n_t + n_delay) dt + v0^2 / (2 mu g)."""
    rng = np.random.default_rng(21)
    dt, mu, v0 = 1e-3, 0.8, 20.0
    r = mu * 9.81
    rows, expect = [], []
    while len(rows) < 60:
        thr, noise, d0 = rng.uniform(1.5, 4.0), rng.normal(0, 0.5), rng.uniform(60, 120)
        delay = rng.uniform(0.0, 0.3)
        q = (d0 + noise - thr * v0) / (v0 * dt)
        nd = math.ceil(delay / dt - 1e-9)
        if abs(q - round(q)) < 1e-3 or abs(delay / dt - round(delay / dt)) < 1e-3 or q < 0:
            continue
        D = v0 * (math.ceil(q) + nd) * dt + v0 * v0 / (2 * r)
        if D > d0 - 0.5:
            continue
        rows.append((v0, d0, mu, 0.0, 1500.0, 0.0, 0.0, delay, noise, thr))
        expect.append((D, math.ceil(q) + nd))
    for row, (D, nb) in zip(rows, expect):
        m = ai.Model(a_cmd=-15.0, lead=1, trigger=1, ttc_thr=row[9])
        o = oracle_mod.rollout(m, one([row[:9]]))
        assert o["status"][0] == 0 and o["n_onset"][0] == nb
        assert abs(o["x_ref"][0] - D) <= r * dt * dt / 8 + 1e-8, (row, D, o["x_ref"][0])


# ---------------------------------------------------------------------------
# Monotonicity of the stopping distance along one-parameter sweeps
# ---------------------------------------------------------------------------

BASE = dict(v0=25.0, d0=0.0, mu=0.6, grade=0.0, mass=1600.0, cd=0.3, tau=0.2, delay=0.2, noise=0.0)
ORDER = ("v0", "d0", "mu", "grade", "mass", "cd", "tau", "delay", "noise")


@pytest.mark.parametrize("name,values,sign", [
    ("v0", np.linspace(5, 40, 36), +1),
    ("mu", np.linspace(0.1, 1.0, 37), -1),
    ("grade", np.linspace(-0.1, 0.1, 41), -1),
    ("mass", np.linspace(800, 3000, 23), +1),
    ("cd", np.linspace(0.0, 0.8, 17), -1),
    ("tau", np.linspace(0.0, 0.5, 26), +1),
    ("delay", np.linspace(0.0, 0.6, 61), +1),
])
def test_monotone_sweeps(oracle_mod, name, values, sign):
    rows = []
    for val in values:
        row = dict(BASE)
        row[name] = val
        rows.append(tuple(row[k] for k in ORDER))
    m = ai.Model(lead=0)
    d = oracle_mod.rollout(m, one(rows))["x_ref"]
    steps = np.diff(d) * sign
    assert np.all(steps >= -1e-9), (name, d)
    assert d[-1] * sign > d[0] * sign


def test_harder_braking_is_shorter(oracle_mod):
    p = one([(25.0, 0.0, 0.9, 0.0, 1600, 0.3, 0.2, 0.2, 0.0)])
    d = [oracle_mod.rollout(ai.Model(lead=0, a_cmd=a), p)["x_ref"][0]
         for a in (-2.0, -4.0, -6.0, -8.0, -10.0)]
    assert all(d[i] > d[i + 1] for i in range(len(d) - 1))


# ---------------------------------------------------------------------------
# Degenerate inputs
# ---------------------------------------------------------------------------

def test_edge_cases(oracle_mod):
    m = ai.single_model()
    p = ai.edge_params(m)
    o = oracle_mod.rollout(m, p)
    st = o["status"]
    # already stopped / negative speed: stop at x = 0, t = 0
    assert st[0] == 0 and o["x_ref"][0] == 0.0 and o["t_end"][0] == 0.0 and o["n_steps"][0] == 0
    assert st[1] == 0 and o["x_ref"][1] == 0.0
    # instantaneous actuator and no delay run to a normal stop
    assert st[2] == 0 and st[3] == 0
    assert o["x_ref"][2] > o["x_ref"][3]  # delay 0.2 s vs none, tau 0 vs 0.2: delay dominates
    # no grip: drag alone cannot stop the car before the lead
    assert st[4] == 1
    # gap already zero / lead behind: contact at t = 0 with the initial speed
    assert st[5] == 1 and o["t_end"][5] == 0.0 and o["v_imp"][5] == 20.0
    assert st[6] == 1 and o["x_ref"][6] == 0.0
    # downhill crawl on ice: the horizon ends the run
    assert st[7] == 2 and o["t_end"][7] == 10.0 and o["n_steps"][7] == 10000
    assert st[8] in (0, 1) and st[9] == 0 and o["x_ref"][9] < 1e-5
    assert st[10] in (0, 1) and st[11] in (0, 1)
    # invalid samples are flagged and carry NaN outputs
    assert np.all(st[12:] == 255)
    assert np.all(np.isnan(o["x_ref"][12:])) and np.all(o["n_steps"][12:] == 0)


def test_steps_to_reach(oracle_mod):
    assert oracle_mod.steps_to_reach(10.0, 1e-3) == 10000
    assert oracle_mod.steps_to_reach(10.0, 1e-4) == 100000
    assert oracle_mod.steps_to_reach(0.0, 1e-3) == 0
    rng = np.random.default_rng(0)
    for t in rng.uniform(0, 0.5, 500):
        n = oracle_mod.steps_to_reach(t, 1e-3)
        assert n * 1e-3 >= t and (n == 0 or (n - 1) * 1e-3 < t)


# ---------------------------------------------------------------------------
# Moving lead (extension): the lead starts d0 ahead at lead_v0 and brakes at
# lead_decel until it stops.  Pins from closed-form kinematics of both cars.
# ---------------------------------------------------------------------------

def coasting_ego(v0, d0, t_max=10.0):
    """Constant-speed ego car: no drag, flat road, brake onset beyond the horizon."""
    return one([(v0, d0, 0.8, 0.0, 1500.0, 0.0, 0.0, 2.0 * t_max, 0.0)])


def test_moving_lead_contact_while_lead_brakes(oracle_mod):
    """Ego at 20 m/s, lead at 15 m/s braking at 3 m/s^2, 10 m ahead: the gap
    10 - 5 t - 1.5 t^2 closes at t* = (-5 + sqrt(85)) / 3, before the lead stops."""
    m = ai.Model(lead=1, lead_v0=15.0, lead_decel=3.0)
    o = oracle_mod.rollout(m, coasting_ego(20.0, 10.0))
    t = (-5.0 + math.sqrt(85.0)) / 3.0
    assert o["status"][0] == 1
    # the gap is quadratic in t; the linear root inside one step is off by < 1e-7 s
    assert abs(o["t_end"][0] - t) < 1e-7
    assert abs(o["x_ref"][0] - 20.0 * t) < 2e-6
    assert abs(o["v_imp"][0] - (20.0 - (15.0 - 3.0 * t))) < 1e-6  # closing speed
    assert o["n_steps"][0] == math.ceil(t / m.dt)


def test_moving_lead_stops_before_contact(oracle_mod):
    """Lead 10 m/s braking at 5 m/s^2 stops after 2 s and 10 m; the ego at
    8 m/s from 20 m behind reaches it at t = 30 / 8 with closing speed 8."""
    m = ai.Model(lead=1, lead_v0=10.0, lead_decel=5.0)
    o = oracle_mod.rollout(m, coasting_ego(8.0, 20.0))
    assert o["status"][0] == 1
    assert abs(o["t_end"][0] - 30.0 / 8.0) < 1e-9
    assert abs(o["x_ref"][0] - 30.0) < 1e-8
    assert abs(o["v_imp"][0] - 8.0) < 1e-12


def test_moving_lead_both_braking(oracle_mod):
    """Both cars from 20 m/s, ego at a constant 6 m/s^2 (instantaneous
    actuator, cap far above the demand), lead at 7 m/s^2, 3 m ahead: the gap
    3 - t^2 / 2 closes at t = sqrt(6) (the lead stops at 20/7 s), closing
    speed t, ego position 20 t - 3 t^2."""
    m = ai.Model(lead=1, lead_v0=20.0, lead_decel=7.0, cap_mode=ai.CAP_LUMPED, a_cmd=-6.0)
    o = oracle_mod.rollout(m, one([(20.0, 3.0, 5.0, 0.0, 1500.0, 0.0, 0.0, 0.0, 0.0)]))
    t = math.sqrt(6.0)
    assert o["status"][0] == 1
    assert abs(o["t_end"][0] - t) < 1e-7
    assert abs(o["v_imp"][0] - t) < 1e-6
    assert abs(o["x_ref"][0] - (20.0 * t - 3.0 * t * t)) < 2e-6
    # same deceleration for both: the gap never closes; the ego stops at 20^2 / 12
    m2 = ai.replace(m, lead_decel=6.0)
    o2 = oracle_mod.rollout(m2, one([(20.0, 3.0, 5.0, 0.0, 1500.0, 0.0, 0.0, 0.0, 0.0)]))
    assert o2["status"][0] == 0
    assert abs(o2["x_ref"][0] - 400.0 / 12.0) <= 6.0 * m.dt ** 2 / 8 + 1e-9


def test_moving_lead_never_caught(oracle_mod):
    """A lead faster than the coasting ego car is never reached."""
    m = ai.Model(lead=1, lead_v0=25.0, lead_decel=0.0, t_max=5.0)
    o = oracle_mod.rollout(m, coasting_ego(20.0, 1.0, t_max=5.0))
    assert o["status"][0] == 2
    assert abs(o["x_ref"][0] - 100.0) < 1e-9


@pytest.mark.parametrize("thr", [1.5, 2.0, 3.2])
def test_moving_lead_ttc_uses_closing_speed(oracle_mod, thr):
    """TTC trigger against a lead at a constant 12 m/s: the ego car at 20 m/s
    closes at 8 m/s, so the first step start with 60.0037 - 8 t <= 8 thr is
    the trigger step (no delay: it is also the onset step)."""
    m = ai.Model(lead=1, lead_v0=12.0, lead_decel=0.0, trigger=ai.TRIGGER_TTC, ttc_thr=thr)
    p = one([(20.0, 60.0037, 0.8, 0.0, 1500.0, 0.0, 0.0, 0.0, 0.0)])
    o = oracle_mod.rollout(m, p)
    t = (60.0037 - 8.0 * thr) / 8.0
    assert o["n_onset"][0] == math.ceil(t / m.dt)


def test_stationary_lead_unchanged_by_lead_decel(oracle_mod):
    """lead_v0 = 0 is the stationary lead whatever lead_decel says."""
    p = ai.draw_params(ai.single_model(), ai.single_scenario(seed=61), 300)
    a = oracle_mod.rollout(ai.single_model(), p)
    b = oracle_mod.rollout(ai.replace(ai.single_model(), lead_decel=4.0), p)
    for k in a:
        assert np.array_equal(np.asarray(a[k]).view(np.uint8), np.asarray(b[k]).view(np.uint8)), k
