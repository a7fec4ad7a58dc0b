"""Seeded synthetic inputs shared by the tests, ``bench.py`` and ``smoke()``.

This module holds workload descriptions (model constants, per-quantity
distributions, scenario grids, request streams) and numpy draws of parameter
columns.  It holds none of the rollout arithmetic: it does not integrate,
cap, refine or reduce anything, and it imports neither the product library nor
the oracle.  Both sides of every parity test consume what it produces.

Workloads (sizes and distributions):
  * paper preset   - Sec. IV-B / Eq. 11-15: v0~N(30,2^2), mu~N(0.8,0.1^2),
                     theta~N(0,0.05^2), m~N(1500,100^2), Cd~N(0.3,0.05^2),
                     tau=0.15 s, no delay, no lead, lumped Eq. 5 cap, dt=1 ms.
  * single scenario - v0~U(15,35), d0~N(60,5) clipped to [30,90], mu~U(0.4,0.9),
                     grade~N(0,0.02), m~N(1600,100), Cd~U(0.28,0.35), A=2.2,
                     rho=1.225, tau~U(0.1,0.3), delay~U(0.1,0.3), range noise
                     ~N(0,0.5); h=0.55, L=2.7, front bias 0.7; dt=1 ms, 10 s.
  * scenario grid  - 16 x 16 x 16 means (v0 10..40, mu 0.2..0.95, d0 20..100),
                     per-scenario N log-uniform in [1e3, 6.4e4].
  * request stream - Poisson arrivals, means as in the grid, road class
                     dry/wet/icy, N log-uniform in [1e3, 1e6].
  * TTC sweep      - 256 thresholds in [0.5, 4.0] s x 64 scenarios.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

FIELDS = ("v0", "d0", "mu", "gs", "gc", "mass", "cd", "tau", "t_delay", "noise")
QUANTITIES = ("v0", "d0", "mu", "grade", "mass", "cd", "tau", "t_delay", "noise")

CONST, UNIFORM, NORMAL = 0, 1, 2
CAP_LUMPED, CAP_PER_AXLE = 0, 1
TRIGGER_IMMEDIATE, TRIGGER_TTC = 0, 1
INF = float("inf")


@dataclass
class Model:
    g: float = 9.81
    rho: float = 1.225
    area: float = 2.2
    h_cg: float = 0.55
    wheelbase: float = 2.7
    beta: float = 0.7
    phi_f: float = 0.6
    a_cmd: float = -6.0
    dt: float = 1e-3
    t_max: float = 10.0
    ttc_thr: float = 0.0
    cap_mode: int = CAP_PER_AXLE
    trigger: int = TRIGGER_IMMEDIATE
    lead: int = 1
    lead_v0: float = 0.0     # moving lead: initial speed [m/s] (0: stationary)
    lead_decel: float = 0.0  # moving lead: constant braking deceleration [m/s^2]
    perc_sigma: float = 0.0    # per-step perception noise scale [m] (TTC trigger)
    perc_drop: float = 0.0     # probability that a step's reading is missing
    perc_latency: float = 0.0  # age of a reading when it is used [s]
    perc_seed: int = 0         # key of the per-step perception stream


@dataclass
class Dist:
    kind: int = CONST
    p0: float = 0.0
    p1: float = 0.0
    lo: float = -INF
    hi: float = INF


def const(x):
    return Dist(CONST, x, 0.0)


def uniform(a, b, lo=-INF, hi=INF):
    return Dist(UNIFORM, a, b, lo, hi)


def normal(mean, sd, lo=-INF, hi=INF):
    return Dist(NORMAL, mean, sd, lo, hi)


@dataclass
class Scenario:
    v0: Dist = field(default_factory=lambda: uniform(15.0, 35.0))
    d0: Dist = field(default_factory=lambda: normal(60.0, 5.0, 30.0, 90.0))
    mu: Dist = field(default_factory=lambda: uniform(0.4, 0.9))
    grade: Dist = field(default_factory=lambda: normal(0.0, 0.02))
    mass: Dist = field(default_factory=lambda: normal(1600.0, 100.0))
    cd: Dist = field(default_factory=lambda: uniform(0.28, 0.35))
    tau: Dist = field(default_factory=lambda: uniform(0.1, 0.3))
    t_delay: Dist = field(default_factory=lambda: uniform(0.1, 0.3))
    noise: Dist = field(default_factory=lambda: normal(0.0, 0.5))
    seed: int = 0
    scenario_id: int = 0


# --------------------------------------------------------------------------
# Presets
# --------------------------------------------------------------------------

def single_model(dt: float = 1e-3) -> Model:
    """Single-scenario workload: lead at d0, per-axle caps, immediate trigger."""
    return Model(dt=dt)


def single_scenario(seed: int = 0) -> Scenario:
    return Scenario(seed=seed)


def paper_model() -> Model:
    """Sec. IV-B: h = 0.5, L = 2.7, a_cmd = -6, dt = 1 ms, T = 10 s, Eq. 5 cap,
    no lead vehicle (the stopping distance itself is the output)."""
    return Model(h_cg=0.5, cap_mode=CAP_LUMPED, lead=0)


def paper_scenario(seed: int = 0) -> Scenario:
    """Eq. 11-15; tau fixed at 0.15 s; the braking command is issued at t = 0."""
    return Scenario(v0=normal(30.0, 2.0), d0=const(0.0), mu=normal(0.8, 0.1),
                    grade=normal(0.0, 0.05), mass=normal(1500.0, 100.0),
                    cd=normal(0.3, 0.05), tau=const(0.15), t_delay=const(0.0),
                    noise=const(0.0), seed=seed)


def grid_means(n_per_axis: int = 16):
    """Scenario grid: linearly spaced means, endpoints included, v0 fastest."""
    v = np.linspace(10.0, 40.0, n_per_axis)
    m = np.linspace(0.2, 0.95, n_per_axis)
    d = np.linspace(20.0, 100.0, n_per_axis)
    out = []
    for di in d:
        for mi in m:
            for vi in v:
                out.append((float(vi), float(mi), float(di)))
    return out


def scenario_from_means(v_mean: float, mu_lo: float, mu_hi: float, d_mean: float,
                        seed: int, scenario_id: int) -> Scenario:
    """Spread of one grid or request scenario around its means: v0 ~ U(0.6 m, 1.4 m),
    d0 ~ N(m, (m/12)^2) clipped to [m/2, 1.5 m]; other quantities as the single
    scenario."""
    return Scenario(v0=uniform(0.6 * v_mean, 1.4 * v_mean),
                    d0=normal(d_mean, d_mean / 12.0, 0.5 * d_mean, 1.5 * d_mean),
                    mu=uniform(mu_lo, mu_hi), seed=seed, scenario_id=scenario_id)


def grid_scenarios(seed: int = 2, n_per_axis: int = 16):
    """The batched workload: (scenario, sample count) pairs."""
    rng = np.random.default_rng(seed)
    out = []
    for j, (v, mu, d) in enumerate(grid_means(n_per_axis)):
        half = 0.3846 * mu
        sc = scenario_from_means(v, mu - half, mu + half, d, seed, j)
        n = int(round(math.exp(rng.uniform(math.log(1e3), math.log(6.4e4)))))
        out.append((sc, n))
    return out


ROAD_CLASSES = {"dry": (0.7, 0.9), "wet": (0.4, 0.6), "icy": (0.1, 0.25)}


def request_stream(rate: float = 200.0, duration: float = 60.0, seed: int = 3,
                   n_lo: float = 1e3, n_hi: float = 1e6):
    """Serving workload: list of (arrival_time_s, scenario, n_samples)."""
    rng = np.random.default_rng(seed)
    t, out, rid = 0.0, [], 0
    classes = list(ROAD_CLASSES.values())
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        v = rng.uniform(10.0, 40.0)
        d = rng.uniform(20.0, 100.0)
        lo, hi = classes[int(rng.integers(0, 3))]
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        out.append((t, scenario_from_means(v, lo, hi, d, seed, rid), n))
        rid += 1
    return out


def ttc_thresholds(n: int = 256):
    return np.linspace(0.5, 4.0, n)


def ttc_scenarios(n: int = 64, seed: int = 4):
    """The first ``n`` scenarios of a seeded draw of request-style means."""
    rng = np.random.default_rng(seed)
    classes = list(ROAD_CLASSES.values())
    out = []
    for j in range(n):
        v = rng.uniform(10.0, 40.0)
        d = rng.uniform(20.0, 100.0)
        lo, hi = classes[int(rng.integers(0, 3))]
        out.append(scenario_from_means(v, lo, hi, d, seed, j))
    return out


def lead_braking_model(lead_v0: float = 50.0 / 3.6, lead_decel: float = 6.0,
                       dt: float = 1e-3) -> Model:
    """Moving-lead workload: a lead ahead at 50 km/h braking hard (6 m/s^2) at
    t = 0, per-axle caps, immediate trigger."""
    return Model(dt=dt, lead_v0=lead_v0, lead_decel=lead_decel)


def lead_braking_scenario(seed: int = 0, scenario_id: int = 0) -> Scenario:
    """The single-scenario distributions with a short headway, d0 ~ U(12, 40) m."""
    return Scenario(d0=uniform(12.0, 40.0), seed=seed, scenario_id=scenario_id)


def rare_event_proposal(nominal: Scenario, scenario_id: int = 7) -> Scenario:
    """Importance-sampling proposal for long stops of the paper preset (Eq. 11-15):
    faster cars, lower friction, downhill, same kinds and clamp bounds."""
    return replace(nominal, v0=normal(34.0, 2.5), mu=normal(0.62, 0.11),
                   grade=normal(-0.02, 0.05), scenario_id=scenario_id)


def ttc_model(thr: float = 2.0, dt: float = 1e-3) -> Model:
    return Model(dt=dt, trigger=TRIGGER_TTC, ttc_thr=thr)


# --------------------------------------------------------------------------
# numpy draws of parameter columns (independent of the Philox samplers)
# --------------------------------------------------------------------------

def _draw(rng: np.random.Generator, d: Dist, n: int) -> np.ndarray:
    if d.kind == UNIFORM:
        x = rng.uniform(d.p0, d.p1, n)
    elif d.kind == NORMAL:
        x = rng.normal(d.p0, d.p1, n)
    else:
        x = np.full(n, d.p0, dtype=np.float64)
    return np.clip(x, d.lo, d.hi)


def draw_params(model: Model, scenario: Scenario, n: int, seed: int | None = None) -> dict:
    """Ten float64 columns with the scenario's distributions, drawn with numpy's
    PCG64 from ``seed`` (default: the scenario's seed)."""
    rng = np.random.default_rng(scenario.seed if seed is None else seed)
    q = {name: _draw(rng, getattr(scenario, name), n) for name in QUANTITIES}
    return {
        "v0": q["v0"], "d0": q["d0"], "mu": q["mu"],
        "gs": model.g * np.sin(q["grade"]), "gc": model.g * np.cos(q["grade"]),
        "mass": q["mass"], "cd": q["cd"], "tau": q["tau"], "t_delay": q["t_delay"],
        "noise": q["noise"],
    }


def concat_params(parts) -> dict:
    return {f: np.concatenate([p[f] for p in parts]) for f in FIELDS}


def edge_params(model: Model) -> dict:
    """Hand-picked degenerate samples: zero / negative speed, tau = 0, no delay,
    mu = 0, lead already reached, horizon-bound crawl, steep grades and one
    invalid sample of each kind."""
    g = model.g
    rows = [
        # v0,  d0,   mu,  grade, mass,   cd,  tau,  delay, noise
        (0.0, 60.0, 0.8, 0.0, 1500.0, 0.3, 0.15, 0.1, 0.0),     # already stopped
        (-1.0, 60.0, 0.8, 0.0, 1500.0, 0.3, 0.15, 0.1, 0.0),    # negative speed
        (20.0, 60.0, 0.8, 0.0, 1500.0, 0.3, 0.0, 0.2, 0.0),     # instantaneous actuator
        (20.0, 60.0, 0.8, 0.0, 1500.0, 0.3, 0.2, 0.0, 0.0),     # no delay
        (20.0, 60.0, 0.0, 0.0, 1500.0, 0.3, 0.2, 0.1, 0.0),     # no grip: drag only
        (20.0, 0.0, 0.8, 0.0, 1500.0, 0.3, 0.2, 0.1, 0.0),      # gap already zero
        (20.0, -5.0, 0.8, 0.0, 1500.0, 0.3, 0.2, 0.1, 0.0),     # lead behind
        (0.5, 900.0, 0.05, -0.2, 1500.0, 0.3, 0.2, 0.1, 0.0),   # downhill crawl
        (35.0, 30.0, 0.9, 0.2, 1500.0, 0.3, 0.1, 0.3, 0.0),     # steep uphill, close
        (1e-3, 60.0, 0.8, 0.0, 1500.0, 0.3, 0.15, 0.0, 0.0),    # tiny speed
        (30.0, 60.0, 0.8, 0.0, 1500.0, 0.0, 0.15, 0.1, 0.0),    # no drag
        (30.0, 60.0, 0.8, 0.0, 1500.0, 0.3, 0.15, 0.1, 0.0),    # nominal
        (float("nan"), 60.0, 0.8, 0.0, 1500.0, 0.3, 0.15, 0.1, 0.0),  # invalid: NaN
        (30.0, 60.0, 0.8, 0.0, 0.0, 0.3, 0.15, 0.1, 0.0),       # invalid: mass 0
        (30.0, 60.0, 0.8, 0.0, 1500.0, 0.3, -0.1, 0.1, 0.0),    # invalid: tau < 0
        (30.0, 60.0, -0.1, 0.0, 1500.0, 0.3, 0.15, 0.1, 0.0),   # invalid: mu < 0
        (30.0, 60.0, 0.8, 0.0, 1500.0, 0.3, 0.15, -0.1, 0.0),   # invalid: delay < 0
        (30.0, float("inf"), 0.8, 0.0, 1500.0, 0.3, 0.15, 0.1, 0.0),  # invalid: inf
    ]
    a = np.array(rows, dtype=np.float64)
    grade = a[:, 3]
    return {"v0": a[:, 0].copy(), "d0": a[:, 1].copy(), "mu": a[:, 2].copy(),
            "gs": g * np.sin(grade), "gc": g * np.cos(grade), "mass": a[:, 4].copy(),
            "cd": a[:, 5].copy(), "tau": a[:, 6].copy(), "t_delay": a[:, 7].copy(),
            "noise": a[:, 8].copy()}


__all__ = [n for n in dir() if not n.startswith("_")] + ["replace"]
