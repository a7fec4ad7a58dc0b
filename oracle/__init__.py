"""Plain FP64 CPU oracle for the AEB Monte Carlo braking rollouts.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_2604_27193_gb300``) never imports, links or executes anything here, and
the two share no code: the C source ``aeb_oracle.c`` is compiled on its own with
``gcc -O2 -ffp-contract=off`` (no fused multiply-add, no fast-math) and loaded
through ctypes.

Every function cites the passage of Karjol & Alawneh, "Real-Time GPU-Accelerated
Monte Carlo Evaluation of Safety-Critical AEB Systems Under Uncertainty", that it
follows; the C file lists the pin of each one.  Nothing here is "parity
unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aeb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libaeb_oracle.so")

FIELDS = ("v0", "d0", "mu", "gs", "gc", "mass", "cd", "tau", "t_delay", "noise")
QUANTITIES = ("v0", "d0", "mu", "grade", "mass", "cd", "tau", "t_delay", "noise")
STOP, CONTACT, HORIZON, INVALID = 0, 1, 2, 255
CAP_LUMPED, CAP_PER_AXLE = 0, 1
TRIGGER_IMMEDIATE, TRIGGER_TTC = 0, 1


class _Model(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "g", "rho", "area", "h_cg", "wheelbase", "beta", "phi_f", "a_cmd", "dt", "t_max",
        "ttc_thr")] + [(n, C.c_int32) for n in ("cap_mode", "trigger", "lead", "pad_")] + [
        (n, C.c_double) for n in ("lead_v0", "lead_decel", "perc_sigma", "perc_drop",
                                  "perc_latency")] + [("perc_seed", C.c_uint64)]


class _Dist(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad_", C.c_int32), ("p0", C.c_double),
                ("p1", C.c_double), ("lo", C.c_double), ("hi", C.c_double)]


class _Scenario(C.Structure):
    _fields_ = [("dist", _Dist * 9), ("seed", C.c_uint64), ("scenario_id", C.c_uint64)]


class _Stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "n", "n_stop", "n_contact", "n_horizon", "n_invalid", "steps")] + [
        (n, C.c_double) for n in ("sum_d", "sumsq_d", "min_d", "max_d",
                                  "sum_v", "sumsq_v", "min_v", "max_v")]


class _Probe(C.Structure):
    _fields_ = [("force", C.c_int64), ("lo", C.c_int64), ("hi", C.c_int64),
                ("x", C.POINTER(C.c_double)), ("gap_meas", C.POINTER(C.c_double)),
                ("thr_closing", C.POINTER(C.c_double)), ("reading", C.POINTER(C.c_int8))]


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``aeb_oracle.c`` into ``oracle/_build/libaeb_oracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    """The loaded oracle.  ``AEB_ORACLE_SO`` may name another build of the same
    source (the mutation tests load deliberately broken copies that way)."""
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(os.environ.get("AEB_ORACLE_SO") or build())
            P = C.POINTER
            L.om_philox4x64_10.argtypes = [P(C.c_uint64), P(C.c_uint64), P(C.c_uint64)]
            L.om_sample.argtypes = [P(_Model), P(_Scenario), C.c_uint64, C.c_uint64,
                                    P(P(C.c_double))]
            L.om_rollout.argtypes = [P(_Model), P(P(C.c_double)), C.c_uint64, C.c_uint64,
                                     P(C.c_uint8), P(C.c_double), P(C.c_double),
                                     P(C.c_double), P(C.c_double), P(C.c_int32),
                                     P(C.c_int32)]
            L.om_reduce.argtypes = [C.c_uint64, P(C.c_uint8), P(C.c_double), P(C.c_double),
                                    P(C.c_int32), P(_Stats),
                                    P(C.c_uint64), C.c_double, C.c_double,
                                    P(C.c_uint64), C.c_double, C.c_double, C.c_int64]
            L.om_axle_cap.argtypes = [P(_Model), C.c_double, C.c_double, C.c_double]
            L.om_axle_cap.restype = C.c_double
            L.om_steps_to_reach.argtypes = [C.c_double, C.c_double]
            L.om_steps_to_reach.restype = C.c_int64
            L.om_perception.argtypes = [P(_Model), C.c_uint64, C.c_int64, P(C.c_double)]
            L.om_perception.restype = C.c_int
            L.om_sample_is.argtypes = [P(_Model), P(_Scenario), P(_Scenario), C.c_uint64,
                                       C.c_uint64, P(P(C.c_double)), P(C.c_double)]
            L.om_sample_is.restype = C.c_int
            L.om_rollout_probe.argtypes = [P(_Model), P(P(C.c_double)), C.c_uint64, C.c_uint64,
                                           P(_Probe), P(C.c_uint8), P(C.c_double),
                                           P(C.c_double), P(C.c_double), P(C.c_double),
                                           P(C.c_int32), P(C.c_int32)]
            L.om_rollout_probe.restype = C.c_int
            _lib = L
    return _lib


def _model(m) -> _Model:
    s = _Model()
    for name, _ in _Model._fields_:
        if name != "pad_":
            setattr(s, name, getattr(m, name))
    return s


def _scenario(sc) -> _Scenario:
    s = _Scenario()
    for j, q in enumerate(QUANTITIES):
        d = getattr(sc, q)
        s.dist[j].kind, s.dist[j].p0, s.dist[j].p1 = d.kind, d.p0, d.p1
        s.dist[j].lo, s.dist[j].hi = d.lo, d.hi
    s.seed, s.scenario_id = sc.seed, sc.scenario_id
    return s


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _cols_array(params: dict, lo: int = 0):
    arr = (C.POINTER(C.c_double) * 10)()
    keep = []
    for j, f in enumerate(FIELDS):
        a = np.ascontiguousarray(params[f], dtype=np.float64)
        keep.append(a)
        arr[j] = C.cast(C.c_void_p(a.ctypes.data + 8 * lo), C.POINTER(C.c_double))
    return arr, keep


# --------------------------------------------------------------------------
# Sampling (Sec. IV-A, IV-C)
# --------------------------------------------------------------------------

def philox4x64_10(ctr, key) -> np.ndarray:
    """One Philox-4x64-10 block for a 4-word counter and a 2-word key."""
    c = (C.c_uint64 * 4)(*[int(x) for x in ctr])
    k = (C.c_uint64 * 2)(*[int(x) for x in key])
    o = (C.c_uint64 * 4)()
    lib().om_philox4x64_10(c, k, o)
    return np.array(list(o), dtype=np.uint64)


def sample(model, scenario, first: int, n: int) -> dict:
    """Parameter sets xi^(first) .. xi^(first+n-1) as ten float64 columns."""
    out = {f: np.empty(n, dtype=np.float64) for f in FIELDS}
    arr = (C.POINTER(C.c_double) * 10)(*[_dptr(out[f]) for f in FIELDS])
    m, s = _model(model), _scenario(scenario)
    lib().om_sample(C.byref(m), C.byref(s), first, n, arr)
    return out


def sample_is(model, nominal, proposal, first: int, n: int):
    """Parameter sets drawn from ``proposal`` (as ``sample`` draws them) and
    their likelihood ratios p(xi) / q(xi) to ``nominal``: (columns, weights)."""
    out = {f: np.empty(n, dtype=np.float64) for f in FIELDS}
    w = np.empty(n, dtype=np.float64)
    arr = (C.POINTER(C.c_double) * 10)(*[_dptr(out[f]) for f in FIELDS])
    m, sp, sq = _model(model), _scenario(nominal), _scenario(proposal)
    if lib().om_sample_is(C.byref(m), C.byref(sp), C.byref(sq), first, n, arr, _dptr(w)) != 0:
        raise ValueError("proposal incompatible with the nominal scenario")
    return out, w


def is_estimate(weights, event):
    """Importance-sampling estimate of P(event) under the nominal scenario, its
    standard error and the 95 % normal interval (plain definitions, fsum)."""
    import math
    n = len(weights)
    y = np.where(event, weights, 0.0)
    p = math.fsum(y) / n
    var = (math.fsum(y * y) - n * p * p) / (n - 1)
    se = math.sqrt(max(var, 0.0) / n)
    return p, se, (p - 1.959963984540054 * se, p + 1.959963984540054 * se)


# --------------------------------------------------------------------------
# Rollouts (Sec. III, IV-D, V-D)
# --------------------------------------------------------------------------

def rollout(model, params: dict, threads: int = 1, row0: int = 0) -> dict:
    """Run every sample of ``params``; ``threads`` > 1 splits the samples into
    contiguous blocks handled by the same single-sample code in parallel (each
    sample keeps its row index, row0 + its position, which keys its
    perception readings)."""
    n = len(params["v0"])
    out = {
        "status": np.empty(n, dtype=np.uint8),
        "x_raw": np.empty(n, dtype=np.float64),
        "x_ref": np.empty(n, dtype=np.float64),
        "v_imp": np.empty(n, dtype=np.float64),
        "t_end": np.empty(n, dtype=np.float64),
        "n_steps": np.empty(n, dtype=np.int32),
        "n_onset": np.empty(n, dtype=np.int32),
    }
    m = _model(model)
    L = lib()

    def run(lo: int, hi: int):
        arr, keep = _cols_array(params, lo)
        P = C.POINTER
        L.om_rollout(C.byref(m), arr, row0 + lo, hi - lo,
                     C.cast(C.c_void_p(out["status"].ctypes.data + lo), P(C.c_uint8)),
                     *[C.cast(C.c_void_p(out[k].ctypes.data + 8 * lo), P(C.c_double))
                       for k in ("x_raw", "x_ref", "v_imp", "t_end")],
                     C.cast(C.c_void_p(out["n_steps"].ctypes.data + 4 * lo), P(C.c_int32)),
                     C.cast(C.c_void_p(out["n_onset"].ctypes.data + 4 * lo), P(C.c_int32)))
        del keep

    threads = max(1, min(int(threads), n)) if n else 1
    if threads == 1:
        run(0, n)
    else:
        edges = np.linspace(0, n, threads + 1).astype(np.int64)
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda t: run(int(edges[t]), int(edges[t + 1])), range(threads)))
    return out


def rollout_probe(model, params: dict, i: int, row: int | None = None, force: int = -2,
                  lo: int = 0, hi: int = 0):
    """Sample i of ``params`` (perception row ``row``, default i) with the TTC
    trigger's test hook: ``force`` >= 0 fires the trigger at that step, -1
    never, -2 leaves the margin test in charge.  Returns (outputs, record):
    outputs as ``rollout`` gives them for this one sample, record a dict of
    arrays over steps [lo, hi): position x_n, measured gap, ttc_thr times the
    closing speed (NaN where the trigger was not tested) and whether the
    reading was present (-1 where not tested).  Test infrastructure for the
    binary32 kernel's trigger ties only."""
    k = max(0, hi - lo)
    rec = {"x": np.full(k, np.nan), "gap_meas": np.full(k, np.nan),
           "thr_closing": np.full(k, np.nan), "reading": np.full(k, -1, dtype=np.int8)}
    pr = _Probe(force, lo, hi, _dptr(rec["x"]), _dptr(rec["gap_meas"]), _dptr(rec["thr_closing"]),
                rec["reading"].ctypes.data_as(C.POINTER(C.c_int8)))
    arr, keep = _cols_array(params)
    st, on, ns = C.c_uint8(), C.c_int32(), C.c_int32()
    xr, xf, vi, te = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    m = _model(model)
    ok = lib().om_rollout_probe(C.byref(m), arr, i, i if row is None else row, C.byref(pr),
                                C.byref(st), C.byref(xr), C.byref(xf), C.byref(vi), C.byref(te),
                                C.byref(ns), C.byref(on))
    del keep
    if not ok:
        raise ValueError("invalid sample")
    out = {"status": st.value, "x_raw": xr.value, "x_ref": xf.value, "v_imp": vi.value,
           "t_end": te.value, "n_steps": ns.value, "n_onset": on.value}
    return out, rec


def axle_cap(model, mu: float, gc: float, D: float) -> float:
    """Realised deceleration for demanded deceleration D (Eq. 5 / per-axle reading)."""
    m = _model(model)
    return lib().om_axle_cap(C.byref(m), mu, gc, D)


def steps_to_reach(t: float, dt: float) -> int:
    return int(lib().om_steps_to_reach(t, dt))


def perception(model, row: int, k: int):
    """(present, noise) of the per-step perception reading of step k for
    parameter row `row`."""
    m = _model(model)
    x = C.c_double(0.0)
    present = lib().om_perception(C.byref(m), row, k, C.byref(x))
    return bool(present), x.value


# --------------------------------------------------------------------------
# Reduction (Sec. VI-B, VI-C)
# --------------------------------------------------------------------------

@dataclass
class Stats:
    n: int
    n_stop: int
    n_contact: int
    n_horizon: int
    n_invalid: int
    steps: int
    sum_d: float
    sumsq_d: float
    min_d: float
    max_d: float
    sum_v: float
    sumsq_v: float
    min_v: float
    max_v: float
    hist_d: np.ndarray
    hist_v: np.ndarray


def reduce(out: dict, lo_d: float = 0.0, w_d: float = 0.125, lo_v: float = 0.0,
           w_v: float = 1.0 / 64.0, nbins: int = 4096) -> Stats:
    n = len(out["status"])
    st = _Stats()
    hd = np.zeros(nbins, dtype=np.uint64)
    hv = np.zeros(nbins, dtype=np.uint64)
    P = C.POINTER
    lib().om_reduce(n, out["status"].ctypes.data_as(P(C.c_uint8)), _dptr(out["x_ref"]),
                    _dptr(out["v_imp"]), out["n_steps"].ctypes.data_as(P(C.c_int32)),
                    C.byref(st), hd.ctypes.data_as(P(C.c_uint64)), lo_d, w_d,
                    hv.ctypes.data_as(P(C.c_uint64)), lo_v, w_v, nbins)
    vals = {name: getattr(st, name) for name, _ in _Stats._fields_}
    return Stats(**vals, hist_d=hd, hist_v=hv)


def moments(values):
    """Mean and unbiased standard deviation of a set of values (Sec. VI-B,
    Table I: mean and standard deviation of the stopping distance), by their
    plain definitions: m = sum(x) / k, sd = sqrt(sum((x - m)^2) / (k - 1)),
    both sums exactly rounded (math.fsum).  (nan, nan) for an empty set; sd is
    nan below two values."""
    import math
    x = np.asarray(values, dtype=np.float64)
    k = len(x)
    if k == 0:
        return float("nan"), float("nan")
    m = math.fsum(x) / k
    if k < 2:
        return m, float("nan")
    r = x - m
    return m, math.sqrt(math.fsum(r * r) / (k - 1))


def quantile(values: np.ndarray, q: float) -> float:
    """Order statistic x_(k), k = ceil(q n) (1-based): the smallest value whose
    empirical CDF reaches q.  The safe headway at risk level p (Sec. VI-C) is
    the (1 - p) quantile of D_stop."""
    s = np.sort(np.asarray(values, dtype=np.float64))
    k = int(np.ceil(q * len(s)))
    k = min(max(k, 1), len(s))
    return float(s[k - 1])


def exceedance(values: np.ndarray, h: float, n_total: int) -> float:
    """P(D_stop > H0) of Eq. 19: the share of all samples whose stopping
    distance exceeds the headway H0."""
    return float(np.count_nonzero(np.asarray(values) > h)) / float(n_total)


def wilson(k: int, n: int, z: float = 1.959963984540054):
    """Wilson score interval for a binomial proportion k/n (the paper gives no
    interval; this is the reading used for collision probabilities)."""
    if n == 0:
        return (0.0, 1.0)
    p = k / n
    den = 1.0 + z * z / n
    centre = (p + z * z / (2.0 * n)) / den
    half = z * np.sqrt(p * (1.0 - p) / n + z * z / (4.0 * n * n)) / den
    return (centre - half, centre + half)
