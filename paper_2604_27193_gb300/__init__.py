"""Python binding of libaeb (GB300 Monte Carlo AEB braking rollouts).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels and host sampler.  The entry points have the names of the C ABI
declared in ``include/aeb.h``.  PyTorch is used for device memory and streams.

Importing this package does not build anything; call ``build()`` first (or
``python -m paper_2604_27193_gb300._build``).  If the library is missing the
import of ``lib()`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

FIELDS = ("v0", "d0", "mu", "gs", "gc", "mass", "cd", "tau", "t_delay", "noise")
QUANTITIES = ("v0", "d0", "mu", "grade", "mass", "cd", "tau", "t_delay", "noise")
OUTPUTS = ("status", "x_raw", "x_ref", "v_imp", "t_end", "n_steps", "n_onset")
OUT_DTYPES = {"status": np.uint8, "x_raw": np.float64, "x_ref": np.float64,
              "v_imp": np.float64, "t_end": np.float64, "n_steps": np.int32,
              "n_onset": np.int32}
ABI_VERSION = 6  # AEB_ABI_VERSION of include/aeb.h
NBINS = 4096

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EAGAIN, ECANCELLED, EDEVICE = range(8)
FP64_PLAIN, FP32_COMP = 0, 1
HIST_D, HIST_V = 0, 1
STOP, CONTACT, HORIZON, INVALID = 0, 1, 2, 255


class AebError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"aeb status {code}: {msg}")
        self.code = code


# --------------------------------------------------------------------------
# ctypes mirrors of include/aeb.h
# --------------------------------------------------------------------------

class Model(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "g", "rho", "area", "h_cg", "wheelbase", "beta", "phi_f", "a_cmd", "dt", "t_max",
        "ttc_thr")] + [(n, C.c_int32) for n in ("cap_mode", "trigger", "lead", "reserved")] + [
        (n, C.c_double) for n in ("lead_v0", "lead_decel", "perc_sigma", "perc_drop",
                                  "perc_latency")] + [("perc_seed", C.c_uint64)]


class Dist(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("p0", C.c_double),
                ("p1", C.c_double), ("lo", C.c_double), ("hi", C.c_double)]


class Scenario(C.Structure):
    _fields_ = [(q, Dist) for q in QUANTITIES] + [("seed", C.c_uint64),
                                                   ("scenario_id", C.c_uint64)]


class Params(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in FIELDS]


class Outputs(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in OUTPUTS]


class HistSpec(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("lo_d", "w_d", "lo_v", "w_v")]


class Stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("n", "n_stop", "n_contact", "n_horizon",
                                          "n_invalid", "steps")] + \
        [(n, C.c_double) for n in ("sum_d", "sumsq_d", "min_d", "max_d", "sum_v", "sumsq_v",
                                   "min_v", "max_v", "lo_d", "w_d", "lo_v", "w_v")] + \
        [("hist_d", C.c_uint64 * NBINS), ("hist_v", C.c_uint64 * NBINS)]


class Job(C.Structure):
    _fields_ = [("param_offset", C.c_uint64), ("out_offset", C.c_uint64), ("n", C.c_uint64),
                ("ttc_thr", C.c_double), ("key_offset", C.c_uint64)]


class JobStats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("n", "n_stop", "n_contact", "n_horizon", "n_invalid",
                                          "steps")] + \
        [(n, C.c_double) for n in ("sum_d", "sumsq_d", "min_d", "max_d", "sum_v", "sumsq_v",
                                   "min_v", "max_v")]


class LaunchConfig(C.Structure):
    _fields_ = [("tile", C.c_int32), ("blocks_per_sm", C.c_int32)]


class ServeCfg(C.Structure):
    _fields_ = [("precision", C.c_int32), ("device", C.c_int32), ("arena_rows", C.c_uint64),
                ("chunk_samples", C.c_uint64), ("wave_samples", C.c_uint64),
                ("max_waves_in_flight", C.c_int32), ("sampler_threads", C.c_int32),
                ("max_request_samples", C.c_uint64), ("wave_timeout_ms", C.c_int32),
                ("reserved", C.c_int32)]


class Latency(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("queue_ms", "sample_ms", "gpu_ms", "total_ms")]


class ServeCounters(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("submitted", "completed", "cancelled", "failed",
                                          "rollouts", "waves", "timed_out", "rows_free")]


class ServeFaults(C.Structure):
    _fields_ = [("fail_admission", C.c_uint64), ("fail_wave_launch", C.c_uint64),
                ("fail_wave_completion", C.c_uint64), ("hold_waves_ms", C.c_int32),
                ("reserved", C.c_int32)]


class SweepResult(C.Structure):
    _fields_ = [("threshold", C.c_double)] + \
        [(n, C.c_uint64) for n in ("n", "n_contact", "n_stop", "n_horizon", "n_invalid")] + \
        [(n, C.c_double) for n in ("p_contact", "ci_lo", "ci_hi")]


class WStats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("n", "n_valid", "n_event")] + [
        (n, C.c_double) for n in ("sum_w", "sumsq_w", "sum_we", "sumsq_we")]


class Summary(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("n", "n_valid", "n_stop", "n_contact", "n_horizon",
                                          "n_invalid", "steps")] + \
        [(n, C.c_double) for n in ("mean_steps", "mean_d", "std_d", "min_d", "max_d", "mean_v",
                                   "std_v", "min_v", "max_v", "p_contact", "p_contact_lo",
                                   "p_contact_hi")]


class Prob(C.Structure):
    _fields_ = [("k", C.c_uint64), ("n", C.c_uint64), ("p", C.c_double), ("ci_lo", C.c_double),
                ("ci_hi", C.c_double)]


class IsResult(C.Structure):
    _fields_ = [("n", C.c_uint64), ("n_event", C.c_uint64)] + [
        (n, C.c_double) for n in ("p", "se", "ci_lo", "ci_hi")]


STATS_BYTES = C.sizeof(Stats)
WSTATS_BYTES = C.sizeof(WStats)
JOB_STATS_BYTES = C.sizeof(JobStats)

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    return _build.build(force=force)


def lib():
    """The loaded libaeb.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise ImportError(f"libaeb.so is not built ({_build.LIB}); run "
                                  "paper_2604_27193_gb300.build() first")
            L = C.CDLL(_build.LIB)
            P = C.POINTER
            L.aeb_abi_version.restype = C.c_int32
            L.aeb_last_error.restype = C.c_char_p
            L.aeb_sample_params.argtypes = [P(Model), P(Scenario), C.c_uint64, C.c_uint64,
                                            P(Params), C.c_int32]
            L.aeb_sample_params_is.argtypes = [P(Model), P(Scenario), P(Scenario), C.c_uint64,
                                               C.c_uint64, P(Params), C.c_void_p, C.c_int32]
            L.aeb_reduce_weighted.argtypes = [P(Outputs), C.c_void_p, C.c_uint64, C.c_double,
                                              C.c_void_p, C.c_void_p]
            L.aeb_rollout.argtypes = [P(Model), P(Params), C.c_uint64, C.c_int32, P(Outputs),
                                      C.c_void_p]
            L.aeb_reduce.argtypes = [P(Outputs), C.c_uint64, P(HistSpec), C.c_void_p,
                                     C.c_void_p]
            L.aeb_evaluate.argtypes = [P(Model), P(Params), C.c_uint64, C.c_int32,
                                       P(HistSpec), P(Stats), P(Outputs), C.c_void_p]
            L.aeb_evaluate_scenario.argtypes = [P(Model), P(Scenario), C.c_uint64, C.c_uint64,
                                                C.c_int32, P(HistSpec), C.c_int32, P(Stats),
                                                C.c_void_p]
            L.aeb_batch_create.argtypes = [P(Model), P(Job), C.c_uint32, P(Params), C.c_int32,
                                           P(Outputs), C.c_void_p, P(C.c_void_p)]
            L.aeb_batch_run.argtypes = [C.c_void_p, C.c_void_p]
            L.aeb_batch_destroy.argtypes = [C.c_void_p]
            L.aeb_batch_destroy.restype = None
            L.aeb_rollout_batched.argtypes = [P(Model), P(Job), C.c_uint32, P(Params), C.c_int32,
                                              P(Outputs), C.c_void_p, C.c_void_p]
            L.aeb_get_launch_config.argtypes = [C.c_int32, P(LaunchConfig)]
            L.aeb_set_launch_config.argtypes = [C.c_int32, P(LaunchConfig)]
            L.aeb_autotune.argtypes = [P(Model), P(Params), C.c_uint64, C.c_int32, P(Outputs),
                                       C.c_void_p, C.c_char_p, P(LaunchConfig)]
            L.aeb_serve_create.argtypes = [P(ServeCfg), P(Model), P(C.c_void_p)]
            L.aeb_serve_submit.argtypes = [C.c_void_p, P(Scenario), C.c_uint64, P(C.c_uint64)]
            L.aeb_serve_poll.argtypes = [C.c_void_p, C.c_uint64, C.c_int32, P(JobStats),
                                         P(Latency)]
            L.aeb_serve_cancel.argtypes = [C.c_void_p, C.c_uint64]
            L.aeb_serve_counters_get.argtypes = [C.c_void_p, P(ServeCounters)]
            L.aeb_serve_inject_faults.argtypes = [C.c_void_p, P(ServeFaults)]
            L.aeb_serve_destroy.argtypes = [C.c_void_p]
            L.aeb_serve_destroy.restype = None
            L.aeb_stats_summary.argtypes = [P(Stats), P(Summary)]
            L.aeb_job_stats_summary.argtypes = [P(JobStats), P(Summary)]
            L.aeb_hist_quantile.argtypes = [P(Stats), C.c_int32, C.c_double, P(C.c_double),
                                            P(C.c_double)]
            L.aeb_hist_exceedance.argtypes = [P(Stats), C.c_int32, C.c_double, P(Prob)]
            L.aeb_is_estimate.argtypes = [P(WStats), P(IsResult)]
            for fn in ("aeb_sample_params", "aeb_rollout", "aeb_reduce", "aeb_evaluate",
                       "aeb_batch_create", "aeb_batch_run", "aeb_rollout_batched",
                       "aeb_get_launch_config", "aeb_set_launch_config", "aeb_autotune",
                       "aeb_serve_create", "aeb_serve_submit", "aeb_serve_poll",
                       "aeb_serve_cancel", "aeb_serve_counters_get", "aeb_sample_params_is",
                       "aeb_reduce_weighted", "aeb_stats_summary", "aeb_job_stats_summary",
                       "aeb_hist_quantile", "aeb_hist_exceedance", "aeb_is_estimate",
                       "aeb_serve_inject_faults", "aeb_evaluate_scenario"):
                getattr(L, fn).restype = C.c_int32
            if L.aeb_abi_version() != ABI_VERSION:
                raise ImportError("libaeb.so ABI version mismatch")
            _lib = L
    return _lib


def _check(code: int):
    if code != OK:
        raise AebError(code, lib().aeb_last_error().decode())


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------

def model(m) -> Model:
    """aeb_model from any object (or dict) with the model's attribute names."""
    get = m.__getitem__ if isinstance(m, dict) else lambda k: getattr(m, k)
    s = Model()
    for name, _ in Model._fields_:
        if name != "reserved":
            setattr(s, name, get(name))
    return s


def scenario(sc) -> Scenario:
    s = Scenario()
    for q in QUANTITIES:
        d = getattr(sc, q)
        dst = getattr(s, q)
        dst.kind, dst.p0, dst.p1, dst.lo, dst.hi = d.kind, d.p0, d.p1, d.lo, d.hi
    s.seed, s.scenario_id = sc.seed, sc.scenario_id
    return s


def hist_spec(lo_d=0.0, w_d=0.125, lo_v=0.0, w_v=1.0 / 64.0) -> HistSpec:
    return HistSpec(lo_d, w_d, lo_v, w_v)


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (host or device)."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def params_struct(cols: dict, offset: int = 0) -> Params:
    p = Params()
    for f in FIELDS:
        col = cols[f]
        item = col.element_size() if hasattr(col, "element_size") else col.itemsize
        setattr(p, f, _ptr(col) + offset * item)
    return p


def outputs_struct(out: dict | None) -> Outputs:
    o = Outputs()
    for f in OUTPUTS:
        setattr(o, f, _ptr(out.get(f)) if out else 0)
    return o


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# --------------------------------------------------------------------------
# entry points (names of the C ABI)
# --------------------------------------------------------------------------

def aeb_sample_params(m, sc, first: int, n: int, out: dict | None = None,
                      n_threads: int = 0) -> dict:
    """Host sampling into ``out`` (dict of float64 host arrays / pinned
    tensors); allocates numpy columns when ``out`` is None."""
    if out is None:
        out = {f: np.empty(n, dtype=np.float64) for f in FIELDS}
    ms, ss, ps = model(m), scenario(sc), params_struct(out)
    _check(lib().aeb_sample_params(C.byref(ms), C.byref(ss), first, n, C.byref(ps), n_threads))
    return out


def aeb_sample_params_is(m, nominal, proposal, first: int, n: int, out: dict | None = None,
                         weights=None, n_threads: int = 0):
    """Importance sampling: host draws from ``proposal`` and their likelihood
    ratios to ``nominal``; returns (columns, weights)."""
    if out is None:
        out = {f: np.empty(n, dtype=np.float64) for f in FIELDS}
    if weights is None:
        weights = np.empty(n, dtype=np.float64)
    ms, ps = model(m), params_struct(out)
    sn, sq = scenario(nominal), scenario(proposal)
    _check(lib().aeb_sample_params_is(C.byref(ms), C.byref(sn), C.byref(sq), first, n,
                                      C.byref(ps), C.c_void_p(_ptr(weights)), n_threads))
    return out, weights


def aeb_reduce_weighted(out: dict, weights, n: int, x_thr: float, wstats_dev, stream=None):
    """Asynchronous weighted event sums into ``wstats_dev`` (``WSTATS_BYTES``
    bytes of device memory); event = contact or x_ref > x_thr."""
    os_ = outputs_struct(out)
    _check(lib().aeb_reduce_weighted(C.byref(os_), C.c_void_p(_ptr(weights)), n,
                                     C.c_double(x_thr), C.c_void_p(_ptr(wstats_dev)),
                                     _stream(stream)))


def wstats_from_buffer(buf) -> WStats:
    raw = buf.cpu().numpy().tobytes() if hasattr(buf, "cpu") else bytes(buf)
    return WStats.from_buffer_copy(raw)


def aeb_is_estimate(ws: WStats) -> IsResult:
    """Importance-sampling estimate of the event probability under the nominal
    law, its standard error and the 95 % interval (computed by the library)."""
    r = IsResult()
    _check(lib().aeb_is_estimate(C.byref(ws), C.byref(r)))
    return r


def aeb_rollout(m, params: dict, n: int, precision: int, out: dict, stream=None):
    """Asynchronous rollout of ``n`` device-resident samples into ``out``."""
    ms, ps, os_ = model(m), params_struct(params), outputs_struct(out)
    _check(lib().aeb_rollout(C.byref(ms), C.byref(ps), n, precision, C.byref(os_),
                             _stream(stream)))


def aeb_reduce(out: dict, n: int, hist: HistSpec, stats_dev, stream=None):
    """Asynchronous reduction into ``stats_dev`` (a device buffer of
    ``STATS_BYTES`` bytes, e.g. a uint8 CUDA tensor)."""
    os_ = outputs_struct(out)
    _check(lib().aeb_reduce(C.byref(os_), n, C.byref(hist), _ptr(stats_dev), _stream(stream)))


REDUCE_NOALLOC_MAX_N = 2097152


def aeb_reduce_noalloc(out: dict, n: int, hist: HistSpec, stats_dev, stream=None):
    """aeb_reduce without device allocation (fixed library scratch; at most
    REDUCE_NOALLOC_MAX_N samples; concurrent calls must not overlap)."""
    L = lib()
    fn = L.aeb_reduce_noalloc
    fn.argtypes = [C.POINTER(Outputs), C.c_uint64, C.POINTER(HistSpec), C.c_void_p, C.c_void_p]
    fn.restype = C.c_int32
    os_ = outputs_struct(out)
    _check(fn(C.byref(os_), n, C.byref(hist), _ptr(stats_dev), _stream(stream)))


def aeb_evaluate(m, params_host: dict, n: int, precision: int, hist: HistSpec,
                 host_out: dict | None = None, stream=None) -> Stats:
    """Whole path from host columns; returns the stats (synchronous)."""
    ms, ps = model(m), params_struct(params_host)
    st = Stats()
    os_ = outputs_struct(host_out) if host_out else None
    _check(lib().aeb_evaluate(C.byref(ms), C.byref(ps), n, precision, C.byref(hist),
                              C.byref(st), C.byref(os_) if os_ is not None else None,
                              _stream(stream)))
    return st


def aeb_evaluate_scenario(m, sc, first: int, n: int, precision: int, hist: HistSpec,
                          n_threads: int = 0, stream=None) -> Stats:
    """Whole path from the seed (host sampling overlapped with the upload and
    rollout of the previous chunk); returns the stats (synchronous)."""
    ms, ss = model(m), scenario(sc)
    st = Stats()
    _check(lib().aeb_evaluate_scenario(C.byref(ms), C.byref(ss), first, n, precision,
                                       C.byref(hist), n_threads, C.byref(st), _stream(stream)))
    return st


def jobs_array(jobs) -> "C.Array":
    """ctypes array of aeb_job from (param_offset, out_offset, n, ttc_thr[,
    key_offset]) tuples; key_offset defaults to param_offset."""
    arr = (Job * len(jobs))()
    for k, jb in enumerate(jobs):
        po, oo, n, thr = jb[:4]
        arr[k] = Job(po, oo, n, thr, jb[4] if len(jb) > 4 else po)
    return arr


class BatchPlan:
    """aeb_batch_create / aeb_batch_run / aeb_batch_destroy."""

    def __init__(self, m, jobs, params: dict, precision: int, out: dict, stats_dev):
        self._jobs = jobs_array(jobs)
        ms, ps, os_ = model(m), params_struct(params), outputs_struct(out)
        self._h = C.c_void_p()
        _check(lib().aeb_batch_create(C.byref(ms), self._jobs, len(jobs), C.byref(ps), precision,
                                      C.byref(os_), _ptr(stats_dev), C.byref(self._h)))

    def run(self, stream=None):
        _check(lib().aeb_batch_run(self._h, _stream(stream)))

    def close(self):
        if self._h:
            lib().aeb_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def aeb_rollout_batched(m, jobs, params: dict, precision: int, out: dict, stats_dev,
                        stream=None):
    arr = jobs_array(jobs)
    ms, ps, os_ = model(m), params_struct(params), outputs_struct(out)
    _check(lib().aeb_rollout_batched(C.byref(ms), arr, len(jobs), C.byref(ps), precision,
                                     C.byref(os_), _ptr(stats_dev), _stream(stream)))


def aeb_get_launch_config(precision: int) -> LaunchConfig:
    c = LaunchConfig()
    _check(lib().aeb_get_launch_config(precision, C.byref(c)))
    return c


def aeb_set_launch_config(precision: int, tile: int, blocks_per_sm: int):
    c = LaunchConfig(tile, blocks_per_sm)
    _check(lib().aeb_set_launch_config(precision, C.byref(c)))


def aeb_autotune(m, params: dict, n: int, precision: int, out: dict, stream=None,
                 cache_path: str | None = None) -> LaunchConfig:
    c = LaunchConfig()
    ms, ps, os_ = model(m), params_struct(params), outputs_struct(out)
    _check(lib().aeb_autotune(C.byref(ms), C.byref(ps), n, precision, C.byref(os_),
                              _stream(stream), cache_path.encode() if cache_path else None,
                              C.byref(c)))
    return c


class Server:
    """aeb_serve_create / submit / poll / cancel / destroy."""

    def __init__(self, m, precision: int = FP32_COMP, device: int = 0,
                 arena_rows: int = 1 << 22, chunk_samples: int = 1 << 18,
                 wave_samples: int = 1 << 21, max_waves_in_flight: int = 2,
                 sampler_threads: int = 0, max_request_samples: int = 1_000_000,
                 wave_timeout_ms: int = 0):
        cfg = ServeCfg(precision, device, arena_rows, chunk_samples, wave_samples,
                       max_waves_in_flight, sampler_threads, max_request_samples,
                       wave_timeout_ms, 0)
        self._h = C.c_void_p()
        ms = model(m)
        _check(lib().aeb_serve_create(C.byref(cfg), C.byref(ms), C.byref(self._h)))

    def submit(self, sc, n: int) -> int:
        t = C.c_uint64()
        ss = scenario(sc)
        _check(lib().aeb_serve_submit(self._h, C.byref(ss), n, C.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """(status, JobStats, Latency); status OK, EAGAIN, ETIMEOUT or ECANCELLED
        (other failures raise AebError)."""
        st, lat = JobStats(), Latency()
        code = lib().aeb_serve_poll(self._h, ticket, timeout_ms, C.byref(st), C.byref(lat))
        if code not in (OK, EAGAIN, ETIMEOUT, ECANCELLED):
            _check(code)
        return code, st, lat

    def cancel(self, ticket: int):
        _check(lib().aeb_serve_cancel(self._h, ticket))

    def counters(self) -> ServeCounters:
        c = ServeCounters()
        _check(lib().aeb_serve_counters_get(self._h, C.byref(c)))
        return c

    def inject_faults(self, fail_admission: int = 0, fail_wave_launch: int = 0,
                      fail_wave_completion: int = 0, hold_waves_ms: int = 0):
        """aeb_serve_inject_faults (host-side failures for tests)."""
        f = ServeFaults(fail_admission, fail_wave_launch, fail_wave_completion, hold_waves_ms, 0)
        _check(lib().aeb_serve_inject_faults(self._h, C.byref(f)))

    def close(self):
        if self._h:
            lib().aeb_serve_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def aeb_ttc_sweep(m, scenarios, n_per_scenario: int, thresholds, precision: int = FP32_COMP,
                  per_job: bool = False, stream=None):
    """Per-threshold SweepResult list (and per-(threshold, scenario) JobStats)."""
    L = lib()
    fn = L.aeb_ttc_sweep
    fn.argtypes = [C.POINTER(Model), C.POINTER(Scenario), C.c_uint32, C.c_uint64,
                   C.POINTER(C.c_double), C.c_uint32, C.c_int32, C.POINTER(SweepResult),
                   C.c_void_p, C.c_void_p]
    fn.restype = C.c_int32
    ms = model(m)
    sc = (Scenario * len(scenarios))(*[scenario(s) for s in scenarios])
    th = (C.c_double * len(thresholds))(*[float(t) for t in thresholds])
    res = (SweepResult * len(thresholds))()
    jobs = (JobStats * (len(thresholds) * len(scenarios)))() if per_job else None
    _check(fn(C.byref(ms), sc, len(scenarios), n_per_scenario, th, len(thresholds), precision,
              res, C.cast(jobs, C.c_void_p) if jobs is not None else None, _stream(stream)))
    return (list(res), list(jobs)) if per_job else list(res)


def aeb_stats_merge(acc: Stats, part: Stats) -> Stats:
    """Add `part` into `acc` (host; counts and histograms exact)."""
    fn = lib().aeb_stats_merge
    fn.argtypes = [C.POINTER(Stats), C.POINTER(Stats)]
    fn.restype = C.c_int32
    _check(fn(C.byref(acc), C.byref(part)))
    return acc


def empty_stats(hist: HistSpec | None = None) -> Stats:
    """Identity element of aeb_stats_merge for a histogram spec."""
    h = hist or hist_spec()
    st = Stats()
    st.min_d = st.min_v = float("inf")
    st.max_d = st.max_v = float("-inf")
    st.lo_d, st.w_d, st.lo_v, st.w_v = h.lo_d, h.w_d, h.lo_v, h.w_v
    return st


def aeb_wilson(k: int, n: int, z: float = 1.959963984540054):
    L = lib()
    fn = L.aeb_wilson
    fn.argtypes = [C.c_uint64, C.c_uint64, C.c_double, C.POINTER(C.c_double),
                   C.POINTER(C.c_double)]
    fn.restype = C.c_int32
    lo, hi = C.c_double(), C.c_double()
    _check(fn(k, n, z, C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def aeb_pipe_peaks(stream=None):
    """Measured (fp32 FMA TFLOP/s, fp64 FMA TFLOP/s, fp64 add Tops/s)."""
    L = lib()
    fn = L.aeb_pipe_peaks
    fn.argtypes = [C.POINTER(C.c_double)] * 3 + [C.c_void_p]
    fn.restype = C.c_int32
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(fn(C.byref(a), C.byref(b), C.byref(c), _stream(stream)))
    return a.value, b.value, c.value


def job_stats_from_buffer(buf, n_jobs: int):
    raw = buf.cpu().numpy().tobytes() if hasattr(buf, "cpu") else bytes(buf)
    return (JobStats * n_jobs).from_buffer_copy(raw[:JOB_STATS_BYTES * n_jobs])


# --------------------------------------------------------------------------
# torch conveniences
# --------------------------------------------------------------------------

def alloc_params(n: int, device="cuda", pin: bool = False) -> dict:
    import torch
    if device == "cpu":
        return {f: torch.empty(n, dtype=torch.float64, pin_memory=pin) for f in FIELDS}
    return {f: torch.empty(n, dtype=torch.float64, device=device) for f in FIELDS}


def alloc_outputs(n: int, device="cuda", which=OUTPUTS, pin: bool = False) -> dict:
    import torch
    tdt = {"status": torch.uint8, "x_raw": torch.float64, "x_ref": torch.float64,
           "v_imp": torch.float64, "t_end": torch.float64, "n_steps": torch.int32,
           "n_onset": torch.int32}
    if device == "cpu":
        return {f: torch.empty(n, dtype=tdt[f], pin_memory=pin) for f in which}
    return {f: torch.empty(n, dtype=tdt[f], device=device) for f in which}


def alloc_stats(device="cuda"):
    import torch
    return torch.empty(STATS_BYTES, dtype=torch.uint8, device=device)


def stats_from_buffer(buf) -> Stats:
    """Copy a device/host stats buffer into a Stats struct (synchronises)."""
    raw = buf.cpu().numpy().tobytes() if hasattr(buf, "cpu") else bytes(buf)
    return Stats.from_buffer_copy(raw)


def aeb_stats_summary(st: Stats) -> Summary:
    """Counts, mean / standard deviation / range of D_stop and v_imp and the
    collision probability with its Wilson interval (library call)."""
    r = Summary()
    _check(lib().aeb_stats_summary(C.byref(st), C.byref(r)))
    return r


def aeb_job_stats_summary(st: JobStats) -> Summary:
    """aeb_stats_summary of a per-job reduction (library call)."""
    r = Summary()
    _check(lib().aeb_job_stats_summary(C.byref(st), C.byref(r)))
    return r


def aeb_hist_quantile(st: Stats, q: float, which: int = HIST_D):
    """(lo, hi): the histogram bin that holds the q-quantile (library call)."""
    lo, hi = C.c_double(), C.c_double()
    _check(lib().aeb_hist_quantile(C.byref(st), which, q, C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def aeb_hist_exceedance(st: Stats, x: float, which: int = HIST_D) -> Prob:
    """P(X >= x) at an inner bin edge x, with its Wilson interval (library call)."""
    r = Prob()
    _check(lib().aeb_hist_exceedance(C.byref(st), which, x, C.byref(r)))
    return r
