"""Failure handling of the serving engine, with every failure made on the host
(aeb_serve_inject_faults; no GPU fault is made): an admission that finds no
rows (AEB_ENOMEM), a wave whose launch reports a CUDA error and a wave whose
completion does (AEB_ECUDA), and a wave that completes late (the watchdog,
AEB_ETIMEOUT).  In each case the failed request's queued chunks are dropped,
its arena rows come back (counters.rows_free returns to the arena size), and
the other requests' statistics are the same bits as on an untouched engine."""
import time

import pytest

import aeb_inputs as ai

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ARENA = 1 << 20


@pytest.fixture(scope="module")
def aeb():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2604_27193_gb300 as aeb
    aeb.build()
    aeb.lib()
    return aeb


def server(aeb, **kw):
    # chunks of 16,384 samples, four to a wave: a 200,000-sample request spans
    # four waves
    args = dict(arena_rows=ARENA, chunk_samples=1 << 14, wave_samples=1 << 16,
                max_waves_in_flight=2, sampler_threads=8, max_request_samples=1 << 19)
    args.update(kw)
    return aeb.Server(ai.single_model(), aeb.FP32_COMP, **args)


def scen(k):
    return ai.scenario_from_means(20.0 + k, 0.4, 0.9, 55.0 + 3 * k, seed=100 + k,
                                  scenario_id=500 + k)


REQS = [(scen(0), 200_000), (scen(1), 120_000), (scen(2), 50_000), (scen(3), 90_000)]


@pytest.fixture(scope="module")
def clean(aeb):
    """Each request's statistics on an engine without faults."""
    srv = server(aeb)
    try:
        out = []
        for sc, n in REQS:
            code, st, _ = srv.poll(srv.submit(sc, n))
            assert code == aeb.OK
            out.append(bytes(st))
        return out
    finally:
        srv.close()


def wait_rows_back(srv, timeout_s=10.0):
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < timeout_s:
        c = srv.counters()
        if c.rows_free == ARENA:
            return c
        time.sleep(0.01)
    raise AssertionError(f"arena rows not returned: {srv.counters().rows_free} of {ARENA}")


def run_all(aeb, srv):
    tickets = [srv.submit(sc, n) for sc, n in REQS]
    res = []
    for t in tickets:
        try:
            code, st, _ = srv.poll(t)
            res.append((code, bytes(st)))
        except aeb.AebError as e:
            res.append((e.code, None))
    return res


def test_admission_failure(aeb, clean):
    srv = server(aeb)
    try:
        srv.inject_faults(fail_admission=2)
        res = run_all(aeb, srv)
        assert res[1][0] == aeb.ENOMEM
        for k in (0, 2, 3):
            assert res[k] == (aeb.OK, clean[k]), k
        c = wait_rows_back(srv)
        assert c.failed == 1 and c.completed == 3
        # the engine keeps serving
        code, st, _ = srv.poll(srv.submit(*REQS[1]))
        assert code == aeb.OK and bytes(st) == clean[1]
    finally:
        srv.close()


def test_wave_launch_failure(aeb, clean):
    srv = server(aeb)
    try:
        srv.inject_faults(fail_wave_launch=1)
        t0 = srv.submit(*REQS[0])
        with pytest.raises(aeb.AebError) as e:
            srv.poll(t0)
        assert e.value.code == aeb.ECUDA
        c = wait_rows_back(srv)
        assert c.failed == 1
        res = run_all(aeb, srv)
        assert [r[0] for r in res] == [aeb.OK] * 4
        assert [r[1] for r in res] == clean
        wait_rows_back(srv)
    finally:
        srv.close()


def test_wave_completion_failure(aeb, clean):
    srv = server(aeb)
    try:
        srv.inject_faults(fail_wave_completion=1)
        t0 = srv.submit(*REQS[0])
        t1 = srv.submit(*REQS[2])
        with pytest.raises(aeb.AebError) as e:
            srv.poll(t0)
        assert e.value.code == aeb.ECUDA
        code, st, _ = srv.poll(t1)
        assert code == aeb.OK and bytes(st) == clean[2]
        c = wait_rows_back(srv)
        assert c.failed == 1 and c.completed == 1
        res = run_all(aeb, srv)
        assert [r[1] for r in res] == clean
    finally:
        srv.close()


def test_wave_watchdog(aeb, clean):
    srv = server(aeb, wave_timeout_ms=200)
    try:
        srv.inject_faults(hold_waves_ms=3000)
        t = srv.submit(*REQS[2])
        t0 = time.perf_counter()
        code, _, _ = srv.poll(t)
        waited = time.perf_counter() - t0
        assert code == aeb.ETIMEOUT and 0.15 < waited < 2.5, (code, waited)
        c = srv.counters()
        assert c.timed_out == 1 and c.failed == 1
        assert c.rows_free < ARENA  # held while the wave is on the GPU
        srv.inject_faults()  # the wave now completes
        wait_rows_back(srv)
        res = run_all(aeb, srv)
        assert [r[1] for r in res] == clean
        assert srv.counters().timed_out == 1
    finally:
        srv.close()
