"""Serving engine (continuous batching of scenario requests): results are the
same alone and in the mix, match the oracle / the flat path, admission waits
for device rows, and poll / cancel behave as documented.  Failures are made
on the host (a full arena, a cancelled ticket, an unknown ticket); nothing here
faults the GPU."""
import math
import time

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


FIELDS_EXACT = ("n", "n_stop", "n_contact", "n_horizon", "n_invalid", "steps")
FIELDS_FP = ("sum_d", "sumsq_d", "min_d", "max_d", "sum_v", "sumsq_v", "min_v", "max_v")


def same(a, b):
    return bytes(a) == bytes(b)


def small_server(aeb, precision, **kw):
    args = dict(arena_rows=1 << 21, chunk_samples=1 << 14, wave_samples=1 << 16,
                max_waves_in_flight=2, sampler_threads=8, max_request_samples=1 << 20)
    args.update(kw)
    return aeb.Server(ai.single_model(), precision, **args)


def test_alone_equals_in_mix(aeb):
    srv = small_server(aeb, aeb.FP32_COMP)
    try:
        sc = ai.scenario_from_means(25.0, 0.4, 0.9, 60.0, seed=5, scenario_id=77)
        t = srv.submit(sc, 300_000)
        code, alone, _ = srv.poll(t)
        assert code == aeb.OK and alone.n == 300_000
        reqs = ai.request_stream(rate=1000.0, duration=0.02, seed=8, n_lo=1e3, n_hi=2e5)
        tickets = [srv.submit(s, n) for _, s, n in reqs[:10]]
        tA = srv.submit(sc, 300_000)
        tickets += [srv.submit(s, n) for _, s, n in reqs[10:20]]
        code, mixed, _ = srv.poll(tA)
        assert code == aeb.OK
        assert same(alone, mixed), "a request's statistics changed with its company"
        for tk in tickets:
            assert srv.poll(tk)[0] == aeb.OK
        c = srv.counters()
        assert c.completed == 2 + len(tickets) and c.failed == 0 and c.waves >= 5
    finally:
        srv.close()


def test_fp64_serving_matches_oracle(aeb, oracle_mod):
    srv = small_server(aeb, aeb.FP64_PLAIN)
    try:
        m = ai.single_model()
        sc = ai.single_scenario(seed=21)
        n = 40_000
        code, st, lat = srv.poll(srv.submit(sc, n))
        assert code == aeb.OK
        p = oracle_mod.sample(m, sc, 0, n)
        ex = oracle_mod.reduce(oracle_mod.rollout(m, p, threads=8))
        for k in FIELDS_EXACT:
            assert getattr(st, k) == getattr(ex, k), k
        assert (st.min_d, st.max_d, st.min_v, st.max_v) == (ex.min_d, ex.max_d, ex.min_v, ex.max_v)
        assert abs(st.sum_d - ex.sum_d) <= 1e-12 * abs(ex.sum_d)
        assert abs(st.sumsq_v - ex.sumsq_v) <= 1e-12 * abs(ex.sumsq_v)
        assert lat.total_ms >= lat.gpu_ms >= 0 and lat.queue_ms >= 0 and lat.sample_ms >= 0
        assert abs(lat.total_ms - (lat.queue_ms + lat.sample_ms + lat.gpu_ms)) < 1e-6
    finally:
        srv.close()


def test_fp32_serving_matches_flat_path(aeb):
    m = ai.single_model()
    sc = ai.single_scenario(seed=22)
    n = 100_000
    srv = small_server(aeb, aeb.FP32_COMP)
    try:
        code, st, _ = srv.poll(srv.submit(sc, n))
    finally:
        srv.close()
    p = aeb.aeb_sample_params(m, sc, 0, n)
    P = {f: torch.from_numpy(p[f]).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(n)
    aeb.aeb_rollout(m, P, n, aeb.FP32_COMP, O)
    S = aeb.alloc_stats()
    aeb.aeb_reduce(O, n, aeb.hist_spec(), S)
    flat = aeb.stats_from_buffer(S)
    for k in FIELDS_EXACT:
        assert getattr(st, k) == getattr(flat, k), k
    assert (st.min_d, st.max_d) == (flat.min_d, flat.max_d)
    assert abs(st.sum_d - flat.sum_d) <= 1e-12 * abs(flat.sum_d)


def test_admission_waits_for_rows(aeb):
    """Ten requests that together need 7.5x the arena all complete."""
    srv = small_server(aeb, aeb.FP32_COMP, arena_rows=200_000, max_request_samples=200_000)
    try:
        sc = ai.single_scenario(seed=23)
        tickets = [srv.submit(ai.replace(sc, scenario_id=k), 150_000) for k in range(10)]
        for tk in tickets:
            code, st, lat = srv.poll(tk, timeout_ms=60_000)
            assert code == aeb.OK and st.n == 150_000
        assert srv.counters().completed == 10
        with pytest.raises(aeb.AebError):
            srv.submit(sc, 200_001)  # larger than max_request_samples
    finally:
        srv.close()


def test_poll_and_cancel(aeb):
    srv = small_server(aeb, aeb.FP32_COMP, arena_rows=300_000, max_request_samples=300_000)
    try:
        sc = ai.single_scenario(seed=24)
        big = [srv.submit(ai.replace(sc, scenario_id=k), 300_000) for k in range(4)]
        code, _, _ = srv.poll(big[-1], timeout_ms=0)
        assert code == aeb.EAGAIN
        srv.cancel(big[-1])  # still waiting for rows: dropped
        code, _, _ = srv.poll(big[-1])
        assert code == aeb.ECANCELLED
        for tk in big[:-1]:
            assert srv.poll(tk)[0] == aeb.OK
        with pytest.raises(aeb.AebError):
            srv.poll(big[0])  # released ticket
        with pytest.raises(aeb.AebError):
            srv.cancel(12345)
        c = srv.counters()
        assert c.submitted == 4 and c.completed == 3 and c.cancelled == 1
    finally:
        srv.close()


def test_destroy_with_work_in_flight(aeb):
    srv = small_server(aeb, aeb.FP32_COMP)
    sc = ai.single_scenario(seed=25)
    for k in range(6):
        srv.submit(ai.replace(sc, scenario_id=k), 200_000)
    time.sleep(0.01)
    srv.close()  # waits for the waves in flight, drops pending requests


def test_perception_request_alone_equals_in_mix(aeb):
    """With per-step perception the readings are keyed by a sample's index in
    its request, so a request's statistics still do not depend on its company
    or on where it lands in the arena."""
    m = ai.replace(ai.ttc_model(thr=2.0), perc_sigma=0.8, perc_drop=0.2, perc_latency=0.03,
                   perc_seed=3)
    srv = aeb.Server(m, aeb.FP32_COMP, arena_rows=1 << 21, chunk_samples=1 << 14,
                     wave_samples=1 << 16, max_waves_in_flight=2, sampler_threads=8,
                     max_request_samples=1 << 20)
    try:
        sc = ai.scenario_from_means(25.0, 0.4, 0.9, 60.0, seed=5, scenario_id=78)
        code, alone, _ = srv.poll(srv.submit(sc, 200_000))
        assert code == aeb.OK
        reqs = ai.request_stream(rate=1000.0, duration=0.02, seed=9, n_lo=1e3, n_hi=2e5)
        tickets = [srv.submit(s, n) for _, s, n in reqs[:8]]
        tA = srv.submit(sc, 200_000)
        tickets += [srv.submit(s, n) for _, s, n in reqs[8:16]]
        code, mixed, _ = srv.poll(tA)
        assert code == aeb.OK
        assert same(alone, mixed), "a perception request's statistics changed with its company"
        for tk in tickets:
            assert srv.poll(tk)[0] == aeb.OK
    finally:
        srv.close()


def test_largest_request_alone_equals_in_mix(aeb):
    """The bench's serving configuration with a request of 1e6 samples (the
    serving maximum): its statistics are the same bits alone and amid a
    stream of requests of 1e3 to 1e6 samples, and it completes well inside the
    530 ms budget alone."""
    srv = aeb.Server(ai.single_model(), aeb.FP32_COMP, arena_rows=1 << 23,
                     chunk_samples=1 << 18, wave_samples=1 << 21, max_waves_in_flight=2,
                     sampler_threads=0, max_request_samples=1_000_000)
    try:
        sc = ai.scenario_from_means(30.0, 0.5, 0.9, 70.0, seed=6, scenario_id=91)
        t = srv.submit(sc, 1_000_000)
        code, alone, lat = srv.poll(t)
        assert code == aeb.OK and alone.n == 1_000_000
        assert lat.total_ms < 530.0, lat.total_ms
        reqs = ai.request_stream(rate=400.0, duration=0.05, seed=12)
        tickets = [srv.submit(s, n) for _, s, n in reqs[:8]]
        tA = srv.submit(sc, 1_000_000)
        tickets += [srv.submit(s, n) for _, s, n in reqs[8:16]]
        code, mixed, _ = srv.poll(tA)
        assert code == aeb.OK
        assert same(alone, mixed), "the 1e6-sample request changed with its company"
        for tk in tickets:
            assert srv.poll(tk)[0] == aeb.OK
    finally:
        srv.close()
