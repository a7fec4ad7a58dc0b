"""Importance sampling on the device path: the weighted event sums against
their plain definition (math.fsum over the same outputs and weights), a
rare-event probability estimated both ways (plain Monte Carlo with 4e6
samples, importance sampling with 4e5) agreeing within their standard errors,
with a variance reduction, and determinism."""
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


def device_run(aeb, m, cols, n, precision):
    P = {f: torch.from_numpy(np.ascontiguousarray(cols[f])).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(max(n, 1))
    aeb.aeb_rollout(m, P, n, precision, O)
    return O


def weighted(aeb, O, w_dev, n, x_thr):
    S = torch.zeros(aeb.WSTATS_BYTES, dtype=torch.uint8, device="cuda")
    aeb.aeb_reduce_weighted(O, w_dev, n, x_thr, S)
    return aeb.wstats_from_buffer(S), bytes(S.cpu().numpy())


@pytest.mark.parametrize("lead,x_thr", [(0, 120.0), (1, math.inf)])
def test_weighted_sums_against_definition(aeb, lead, x_thr):
    m = ai.replace(ai.paper_model(), lead=lead)
    p = ai.replace(ai.paper_scenario(seed=8), d0=ai.uniform(60.0, 140.0) if lead else ai.const(0.0))
    q = ai.rare_event_proposal(p)
    n = 300_001
    cols, w = aeb.aeb_sample_params_is(m, p, q, 0, n)
    O = device_run(aeb, m, cols, n, aeb.FP64_PLAIN)
    ws, _ = weighted(aeb, O, torch.from_numpy(w).cuda(), n, x_thr)
    st, xr = O["status"].cpu().numpy(), O["x_ref"].cpu().numpy()
    valid = st != 255
    ev = valid & ((st == 1) | (xr > x_thr))
    assert (ws.n, ws.n_valid, ws.n_event) == (n, int(valid.sum()), int(ev.sum()))
    assert ws.n_event > 100
    for got, terms in ((ws.sum_w, w[valid]), (ws.sumsq_w, w[valid] ** 2),
                       (ws.sum_we, w[ev]), (ws.sumsq_we, w[ev] ** 2)):
        exp = math.fsum(terms)
        assert abs(got - exp) <= n * 2.0 ** -52 * math.fsum(np.abs(terms)), (got, exp)
    # importance weights average to one over valid samples
    assert abs(ws.sum_w / ws.n_valid - 1.0) < 5 * np.std(w) / math.sqrt(n)


def test_rare_event_plain_vs_importance(aeb):
    """P(D_stop > 125 m) for the paper preset: plain Monte Carlo on 4e6
    nominal samples against importance sampling on 4e5 proposal samples."""
    m = ai.paper_model()
    p = ai.paper_scenario(seed=9)
    h0 = 125.0
    n_mc, n_is = 4_000_000, 400_000
    cols = aeb.aeb_sample_params(m, p, 0, n_mc)
    O = device_run(aeb, m, cols, n_mc, aeb.FP32_COMP)
    xr = O["x_ref"].cpu().numpy()
    st = O["status"].cpu().numpy()
    p_mc = float(np.mean((st != 255) & (xr > h0)))
    se_mc = math.sqrt(p_mc * (1 - p_mc) / n_mc)
    cols_q, w = aeb.aeb_sample_params_is(m, p, ai.rare_event_proposal(p), 0, n_is)
    Oq = device_run(aeb, m, cols_q, n_is, aeb.FP32_COMP)
    ws, _ = weighted(aeb, Oq, torch.from_numpy(w).cuda(), n_is, h0)
    r = aeb.aeb_is_estimate(ws)
    p_is, se_is = r.p, r.se
    assert abs(p_is - p_mc) < 4 * math.hypot(se_is, se_mc), (p_is, se_is, p_mc, se_mc)
    # variance per sample: plain p (1 - p) against the weighted estimator's
    vr = (p_mc * (1 - p_mc)) / (se_is ** 2 * n_is)
    assert vr > 5, vr
    print("rare event", {"p_mc": p_mc, "se_mc": se_mc, "p_is": p_is, "se_is": se_is, "vr": vr})


def test_deterministic_and_empty(aeb):
    m = ai.paper_model()
    p = ai.paper_scenario(seed=10)
    n = 50_000
    cols, w = aeb.aeb_sample_params_is(m, p, ai.rare_event_proposal(p), 0, n)
    O = device_run(aeb, m, cols, n, aeb.FP32_COMP)
    wd = torch.from_numpy(w).cuda()
    a = weighted(aeb, O, wd, n, 110.0)[1]
    b = weighted(aeb, O, wd, n, 110.0)[1]
    assert a == b
    ws, _ = weighted(aeb, O, wd, 0, 110.0)
    assert (ws.n, ws.n_valid, ws.n_event, ws.sum_w) == (0, 0, 0, 0.0)
