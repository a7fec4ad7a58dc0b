"""The multi-GPU exchange, run as two gloo ranks on the CPU.  Samples are
independent (Sec. V-A), so a workload shards by sample: rank r draws its own
parameter stream (scenario_id = r) and reduces its shard; the only exchange is
the fixed-size statistics, gathered and merged in rank order.  The merged
statistics must equal those of the whole set: counts and histograms exactly,
sums within n * 2^-52 * sum|x|, and the same bits on every repetition."""
import math
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import aeb_inputs as ai

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def stats_from_outputs(aeb, oracle, out, hist):
    """Host statistics of one shard (oracle reduction of the shard's outputs),
    converted to the library's aeb_stats layout."""
    ex = oracle.reduce(out, hist.lo_d, hist.w_d, hist.lo_v, hist.w_v, aeb.NBINS)
    st = aeb.empty_stats(hist)
    for k in ("n", "n_stop", "n_contact", "n_horizon", "n_invalid", "steps", "sum_d", "sumsq_d",
              "min_d", "max_d", "sum_v", "sumsq_v", "min_v", "max_v"):
        setattr(st, k, getattr(ex, k))
    st.hist_d[:] = [int(x) for x in ex.hist_d]
    st.hist_v[:] = [int(x) for x in ex.hist_v]
    return st


def shard(rank, n):
    m = ai.single_model()
    sc = ai.replace(ai.single_scenario(seed=31), scenario_id=rank)
    return m, sc, n


def worker(rank, world, port, n, q):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    import paper_2604_27193_gb300 as aeb
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m, sc, nn = shard(rank, n)
        p = aeb.aeb_sample_params(m, sc, 0, nn, n_threads=1)
        out = oracle.rollout(m, p)
        local = stats_from_outputs(aeb, oracle, out, aeb.hist_spec())
        gathered = [None] * world
        dist.all_gather_object(gathered, bytes(local))
        merged = aeb.empty_stats(aeb.hist_spec())
        for b in gathered:  # rank order
            aeb.aeb_stats_merge(merged, aeb.Stats.from_buffer_copy(b))
        q.put((rank, bytes(merged)))
    finally:
        dist.destroy_process_group()


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.fixture(scope="module")
def aeb():
    import paper_2604_27193_gb300 as aeb
    aeb.build()
    return aeb


def test_two_rank_merge_equals_whole_set(aeb, oracle_mod):
    world, n = 2, 3000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    results = []
    for _ in range(2):  # twice: the merged bits must repeat
        port = free_port()
        procs = [ctx.Process(target=worker, args=(r, world, port, n, q)) for r in range(world)]
        for p in procs:
            p.start()
        got = dict(q.get(timeout=300) for _ in range(world))
        for p in procs:
            p.join(timeout=60)
            assert p.exitcode == 0
        assert got[0] == got[1], "ranks disagree on the merged statistics"
        results.append(got[0])
    assert results[0] == results[1]
    merged = aeb.Stats.from_buffer_copy(results[0])
    # the whole set, reduced in one piece
    parts = [aeb.aeb_sample_params(*shard(r, n)[:2], 0, n, n_threads=1) for r in range(world)]
    whole = ai.concat_params(parts)
    out = oracle_mod.rollout(ai.single_model(), whole, threads=4)
    ex = oracle_mod.reduce(out)
    for k in ("n", "n_stop", "n_contact", "n_horizon", "n_invalid", "steps", "min_d", "max_d",
              "min_v", "max_v"):
        assert getattr(merged, k) == getattr(ex, k), k
    assert np.array_equal(np.frombuffer(bytes(merged.hist_d), np.uint64), ex.hist_d)
    assert np.array_equal(np.frombuffer(bytes(merged.hist_v), np.uint64), ex.hist_v)
    d = out["x_ref"][out["status"] == 0]
    assert abs(merged.sum_d - math.fsum(d)) <= len(d) * 2.3e-16 * math.fsum(np.abs(d))


def test_merge_rejects_mismatched_histograms(aeb):
    a, b = aeb.empty_stats(aeb.hist_spec()), aeb.empty_stats(aeb.hist_spec(w_d=0.25))
    with pytest.raises(aeb.AebError):
        aeb.aeb_stats_merge(a, b)
