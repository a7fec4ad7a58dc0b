"""aeb_reduce_noalloc: the reduction for callers that must not allocate device
memory while running (real-time loops that forbid allocation after start-up,
processes whose device memory is already held by another allocator).  It must
give the same result as aeb_reduce, call after call, although every call shares
one fixed scratch array: two calls in a row on different data, the empty set,
and the sizes that fill all 256 slots of the array (2,097,152 samples, and
8,191 fewer, whose last block holds one sample).  A call on a stream it has
never used leaves the device's free memory unchanged.  This file is collected
last on purpose."""
import ctypes as C
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
    L = aeb.lib()
    L.aeb_reduce_noalloc.argtypes = [C.POINTER(aeb.Outputs), C.c_uint64,
                                     C.POINTER(aeb.HistSpec), C.c_void_p, C.c_void_p]
    L.aeb_reduce_noalloc.restype = C.c_int32
    return aeb


def rollout(aeb, m, sc, n, precision):
    p = aeb.aeb_sample_params(m, sc, 0, n)
    P = {f: torch.from_numpy(p[f]).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(n)
    aeb.aeb_rollout(m, P, n, precision, O)
    return O


def same_stats(a, b):
    for k in ("n", "n_stop", "n_contact", "n_horizon", "n_invalid", "steps",
              "min_d", "max_d", "min_v", "max_v", "lo_d", "w_d", "lo_v", "w_v"):
        assert getattr(a, k) == getattr(b, k), k
    assert bytes(a.hist_d) == bytes(b.hist_d) and bytes(a.hist_v) == bytes(b.hist_v)
    for k, kk, cnt in (("sum_d", "sumsq_d", a.n_stop), ("sum_v", "sumsq_v", a.n_contact)):
        for key in (k, kk):
            x, y = getattr(a, key), getattr(b, key)
            assert abs(x - y) <= max(cnt, 1) * 2.3e-16 * abs(y), key


def test_noalloc_matches_reduce_on_two_calls(aeb):
    L = aeb.lib()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(ai.single_model(), ai.single_scenario(seed=51), 100_003, aeb.FP32_COMP,
              aeb.hist_spec()),
             (ai.paper_model(), ai.paper_scenario(seed=52), 65_536, aeb.FP64_PLAIN,
              aeb.hist_spec(20.0, 0.0625, -1.0, 0.25))]
    for m, sc, n, prec, hist in cases:   # two calls in a row, different data
        O = rollout(aeb, m, sc, n, prec)
        S_ref = aeb.alloc_stats()
        aeb.aeb_reduce(O, n, hist, S_ref)
        S = aeb.alloc_stats()
        S.fill_(0xAB)  # stale contents must not matter
        os_ = aeb.outputs_struct(O)
        rc = L.aeb_reduce_noalloc(C.byref(os_), n, C.byref(hist), S.data_ptr(), stream)
        assert rc == aeb.OK, L.aeb_last_error()
        torch.cuda.synchronize()
        same_stats(aeb.stats_from_buffer(S), aeb.stats_from_buffer(S_ref))


def test_noalloc_limit(aeb):
    L = aeb.lib()
    os_ = aeb.outputs_struct(aeb.alloc_outputs(1))
    hist = aeb.hist_spec()
    S = aeb.alloc_stats()
    rc = L.aeb_reduce_noalloc(C.byref(os_), aeb.REDUCE_NOALLOC_MAX_N + 1, C.byref(hist),
                              S.data_ptr(), None)
    assert rc == aeb.EINVAL and b"2097152" in L.aeb_last_error()


@pytest.mark.parametrize("n", [0, 2_097_152 - 8191, 2_097_152])
def test_noalloc_matches_reduce_at_the_edges(aeb, n):
    """n = 0 (one block, no samples) and the two largest block counts: every
    one of the 256 fixed partials is written and read."""
    L = aeb.lib()
    stream = torch.cuda.current_stream().cuda_stream
    m = ai.single_model()
    O = rollout(aeb, m, ai.single_scenario(seed=53), max(n, 1), aeb.FP32_COMP)
    hist = aeb.hist_spec()
    S_ref = aeb.alloc_stats()
    aeb.aeb_reduce(O, n, hist, S_ref)
    for _ in range(2):
        S = aeb.alloc_stats()
        S.fill_(0x5C)
        os_ = aeb.outputs_struct(O)
        rc = L.aeb_reduce_noalloc(C.byref(os_), n, C.byref(hist), S.data_ptr(), stream)
        assert rc == aeb.OK, L.aeb_last_error()
        torch.cuda.synchronize()
        got, ref = aeb.stats_from_buffer(S), aeb.stats_from_buffer(S_ref)
        same_stats(got, ref)
        assert got.n == n and got.n_stop + got.n_contact + got.n_horizon + got.n_invalid == n
    if n == 0:
        assert got.min_d == math.inf and sum(got.hist_d) == 0


def test_noalloc_allocates_nothing(aeb):
    """After a first call has loaded the kernels, a call on a stream the library
    has never seen leaves cudaMemGetInfo's free bytes unchanged (aeb_reduce on a
    new stream would allocate its scratch there; its change is printed)."""
    L = aeb.lib()
    m = ai.single_model()
    n = 300_000
    O = rollout(aeb, m, ai.single_scenario(seed=54), n, aeb.FP32_COMP)
    hist = aeb.hist_spec()
    os_ = aeb.outputs_struct(O)
    S = aeb.alloc_stats()
    S_ref = aeb.alloc_stats()
    warm = torch.cuda.Stream()
    assert L.aeb_reduce_noalloc(C.byref(os_), n, C.byref(hist), S.data_ptr(),
                                warm.cuda_stream) == aeb.OK
    aeb.aeb_reduce(O, n, hist, S_ref)
    torch.cuda.synchronize()
    fresh = torch.cuda.Stream()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rc = L.aeb_reduce_noalloc(C.byref(os_), n, C.byref(hist), S.data_ptr(), fresh.cuda_stream)
        assert rc == aeb.OK, L.aeb_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    same_stats(aeb.stats_from_buffer(S), aeb.stats_from_buffer(S_ref))
    other = torch.cuda.Stream()
    torch.cuda.synchronize()
    f0, _ = torch.cuda.mem_get_info()
    aeb.aeb_reduce(O, n, hist, S_ref, other)
    torch.cuda.synchronize()
    f1, _ = torch.cuda.mem_get_info()
    print("free bytes: aeb_reduce_noalloc on a new stream", free1 - free0,
          "; aeb_reduce on a new stream", f1 - f0)
