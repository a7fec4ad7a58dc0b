"""Helpers of the statistics tests: the oracle's reduction as an aeb_stats, and
the rounding bounds of means and standard deviations formed from sums."""
import ctypes as C
import math

import numpy as np

U = 2.0 ** -53


def to_stats(aeb, st, spec):
    """aeb_stats from the oracle's reduction (sums in sample order)."""
    s = aeb.Stats()
    for name, _ in aeb.JobStats._fields_:
        setattr(s, name, getattr(st, name))
    s.lo_d, s.w_d, s.lo_v, s.w_v = spec
    C.memmove(s.hist_d, st.hist_d.ctypes.data, 8 * aeb.NBINS)
    C.memmove(s.hist_v, st.hist_v.ctypes.data, 8 * aeb.NBINS)
    return s


def moment_bounds(vals, n_sum_terms=None):
    """Bounds on |mean_lib - mean| and |sd_lib - sd| when the library forms
    them from sums that carry at most gamma = k u relative error of the sum of
    magnitudes (any summation order), k = the number of terms:
      |d mean| <= gamma sum|x| / k + u |mean|
      |d (k - 1) var| <= (3 gamma + 6 u) sum x^2, so
      |d sd| <= (3 gamma + 6 u) sum x^2 / (k - 1) / (2 sd) + 4 u sd."""
    x = np.asarray(vals, dtype=np.float64)
    k = len(x)
    g = (n_sum_terms or k) * U
    mean = math.fsum(x) / k
    s2 = math.fsum(x * x)
    dm = g * math.fsum(np.abs(x)) / k + U * abs(mean)
    sd = math.sqrt(max(math.fsum((x - mean) ** 2) / (k - 1), 0.0)) if k > 1 else float("nan")
    dsd = (3 * g + 6 * U) * s2 / (k - 1) / (2 * sd) + 4 * U * sd if k > 1 else float("nan")
    return dm, dsd


def check_summary(aeb, oracle_mod, out, sm):
    st = out["status"]
    d = out["x_ref"][st == 0]
    v = out["v_imp"][st == 1]
    n_valid = int(np.count_nonzero(st != 255))
    assert (sm.n, sm.n_valid) == (len(st), n_valid)
    assert (sm.n_stop, sm.n_contact) == (len(d), len(v))
    assert sm.n_horizon == int(np.count_nonzero(st == 2))
    assert sm.n_invalid == int(np.count_nonzero(st == 255))
    for vals, mean, sd, lo, hi in ((d, sm.mean_d, sm.std_d, sm.min_d, sm.max_d),
                                   (v, sm.mean_v, sm.std_v, sm.min_v, sm.max_v)):
        if len(vals) == 0:
            assert math.isnan(mean) and math.isnan(sd) and math.isnan(lo) and math.isnan(hi)
            continue
        m_o, sd_o = oracle_mod.moments(vals)
        dm, dsd = moment_bounds(vals)
        assert abs(mean - m_o) <= dm, (mean, m_o, dm)
        if len(vals) > 1:
            assert abs(sd - sd_o) <= dsd, (sd, sd_o, dsd)
        else:
            assert math.isnan(sd)
        assert lo == vals.min() and hi == vals.max()
    assert sm.p_contact == len(v) / n_valid
    lo, hi = oracle_mod.wilson(len(v), n_valid)
    assert abs(sm.p_contact_lo - lo) <= 1e-15 and abs(sm.p_contact_hi - hi) <= 1e-15
