// stats.cpp -- statistics read off a reduction, on the host: the summary of
// Sec. VI-B (Table I: mean, standard deviation and range of the stopping
// distance; collision probability), the quantiles and exceedance
// probabilities of the fixed-bin histograms (Sec. VI-C, Eq. 19 and the safe
// headways), the importance-sampling estimate (rare events, Sec. VIII), the
// Wilson interval, and the merge of statistics of disjoint sample sets.
// Every function reads fixed-size structs and allocates nothing.
#include <cmath>
#include <cstring>
#include <limits>

#include "aeb_internal.h"
#include "host_util.h"

namespace {

constexpr double kZ95 = 1.959963984540054;  // standard normal 0.975 quantile
constexpr double kNaN = std::numeric_limits<double>::quiet_NaN();
constexpr double kInf = std::numeric_limits<double>::infinity();

// Mean and unbiased standard deviation of k values from their sum and sum of
// squares: m = s / k, var = (ss - (k m) m) / (k - 1) (NaN below two values;
// a negative var from cancellation is clamped to 0).
void mean_std(uint64_t k, double s, double ss, double *mean, double *sd)
{
    if (k == 0) {
        *mean = kNaN;
        *sd = kNaN;
        return;
    }
    const double kk = (double)k;
    const double m = s / kk;
    *mean = m;
    if (k < 2) {
        *sd = kNaN;
        return;
    }
    const double var = (ss - (kk * m) * m) / (kk - 1.0);
    *sd = std::sqrt(var > 0.0 ? var : 0.0);
}

template <class S>
aeb_status summarize(const S &st, aeb_summary *out)
{
    const uint64_t valid = st.n_stop + st.n_contact + st.n_horizon;
    if (valid + st.n_invalid != st.n)
        return aeb::fail(AEB_EINVAL, "statistics are inconsistent: counts do not add up to n");
    aeb_summary r;
    std::memset(&r, 0, sizeof r);
    r.n = st.n;
    r.n_valid = valid;
    r.n_stop = st.n_stop;
    r.n_contact = st.n_contact;
    r.n_horizon = st.n_horizon;
    r.n_invalid = st.n_invalid;
    r.steps = st.steps;
    r.mean_steps = st.n ? (double)st.steps / (double)st.n : kNaN;
    mean_std(st.n_stop, st.sum_d, st.sumsq_d, &r.mean_d, &r.std_d);
    mean_std(st.n_contact, st.sum_v, st.sumsq_v, &r.mean_v, &r.std_v);
    r.min_d = st.n_stop ? st.min_d : kNaN;
    r.max_d = st.n_stop ? st.max_d : kNaN;
    r.min_v = st.n_contact ? st.min_v : kNaN;
    r.max_v = st.n_contact ? st.max_v : kNaN;
    r.p_contact = valid ? (double)st.n_contact / (double)valid : kNaN;
    aeb_wilson(st.n_contact, valid, kZ95, &r.p_contact_lo, &r.p_contact_hi);
    *out = r;
    return AEB_OK;
}

// The histogram `which` of a reduction: its bins, origin, width and the
// number of samples it counts.
aeb_status hist_of(const aeb_stats *st, int32_t which, const uint64_t **h, double *lo, double *w,
                   uint64_t *count)
{
    if (which == AEB_HIST_D) {
        *h = st->hist_d;
        *lo = st->lo_d;
        *w = st->w_d;
        *count = st->n_stop;
    } else if (which == AEB_HIST_V) {
        *h = st->hist_v;
        *lo = st->lo_v;
        *w = st->w_v;
        *count = st->n_contact;
    } else {
        return aeb::fail(AEB_EINVAL, "histogram selector must be AEB_HIST_D or AEB_HIST_V");
    }
    if (!std::isfinite(*lo) || !(*w > 0.0) || !std::isfinite(*w))
        return aeb::fail(AEB_EINVAL, "histogram spec of the statistics is not valid");
    uint64_t total = 0;
    for (int j = 0; j < AEB_NBINS; ++j) total += (*h)[j];
    if (total != *count)
        return aeb::fail(AEB_EINVAL, "histogram does not hold the samples its count says");
    return AEB_OK;
}

template <class S>
void merge_common(S &a, const S &b)
{
    a.n += b.n;
    a.n_stop += b.n_stop;
    a.n_contact += b.n_contact;
    a.n_horizon += b.n_horizon;
    a.n_invalid += b.n_invalid;
    a.steps += b.steps;
    a.sum_d += b.sum_d;
    a.sumsq_d += b.sumsq_d;
    a.sum_v += b.sum_v;
    a.sumsq_v += b.sumsq_v;
    a.min_d = std::fmin(a.min_d, b.min_d);
    a.max_d = std::fmax(a.max_d, b.max_d);
    a.min_v = std::fmin(a.min_v, b.min_v);
    a.max_v = std::fmax(a.max_v, b.max_v);
}

}  // namespace

extern "C" aeb_status aeb_wilson(uint64_t k, uint64_t n, double z, double *lo, double *hi)
{
    aeb::clear_error();
    if (!lo || !hi || k > n || !(z > 0.0)) return aeb::fail(AEB_EINVAL, "aeb_wilson: bad argument");
    if (n == 0) {
        *lo = 0.0;
        *hi = 1.0;
        return AEB_OK;
    }
    const double nn = (double)n, p = (double)k / nn, z2 = z * z;
    const double den = 1.0 + z2 / nn;
    const double centre = (p + z2 / (2.0 * nn)) / den;
    const double half = z * std::sqrt(p * (1.0 - p) / nn + z2 / (4.0 * nn * nn)) / den;
    *lo = centre - half;
    *hi = centre + half;
    return AEB_OK;
}

extern "C" aeb_status aeb_stats_summary(const aeb_stats *st, aeb_summary *out)
{
    aeb::clear_error();
    if (!st || !out) return aeb::fail(AEB_EINVAL, "aeb_stats_summary: NULL argument");
    return summarize(*st, out);
}

extern "C" aeb_status aeb_job_stats_summary(const aeb_job_stats *st, aeb_summary *out)
{
    aeb::clear_error();
    if (!st || !out) return aeb::fail(AEB_EINVAL, "aeb_job_stats_summary: NULL argument");
    return summarize(*st, out);
}

extern "C" aeb_status aeb_hist_quantile(const aeb_stats *st, int32_t which, double q, double *lo,
                                        double *hi)
{
    aeb::clear_error();
    if (!st || !lo || !hi) return aeb::fail(AEB_EINVAL, "aeb_hist_quantile: NULL argument");
    if (!(q >= 0.0 && q <= 1.0)) return aeb::fail(AEB_EINVAL, "aeb_hist_quantile: q must be in [0, 1]");
    const uint64_t *h = nullptr;
    double o = 0.0, w = 0.0;
    uint64_t count = 0;
    aeb_status s = hist_of(st, which, &h, &o, &w, &count);
    if (s != AEB_OK) return s;
    if (count == 0) return aeb::fail(AEB_EINVAL, "aeb_hist_quantile: the histogram is empty");
    // rank of the order statistic: k = ceil(q N), clamped to [1, N]
    const double kq = std::ceil(q * (double)count);
    uint64_t k = kq < 1.0 ? 1 : (uint64_t)kq;
    if (k > count) k = count;
    uint64_t cum = 0;
    int j = 0;
    for (; j < AEB_NBINS; ++j) {
        cum += h[j];
        if (cum >= k) break;
    }
    // the end bins also hold the values clamped into them
    *lo = (j == 0) ? -kInf : o + (double)j * w;
    *hi = (j == AEB_NBINS - 1) ? kInf : o + (double)(j + 1) * w;
    return AEB_OK;
}

extern "C" aeb_status aeb_hist_exceedance(const aeb_stats *st, int32_t which, double x,
                                          aeb_prob *out)
{
    aeb::clear_error();
    if (!st || !out) return aeb::fail(AEB_EINVAL, "aeb_hist_exceedance: NULL argument");
    const uint64_t *h = nullptr;
    double o = 0.0, w = 0.0;
    uint64_t count = 0;
    aeb_status s = hist_of(st, which, &h, &o, &w, &count);
    if (s != AEB_OK) return s;
    if (!std::isfinite(x)) return aeb::fail(AEB_EINVAL, "aeb_hist_exceedance: threshold not finite");
    const double jd = (x - o) / w;
    if (!(jd >= 1.0 && jd <= (double)(AEB_NBINS - 1)) || jd != std::floor(jd) ||
        o + jd * w != x)
        return aeb::fail(AEB_EINVAL, "aeb_hist_exceedance: threshold is not an inner bin edge "
                                     "lo + j w, 1 <= j <= AEB_NBINS - 1");
    uint64_t k = 0;
    for (int j = (int)jd; j < AEB_NBINS; ++j) k += h[j];
    const uint64_t valid = st->n_stop + st->n_contact + st->n_horizon;
    aeb_prob r;
    r.k = k;
    r.n = valid;
    r.p = valid ? (double)k / (double)valid : kNaN;
    aeb_wilson(k, valid, kZ95, &r.ci_lo, &r.ci_hi);
    *out = r;
    return AEB_OK;
}

extern "C" aeb_status aeb_is_estimate(const aeb_wstats *ws, aeb_is_result *out)
{
    aeb::clear_error();
    if (!ws || !out) return aeb::fail(AEB_EINVAL, "aeb_is_estimate: NULL argument");
    if (ws->n_valid > ws->n || ws->n_event > ws->n_valid)
        return aeb::fail(AEB_EINVAL, "aeb_is_estimate: counts are inconsistent");
    aeb_is_result r;
    r.n = ws->n;
    r.n_event = ws->n_event;
    if (ws->n == 0) {
        r.p = r.se = r.ci_lo = r.ci_hi = kNaN;
        *out = r;
        return AEB_OK;
    }
    const double n = (double)ws->n;
    // P = sum(w 1[E]) / n; standard error sqrt(var / n) with the unbiased
    // sample variance var = (sum((w 1[E])^2) - (n P) P) / (n - 1)
    const double p = ws->sum_we / n;
    r.p = p;
    if (ws->n < 2) {
        r.se = r.ci_lo = r.ci_hi = kNaN;
    } else {
        const double var = (ws->sumsq_we - (n * p) * p) / (n - 1.0);
        r.se = std::sqrt((var > 0.0 ? var : 0.0) / n);
        r.ci_lo = p - kZ95 * r.se;
        r.ci_hi = p + kZ95 * r.se;
    }
    *out = r;
    return AEB_OK;
}

extern "C" aeb_status aeb_stats_merge(aeb_stats *acc, const aeb_stats *part)
{
    aeb::clear_error();
    if (!acc || !part) return aeb::fail(AEB_EINVAL, "aeb_stats_merge: NULL argument");
    if (acc->lo_d != part->lo_d || acc->w_d != part->w_d || acc->lo_v != part->lo_v ||
        acc->w_v != part->w_v)
        return aeb::fail(AEB_EINVAL, "aeb_stats_merge: histogram specs differ");
    merge_common(*acc, *part);
    for (int j = 0; j < AEB_NBINS; ++j) {
        acc->hist_d[j] += part->hist_d[j];
        acc->hist_v[j] += part->hist_v[j];
    }
    return AEB_OK;
}

extern "C" aeb_status aeb_job_stats_merge(aeb_job_stats *acc, const aeb_job_stats *part)
{
    aeb::clear_error();
    if (!acc || !part) return aeb::fail(AEB_EINVAL, "aeb_job_stats_merge: NULL argument");
    merge_common(*acc, *part);
    return AEB_OK;
}
