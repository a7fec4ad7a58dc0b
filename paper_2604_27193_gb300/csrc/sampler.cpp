// sampler.cpp -- deterministic host sampling of parameter sets (Sec. IV-A,
// IV-C: random numbers are drawn on the CPU from a fixed seed and the
// parameter vectors are then transferred to the GPU).
//
// Counter-based: sample i, quantity q draws from Philox-4x64-10 (Salmon et al.,
// SC'11) at counter (i, q / 2, 0, 0) under key (seed, scenario_id), words 0-1
// for even q and 2-3 for odd q.  Any sample range can therefore be produced by
// any thread, in any order, with the same result; threads split [0, n) into
// contiguous blocks.  Built with -ffp-contract=off so the binary64 transforms
// round the same on every host.
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "aeb_internal.h"
#include "host_util.h"

namespace aeb {
namespace {

inline void mul_hi_lo(uint64_t a, uint64_t b, uint64_t &hi, uint64_t &lo)
{
    const unsigned __int128 p = (unsigned __int128)a * b;
    hi = (uint64_t)(p >> 64);
    lo = (uint64_t)p;
}

// Philox-4x64 with 10 rounds: multipliers 0xD2E7470EE14C6C93, 0xCA5A826395121157,
// Weyl key increments 0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B.
inline void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1)
{
    for (int r = 0; r < 10; ++r) {
        uint64_t h0, l0, h1, l1;
        mul_hi_lo(0xD2E7470EE14C6C93ull, c[0], h0, l0);
        mul_hi_lo(0xCA5A826395121157ull, c[2], h1, l1);
        const uint64_t n0 = h1 ^ c[1] ^ k0, n2 = h0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = l1;
        c[2] = n2;
        c[3] = l0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
}

constexpr double kTwoM53 = 1.0 / 9007199254740992.0;

inline double transform(const aeb_dist &d, uint64_t w0, uint64_t w1)
{
    double x;
    switch (d.kind) {
    case AEB_DIST_UNIFORM:
        x = d.p0 + (d.p1 - d.p0) * ((double)(w0 >> 11) * kTwoM53);
        break;
    case AEB_DIST_NORMAL: {
        const double u1 = (double)((w0 >> 11) + 1) * kTwoM53;  // (0, 1]
        const double u2 = (double)(w1 >> 11) * kTwoM53;        // [0, 1)
        x = d.p0 + d.p1 * (std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        break;
    }
    default:
        x = d.p0;
    }
    if (x < d.lo) x = d.lo;
    if (x > d.hi) x = d.hi;
    return x;
}

// Importance sampling: probability that an unclamped draw of d lies at or
// below x, or above x.
double mass_below(const aeb_dist &d, double x)
{
    if (d.kind == AEB_DIST_UNIFORM) {
        const double u = (x - d.p0) / (d.p1 - d.p0);
        return u <= 0.0 ? 0.0 : (u >= 1.0 ? 1.0 : u);
    }
    return 0.5 * std::erfc((d.p0 - x) / (d.p1 * std::sqrt(2.0)));
}

double mass_above(const aeb_dist &d, double x)
{
    if (d.kind == AEB_DIST_UNIFORM) return 1.0 - mass_below(d, x);
    return 0.5 * std::erfc((x - d.p0) / (d.p1 * std::sqrt(2.0)));
}

// Likelihood ratio p(x) / q(x) of one quantity drawn from q with clamped
// value x: a clamp bound holding mass under q compares the masses there,
// elsewhere the densities compare.
double likelihood_ratio(const aeb_dist &p, const aeb_dist &q, double x)
{
    if (q.kind == AEB_DIST_CONST) return 1.0;
    if (x <= q.lo) {
        const double mq = mass_below(q, q.lo);
        if (mq > 0.0) return mass_below(p, p.lo) / mq;
    }
    if (x >= q.hi) {
        const double mq = mass_above(q, q.hi);
        if (mq > 0.0) return mass_above(p, p.hi) / mq;
    }
    if (q.kind == AEB_DIST_UNIFORM)
        return (x >= p.p0 && x < p.p1) ? (q.p1 - q.p0) / (p.p1 - p.p0) : 0.0;
    const double zp = (x - p.p0) / p.p1, zq = (x - q.p0) / q.p1;
    return (q.p1 / p.p1) * std::exp(0.5 * (zq * zq - zp * zp));
}

bool is_compatible(const aeb_dist &p, const aeb_dist &q)
{
    if (p.kind != q.kind || p.lo != q.lo || p.hi != q.hi) return false;
    switch (q.kind) {
    case AEB_DIST_CONST: return p.p0 == q.p0;
    case AEB_DIST_UNIFORM: return q.p0 <= p.p0 && p.p1 <= q.p1 && p.p1 > p.p0;
    default: return p.p1 > 0.0 && q.p1 > 0.0;
    }
}

// Samples [lo, hi) of the call; with `nominal`, also their likelihood ratios.
void sample_block(double g, const aeb_scenario &sc, uint64_t first, uint64_t lo, uint64_t hi,
                  const aeb_params &out, const aeb_scenario *nominal, double *weights)
{
    const aeb_dist *dist[9] = {&sc.v0, &sc.d0, &sc.mu, &sc.grade, &sc.mass,
                               &sc.cd, &sc.tau, &sc.t_delay, &sc.noise};
    const aeb_dist *ndist[9] = {};
    if (nominal) {
        const aeb_dist *nd[9] = {&nominal->v0, &nominal->d0, &nominal->mu, &nominal->grade,
                                 &nominal->mass, &nominal->cd, &nominal->tau,
                                 &nominal->t_delay, &nominal->noise};
        for (int q = 0; q < 9; ++q) ndist[q] = nd[q];
    }
    for (uint64_t j = lo; j < hi; ++j) {
        double q[10];
        for (uint64_t b = 0; b < 5; ++b) {
            uint64_t c[4] = {first + j, b, 0, 0};
            philox4x64_10(c, sc.seed, sc.scenario_id);
            q[2 * b] = transform(*dist[2 * b], c[0], c[1]);
            if (2 * b + 1 < 9) q[2 * b + 1] = transform(*dist[2 * b + 1], c[2], c[3]);
        }
        out.v0[j] = q[0];
        out.d0[j] = q[1];
        out.mu[j] = q[2];
        out.gs[j] = g * std::sin(q[3]);
        out.gc[j] = g * std::cos(q[3]);
        out.mass[j] = q[4];
        out.cd[j] = q[5];
        out.tau[j] = q[6];
        out.t_delay[j] = q[7];
        out.noise[j] = q[8];
        if (nominal) {
            double w = 1.0;
            for (int k = 0; k < 9; ++k) w *= likelihood_ratio(*ndist[k], *dist[k], q[k]);
            weights[j] = w;
        }
    }
}

bool dist_ok(const aeb_dist &d)
{
    if (d.reserved != 0) return false;
    if (d.kind != AEB_DIST_CONST && d.kind != AEB_DIST_UNIFORM && d.kind != AEB_DIST_NORMAL)
        return false;
    if (!std::isfinite(d.p0) || !std::isfinite(d.p1)) return false;
    if (std::isnan(d.lo) || std::isnan(d.hi) || d.lo > d.hi) return false;
    return true;
}

}  // namespace
}  // namespace aeb

namespace aeb {
namespace {

aeb_status sample_impl(const char *who, const aeb_model *model, const aeb_scenario *scenario,
                       const aeb_scenario *nominal, uint64_t first, uint64_t n,
                       const aeb_params *out, double *weights, int32_t n_threads)
{
    const std::string w = who;
    if (!model || !scenario || !out) return fail(AEB_EINVAL, w + ": NULL argument");
    if (!std::isfinite(model->g)) return fail(AEB_EINVAL, w + ": g is not finite");
    const aeb_dist *dist[9] = {&scenario->v0, &scenario->d0, &scenario->mu, &scenario->grade,
                               &scenario->mass, &scenario->cd, &scenario->tau,
                               &scenario->t_delay, &scenario->noise};
    for (int q = 0; q < 9; ++q)
        if (!dist_ok(*dist[q]))
            return fail(AEB_EINVAL, w + ": invalid distribution for quantity " + std::to_string(q));
    if (nominal) {
        if (!weights) return fail(AEB_EINVAL, w + ": NULL weights");
        const aeb_dist *nd[9] = {&nominal->v0, &nominal->d0, &nominal->mu, &nominal->grade,
                                 &nominal->mass, &nominal->cd, &nominal->tau,
                                 &nominal->t_delay, &nominal->noise};
        for (int q = 0; q < 9; ++q)
            if (!dist_ok(*nd[q]) || !is_compatible(*nd[q], *dist[q]))
                return fail(AEB_EINVAL, w + ": proposal incompatible with the nominal scenario "
                                            "for quantity " + std::to_string(q));
    }
    if (n == 0) return AEB_OK;
    const double *cols[AEB_NFIELDS] = {out->v0, out->d0, out->mu, out->gs, out->gc,
                                       out->mass, out->cd, out->tau, out->t_delay, out->noise};
    for (int j = 0; j < AEB_NFIELDS; ++j)
        if (!cols[j]) return fail(AEB_EINVAL, w + ": NULL output column");

    unsigned hw = std::thread::hardware_concurrency();
    uint64_t t = n_threads > 0 ? (uint64_t)n_threads : (hw ? hw : 1);
    const uint64_t min_per_thread = 2048;
    if (t > (n + min_per_thread - 1) / min_per_thread) t = (n + min_per_thread - 1) / min_per_thread;
    if (t < 1) t = 1;
    const aeb_scenario sc = *scenario;
    const aeb_params o = *out;
    if (t == 1) {
        sample_block(model->g, sc, first, 0, n, o, nominal, weights);
        return AEB_OK;
    }
    std::vector<std::thread> pool;
    pool.reserve(t);
    try {
        for (uint64_t k = 0; k < t; ++k) {
            const uint64_t lo = n * k / t, hi = n * (k + 1) / t;
            pool.emplace_back(sample_block, model->g, std::cref(sc), first, lo, hi, std::cref(o),
                              nominal, weights);
        }
    } catch (...) {
        for (auto &th : pool) th.join();
        return fail(AEB_ENOMEM, w + ": could not start sampling threads");
    }
    for (auto &th : pool) th.join();
    return AEB_OK;
}

}  // namespace
}  // namespace aeb

extern "C" aeb_status aeb_sample_params(const aeb_model *model, const aeb_scenario *scenario,
                                        uint64_t first, uint64_t n, const aeb_params *out,
                                        int32_t n_threads)
{
    aeb::clear_error();
    return aeb::sample_impl("aeb_sample_params", model, scenario, nullptr, first, n, out,
                            nullptr, n_threads);
}

extern "C" aeb_status aeb_sample_params_is(const aeb_model *model, const aeb_scenario *nominal,
                                           const aeb_scenario *proposal, uint64_t first,
                                           uint64_t n, const aeb_params *out, double *weights,
                                           int32_t n_threads)
{
    aeb::clear_error();
    if (!nominal) return aeb::fail(AEB_EINVAL, "aeb_sample_params_is: NULL nominal scenario");
    return aeb::sample_impl("aeb_sample_params_is", model, proposal, nominal, first, n, out,
                            weights, n_threads);
}
