// capi.cpp -- the C ABI entry points other than sampling: argument checks,
// conversion of the model to the kernels' form, library scratch, dispatch.
#include <algorithm>
#include <cmath>
#include <initializer_list>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "aeb_internal.h"
#include "host_util.h"

namespace aeb {

namespace {
thread_local std::string t_error;
}

void clear_error() { t_error.clear(); }

aeb_status fail(aeb_status code, const std::string &msg)
{
    t_error = msg;
    return code;
}

aeb_status cuda_fail(cudaError_t e, const char *what)
{
    const aeb_status code = (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ||
                             e == cudaErrorNoKernelImageForDevice ||
                             e == cudaErrorInvalidDevice)
                                ? AEB_EDEVICE
                                : (e == cudaErrorMemoryAllocation ? AEB_ENOMEM : AEB_ECUDA);
    return fail(code, std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                          cudaGetErrorString(e) + ")");
}

namespace {

bool is_pow2(double w)
{
    if (!(w > 0.0) || !std::isfinite(w)) return false;
    int ex = 0;
    return std::frexp(w, &ex) == 0.5;
}

}  // namespace

aeb_status check_model(const aeb_model *m, ModelDev *out)
{
    if (!m) return fail(AEB_EINVAL, "model is NULL");
    const double v[] = {m->g, m->rho, m->area, m->h_cg, m->wheelbase, m->beta,
                        m->phi_f, m->a_cmd, m->dt, m->t_max, m->ttc_thr,
                        m->lead_v0, m->lead_decel, m->perc_sigma, m->perc_drop,
                        m->perc_latency};
    for (double x : v)
        if (!std::isfinite(x)) return fail(AEB_EINVAL, "model constant is not finite");
    if (!(m->dt > 0.0)) return fail(AEB_EINVAL, "model.dt must be > 0");
    if (m->t_max < 0.0) return fail(AEB_EINVAL, "model.t_max must be >= 0");
    if (!(m->wheelbase > 0.0)) return fail(AEB_EINVAL, "model.wheelbase must be > 0");
    if (m->cap_mode != AEB_CAP_LUMPED && m->cap_mode != AEB_CAP_PER_AXLE)
        return fail(AEB_EINVAL, "model.cap_mode unknown");
    if (m->trigger != AEB_TRIGGER_IMMEDIATE && m->trigger != AEB_TRIGGER_TTC)
        return fail(AEB_EINVAL, "model.trigger unknown");
    if (m->lead != 0 && m->lead != 1) return fail(AEB_EINVAL, "model.lead must be 0 or 1");
    if (m->reserved != 0) return fail(AEB_EINVAL, "model.reserved must be 0");
    if (m->lead_v0 < 0.0 || m->lead_decel < 0.0)
        return fail(AEB_EINVAL, "model.lead_v0 and model.lead_decel must be >= 0");
    if (m->perc_sigma < 0.0 || m->perc_latency < 0.0 || m->perc_drop < 0.0 || m->perc_drop > 1.0)
        return fail(AEB_EINVAL, "model.perc_sigma, perc_latency >= 0 and perc_drop in [0, 1]");
    const int64_t perc_lat = steps_to_reach_host(m->perc_latency, m->dt);
    if (perc_lat > 1000000000) return fail(AEB_EINVAL, "model.perc_latency / model.dt too large");
    const int64_t n_max = steps_to_reach_host(m->t_max, m->dt);
    if (n_max > 2147483646) return fail(AEB_EINVAL, "model.t_max / model.dt exceeds 2^31 - 2 steps");
    out->g = m->g;
    out->rho = m->rho;
    out->area = m->area;
    out->hl = m->h_cg / m->wheelbase;
    out->beta = m->beta;
    out->phi_f = m->phi_f;
    out->a_cmd = m->a_cmd;
    out->dt = m->dt;
    out->h2 = 0.5 * m->dt;
    out->h6 = m->dt / 6.0;
    out->ttc_thr = m->ttc_thr;
    out->n_max = (int32_t)n_max;
    out->cap_mode = m->cap_mode;
    out->trigger = m->trigger;
    out->lead = m->lead;
    out->lead_v0 = m->lead_v0;
    out->lead_decel = m->lead_decel;
    out->lead_ts = (m->lead_decel > 0.0) ? m->lead_v0 / m->lead_decel
                                         : std::numeric_limits<double>::infinity();
    out->lead_xs = 0.5 * (m->lead_v0 * out->lead_ts);
    out->lead_moving = (m->lead == 1 && m->lead_v0 > 0.0) ? 1 : 0;
    out->perc_sigma = m->perc_sigma;
    out->perc_drop = m->perc_drop;
    out->perc_seed = m->perc_seed;
    out->perc = (m->perc_sigma > 0.0 || m->perc_drop > 0.0 || m->perc_latency > 0.0) ? 1 : 0;
    out->perc_lat = out->perc ? (int32_t)perc_lat : 0;
    return AEB_OK;
}

aeb_status check_params(const aeb_params *p, ParamsDev *out)
{
    if (!p) return fail(AEB_EINVAL, "params is NULL");
    const double *c[AEB_NFIELDS] = {p->v0, p->d0, p->mu, p->gs, p->gc,
                                    p->mass, p->cd, p->tau, p->t_delay, p->noise};
    for (int j = 0; j < AEB_NFIELDS; ++j) {
        if (!c[j]) return fail(AEB_EINVAL, "params column is NULL");
        if (reinterpret_cast<uintptr_t>(c[j]) % 8 != 0)
            return fail(AEB_EINVAL, "params column is not 8-byte aligned");
        out->col[j] = c[j];
    }
    return AEB_OK;
}

aeb_status check_hist(const aeb_hist_spec *h)
{
    if (!h) return fail(AEB_EINVAL, "hist spec is NULL");
    if (!std::isfinite(h->lo_d) || !std::isfinite(h->lo_v))
        return fail(AEB_EINVAL, "hist origin is not finite");
    if (!is_pow2(h->w_d) || !is_pow2(h->w_v))
        return fail(AEB_EINVAL, "hist width must be a positive power of two");
    return AEB_OK;
}

OutDev out_dev(const aeb_outputs *o)
{
    OutDev d{};
    if (o) {
        d.status = o->status;
        d.x_raw = o->x_raw;
        d.x_ref = o->x_ref;
        d.v_imp = o->v_imp;
        d.t_end = o->t_end;
        d.n_steps = o->n_steps;
        d.n_onset = o->n_onset;
    }
    return d;
}

// The output columns from row `off` on (NULL columns stay NULL).
OutDev offset_out(const OutDev &o, uint64_t off)
{
    OutDev d = o;
    if (d.status) d.status += off;
    if (d.x_raw) d.x_raw += off;
    if (d.x_ref) d.x_ref += off;
    if (d.v_imp) d.v_imp += off;
    if (d.t_end) d.t_end += off;
    if (d.n_steps) d.n_steps += off;
    if (d.n_onset) d.n_onset += off;
    return d;
}

namespace {

// Library scratch, one region per (device, stream): work on one stream is
// ordered, so consecutive calls on a stream may reuse its region, while calls
// on different streams never share one.
struct Region {
    void *base = nullptr;
    size_t bytes = 0;
};
std::mutex g_mu;
std::map<std::pair<int, uintptr_t>, Region> g_scratch;

constexpr size_t kCounterBytes = 256;
size_t partial_bytes() { return sizeof(RedPartial) * 1024; }

aeb_status scratch_for(cudaStream_t s, size_t bytes, void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_mu);
    Region &r = g_scratch[{dev, reinterpret_cast<uintptr_t>(s)}];
    if (r.bytes < bytes) {
        if (r.base) {
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
            cudaFree(r.base);
            r.base = nullptr;
            r.bytes = 0;
        }
        e = cudaMalloc(&r.base, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(scratch)");
        r.bytes = bytes;
    }
    *out = r.base;
    return AEB_OK;
}

std::mutex g_cfg_mu;
LaunchCfg g_cfg[2] = {{128, 0, 256}, {128, 0, 32}};

aeb_status rollout_impl(const ModelDev &md, const ParamsDev &pd, uint64_t n,
                        aeb_precision precision, const OutDev &od, cudaStream_t s,
                        uint64_t key_base)
{
    void *scratch = nullptr;
    aeb_status st = scratch_for(s, kCounterBytes + partial_bytes(), &scratch);
    if (st != AEB_OK) return st;
    auto *counter = static_cast<unsigned long long *>(scratch);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counter)");
    const LaunchCfg cfg = launch_cfg(precision);
    WorkDev w{n, (uint32_t)cfg.tile, counter, nullptr, 0, nullptr, key_base};
    e = (precision == AEB_FP64_PLAIN) ? launch_rollout_fp64(md, pd, od, w, cfg, s)
                                      : launch_rollout_fp32(md, pd, od, w, cfg, s);
    if (e != cudaSuccess) return cuda_fail(e, "rollout launch");
    return AEB_OK;
}

aeb_status reduce_impl(const aeb_outputs *out, uint64_t n, const aeb_hist_spec &h,
                       aeb_stats *stats, cudaStream_t s)
{
    void *scratch = nullptr;
    aeb_status st = scratch_for(s, kCounterBytes + partial_bytes(), &scratch);
    if (st != AEB_OK) return st;
    auto *partials = reinterpret_cast<RedPartial *>(static_cast<char *>(scratch) + kCounterBytes);
    cudaError_t e = launch_reduce(out->status, out->x_ref, out->v_imp, out->n_steps, n, h,
                                  partials, stats, s);
    if (e != cudaSuccess) return cuda_fail(e, "reduce launch");
    return AEB_OK;
}

// Device buffers, streams and events of aeb_evaluate, one set per (device,
// stream).  The parameter upload is cut into chunks: chunk k is copied on
// `copy` while chunk k - 1 rolls out on comp[(k - 1) % 2], so the copies hide
// behind the arithmetic, and two compute streams let a chunk's launch start
// while the previous one drains its last rollouts.  The first chunk is small,
// so the arithmetic starts after a short upload; each later one is kEvalGrow
// times the one before.  A chunk's copy must end before the previous chunk's
// rollouts do: an upload moves 80 B per sample (~1.3 ns per sample at the
// pinned-host copy rate measured on GB300) against ~2.7 ns per sample of
// FP32 rollout, so a chunk may be at most about twice the one before (six
// times left the GPU waiting for the last chunk's copy).  The host-to-device
// copy rate differs between machines (60-200 GB/s measured on GB300 machines), so
// each call times its own uploads and its first chunk's rollouts (the first
// chunk runs alone) and sets the growth of the next call on that stream to
// 0.8 x (rollout time per sample) / (upload time per sample), within
// [kEvalGrowMin, kEvalGrowMax]; the first call grows by 2.  Results do not
// depend on the chunks.
constexpr int kEvalMaxChunks = 12;
constexpr uint64_t kEvalFirstChunk = uint64_t(1) << 18;
constexpr double kEvalGrowFirst = 2.0, kEvalGrowMin = 1.25, kEvalGrowMax = 4.0;
// aeb_evaluate_scenario draws chunks of kSampledChunk samples on the host into
// two pinned staging buffers (pin[k % 2]); the upload of chunk k records
// uploaded[k % 2], after which the host may draw chunk k + 2 into that buffer.
constexpr uint64_t kSampledChunk = uint64_t(1) << 20;
struct EvalBuffers {
    void *base = nullptr;
    uint64_t cap = 0;  // samples
    cudaStream_t copy = nullptr, comp[2] = {nullptr, nullptr};
    cudaEvent_t start = nullptr, copied[kEvalMaxChunks] = {}, done[2] = {nullptr, nullptr};
    double *pin[2] = {nullptr, nullptr};  // AEB_NFIELDS columns of kSampledChunk each
    cudaEvent_t uploaded[2] = {nullptr, nullptr};
    // timing of the last aeb_evaluate on this stream: every upload (up0 .. up1)
    // and the first chunk's rollouts (run0 .. run1); the next call's growth
    cudaEvent_t up0 = nullptr, up1 = nullptr, run0 = nullptr, run1 = nullptr;
    double grow = kEvalGrowFirst;
};

cudaError_t eval_streams(EvalBuffers &b)
{
    if (b.copy) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&b.copy, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaStreamCreateWithFlags(&b.comp[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.start, cudaEventDisableTiming);
    for (int i = 0; i < kEvalMaxChunks && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&b.copied[i], cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&b.done[i], cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&b.uploaded[i], cudaEventDisableTiming);
    for (cudaEvent_t *t : {&b.up0, &b.up1, &b.run0, &b.run1})
        if (e == cudaSuccess) e = cudaEventCreate(t);
    return e;
}
std::map<std::pair<int, uintptr_t>, EvalBuffers> g_eval;

constexpr size_t kEvalBytesPerSample = 8 * AEB_NFIELDS + 1 + 8 * 4 + 4 * 2;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// The evaluate buffers of (current device, s), grown to at least cap samples.
aeb_status eval_acquire(cudaStream_t s, uint64_t cap, EvalBuffers **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_mu);
    EvalBuffers &b = g_eval[{dev, reinterpret_cast<uintptr_t>(s)}];
    e = eval_streams(b);
    if (e != cudaSuccess) return cuda_fail(e, "evaluate: streams");
    if (b.cap < cap) {
        if (b.base) {
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
            cudaFree(b.base);
            b.base = nullptr;
            b.cap = 0;
        }
        const size_t bytes = align256(sizeof(aeb_stats)) + cap * kEvalBytesPerSample + 16 * 256;
        e = cudaMalloc(&b.base, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(evaluate buffers)");
        b.cap = cap;
    }
    *out = &b;
    return AEB_OK;
}

// The device stats, parameter columns and outputs of n <= b.cap samples in
// the buffers of b.
struct EvalLayout {
    aeb_stats *stats;
    aeb_params params;
    aeb_outputs out;
};
EvalLayout eval_layout(const EvalBuffers &b)
{
    const uint64_t cap = b.cap;
    char *p = static_cast<char *>(b.base);
    auto take = [&](size_t bytes) {
        char *r = p;
        p += align256(bytes);
        return r;
    };
    EvalLayout L;
    L.stats = reinterpret_cast<aeb_stats *>(take(sizeof(aeb_stats)));
    double **dcols[AEB_NFIELDS] = {&L.params.v0, &L.params.d0, &L.params.mu, &L.params.gs,
                                   &L.params.gc, &L.params.mass, &L.params.cd, &L.params.tau,
                                   &L.params.t_delay, &L.params.noise};
    for (int j = 0; j < AEB_NFIELDS; ++j) *dcols[j] = reinterpret_cast<double *>(take(8 * cap));
    L.out.status = reinterpret_cast<uint8_t *>(take(cap));
    L.out.x_raw = reinterpret_cast<double *>(take(8 * cap));
    L.out.x_ref = reinterpret_cast<double *>(take(8 * cap));
    L.out.v_imp = reinterpret_cast<double *>(take(8 * cap));
    L.out.t_end = reinterpret_cast<double *>(take(8 * cap));
    L.out.n_steps = reinterpret_cast<int32_t *>(take(4 * cap));
    L.out.n_onset = reinterpret_cast<int32_t *>(take(4 * cap));
    return L;
}

}  // namespace

LaunchCfg launch_cfg(aeb_precision precision)
{
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    return g_cfg[precision == AEB_FP64_PLAIN ? 0 : 1];
}

void set_launch_cfg(aeb_precision precision, const LaunchCfg &cfg)
{
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    g_cfg[precision == AEB_FP64_PLAIN ? 0 : 1] = cfg;
}

int64_t steps_to_reach_host(double t, double dt)
{
    if (!(t > 0.0)) return 0;
    const double q = std::ceil(t / dt);
    if (!(q <= 2147483647.0)) return 2147483647;
    int64_t n = (int64_t)q;
    while (n > 0 && (double)(n - 1) * dt >= t) --n;
    while ((double)n * dt < t) ++n;
    return n;
}

}  // namespace aeb

using namespace aeb;

extern "C" int32_t aeb_abi_version(void) { return AEB_ABI_VERSION; }

extern "C" const char *aeb_last_error(void) { return t_error.c_str(); }

extern "C" aeb_status aeb_rollout(const aeb_model *model, const aeb_params *params, uint64_t n,
                                  aeb_precision precision, const aeb_outputs *out, void *stream)
{
    clear_error();
    ModelDev md;
    ParamsDev pd;
    aeb_status st = check_model(model, &md);
    if (st != AEB_OK) return st;
    st = check_params(params, &pd);
    if (st != AEB_OK) return st;
    if (precision != AEB_FP64_PLAIN && precision != AEB_FP32_COMP)
        return fail(AEB_EINVAL, "unknown precision");
    if (n == 0) return AEB_OK;
    return rollout_impl(md, pd, n, precision, out_dev(out), static_cast<cudaStream_t>(stream), 0);
}

extern "C" aeb_status aeb_reduce(const aeb_outputs *out, uint64_t n, const aeb_hist_spec *hist,
                                 aeb_stats *stats, void *stream)
{
    clear_error();
    if (!out || !stats) return fail(AEB_EINVAL, "aeb_reduce: NULL argument");
    if (n > 0 && (!out->status || !out->x_ref || !out->v_imp || !out->n_steps))
        return fail(AEB_EINVAL, "aeb_reduce: status, x_ref, v_imp and n_steps are required");
    if (reinterpret_cast<uintptr_t>(stats) % 8 != 0)
        return fail(AEB_EINVAL, "aeb_reduce: stats is not 8-byte aligned");
    aeb_status st = check_hist(hist);
    if (st != AEB_OK) return st;
    return reduce_impl(out, n, *hist, stats, static_cast<cudaStream_t>(stream));
}

extern "C" aeb_status aeb_reduce_weighted(const aeb_outputs *out, const double *weights,
                                          uint64_t n, double x_thr, aeb_wstats *stats,
                                          void *stream)
{
    clear_error();
    if (!out || !stats || (n > 0 && (!weights || !out->status || !out->x_ref)))
        return fail(AEB_EINVAL, "aeb_reduce_weighted: NULL argument (status, x_ref, weights "
                                "and stats are required)");
    if (reinterpret_cast<uintptr_t>(stats) % 8 != 0 ||
        reinterpret_cast<uintptr_t>(weights) % 8 != 0)
        return fail(AEB_EINVAL, "aeb_reduce_weighted: stats or weights not 8-byte aligned");
    if (std::isnan(x_thr)) return fail(AEB_EINVAL, "aeb_reduce_weighted: x_thr is NaN");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *scratch = nullptr;
    aeb_status st = scratch_for(s, kCounterBytes + partial_bytes(), &scratch);
    if (st != AEB_OK) return st;
    static_assert(sizeof(RedPartial) * 1024 >= 48 * 1024, "scratch too small for weighted partials");
    cudaError_t e = launch_reduce_weighted(out->status, out->x_ref, weights, n, x_thr,
                                           static_cast<char *>(scratch) + kCounterBytes, stats, s);
    if (e != cudaSuccess) return cuda_fail(e, "aeb_reduce_weighted launch");
    return AEB_OK;
}

extern "C" aeb_status aeb_evaluate(const aeb_model *model, const aeb_params *params, uint64_t n,
                                   aeb_precision precision, const aeb_hist_spec *hist,
                                   aeb_stats *host_stats, const aeb_outputs *host_out,
                                   void *stream)
{
    clear_error();
    ModelDev md;
    ParamsDev hp;
    aeb_status st = check_model(model, &md);
    if (st != AEB_OK) return st;
    st = check_params(params, &hp);
    if (st != AEB_OK) return st;
    if (precision != AEB_FP64_PLAIN && precision != AEB_FP32_COMP)
        return fail(AEB_EINVAL, "unknown precision");
    st = check_hist(hist);
    if (st != AEB_OK) return st;
    if (!host_stats) return fail(AEB_EINVAL, "aeb_evaluate: host_stats is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    EvalBuffers *eb = nullptr;
    st = eval_acquire(s, n > 0 ? n : 1, &eb);
    if (st != AEB_OK) return st;
    const EvalLayout lay = eval_layout(*eb);
    aeb_stats *dstats = lay.stats;
    const aeb_params dp = lay.params;
    const aeb_outputs dout = lay.out;
    cudaError_t e = cudaSuccess;

    ParamsDev pd;
    check_params(&dp, &pd);
    uint64_t timed_first = 0;  // samples of the timed first chunk (0: not timed)
    if (n > 0) {
        aeb_outputs want = dout;
        if (!host_out || !host_out->x_raw) want.x_raw = nullptr;
        if (!host_out || !host_out->t_end) want.t_end = nullptr;
        if (!host_out || !host_out->n_onset) want.n_onset = nullptr;
        const OutDev od = out_dev(&want);
        // chunk boundaries: lengths kEvalFirstChunk, kEvalGrow times that, ...;
        // the chunk whose length reaches the rest takes the rest (one chunk up
        // to 2 kEvalFirstChunk samples)
        uint64_t bound[kEvalMaxChunks + 1] = {0};
        int chunks = 0;
        for (double lenf = (double)kEvalFirstChunk; bound[chunks] < n; lenf *= eb->grow) {
            const uint64_t len = (uint64_t)lenf, rest = n - bound[chunks];
            const bool last = chunks == kEvalMaxChunks - 1 || rest <= len ||
                              (chunks == 0 && rest <= 2 * kEvalFirstChunk);
            bound[chunks + 1] = bound[chunks] + (last ? rest : len);
            ++chunks;
        }
        // the copies start after the work already queued on the caller's stream
        e = cudaEventRecord(eb->start, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(eb->copy, eb->start, 0);
        if (e == cudaSuccess) e = cudaEventRecord(eb->up0, eb->copy);
        if (e != cudaSuccess) return cuda_fail(e, "aeb_evaluate: stream order");
        for (int k = 0; k < chunks; ++k) {
            const uint64_t off = bound[k], len = bound[k + 1] - bound[k];
            ParamsDev pk = pd;
            for (int j = 0; j < AEB_NFIELDS; ++j) {
                e = cudaMemcpyAsync(const_cast<double *>(pd.col[j]) + off, hp.col[j] + off, 8 * len,
                                    cudaMemcpyHostToDevice, eb->copy);
                if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(params)");
                pk.col[j] = pd.col[j] + off;
            }
            cudaStream_t cs = eb->comp[k % 2];
            e = cudaEventRecord(eb->copied[k], eb->copy);
            if (e == cudaSuccess && k == chunks - 1) e = cudaEventRecord(eb->up1, eb->copy);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, eb->copied[k], 0);
            if (e == cudaSuccess && k == 0) e = cudaEventRecord(eb->run0, cs);
            if (e != cudaSuccess) return cuda_fail(e, "aeb_evaluate: chunk order");
            st = rollout_impl(md, pk, len, precision, offset_out(od, off), cs, off);
            if (st != AEB_OK) return st;
            if (k == 0) {
                e = cudaEventRecord(eb->run1, cs);
                if (e != cudaSuccess) return cuda_fail(e, "aeb_evaluate: chunk timing");
            }
        }
        timed_first = chunks > 1 ? bound[1] : 0;
        for (int i = 0; i < 2; ++i) {
            e = cudaEventRecord(eb->done[i], eb->comp[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, eb->done[i], 0);
            if (e != cudaSuccess) return cuda_fail(e, "aeb_evaluate: join");
        }
    }
    st = reduce_impl(&dout, n, *hist, dstats, s);
    if (st != AEB_OK) return st;
    e = cudaMemcpyAsync(host_stats, dstats, sizeof(aeb_stats), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(stats)");
    if (host_out && n > 0) {
        struct {
            void *h;
            const void *d;
            size_t sz;
        } cp[] = {{host_out->status, dout.status, 1},   {host_out->x_raw, dout.x_raw, 8},
                  {host_out->x_ref, dout.x_ref, 8},     {host_out->v_imp, dout.v_imp, 8},
                  {host_out->t_end, dout.t_end, 8},     {host_out->n_steps, dout.n_steps, 4},
                  {host_out->n_onset, dout.n_onset, 4}};
        for (auto &c : cp) {
            if (!c.h) continue;
            e = cudaMemcpyAsync(c.h, c.d, c.sz * n, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(outputs)");
        }
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (timed_first > 0) {  // the next call's chunk growth (see EvalBuffers)
        float up_ms = 0.0f, run_ms = 0.0f;
        if (cudaEventElapsedTime(&up_ms, eb->up0, eb->up1) == cudaSuccess &&
            cudaEventElapsedTime(&run_ms, eb->run0, eb->run1) == cudaSuccess && up_ms > 0.0f &&
            run_ms > 0.0f) {
            const double g = 0.8 * ((double)run_ms / (double)timed_first) /
                             ((double)up_ms / (double)n);
            eb->grow = std::min(kEvalGrowMax, std::max(kEvalGrowMin, g));
        }
    }
    return AEB_OK;
}

extern "C" aeb_status aeb_evaluate_scenario(const aeb_model *model, const aeb_scenario *scenario,
                                            uint64_t first, uint64_t n, aeb_precision precision,
                                            const aeb_hist_spec *hist, int32_t n_threads,
                                            aeb_stats *host_stats, void *stream)
{
    clear_error();
    ModelDev md;
    aeb_status st = check_model(model, &md);
    if (st != AEB_OK) return st;
    if (precision != AEB_FP64_PLAIN && precision != AEB_FP32_COMP)
        return fail(AEB_EINVAL, "unknown precision");
    st = check_hist(hist);
    if (st != AEB_OK) return st;
    if (!host_stats) return fail(AEB_EINVAL, "aeb_evaluate_scenario: host_stats is NULL");
    {  // the scenario's checks (no samples drawn)
        aeb_params none;
        std::memset(&none, 0, sizeof none);
        st = aeb_sample_params(model, scenario, first, 0, &none, n_threads);
        if (st != AEB_OK) return st;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    EvalBuffers *eb = nullptr;
    st = eval_acquire(s, n > 0 ? n : 1, &eb);
    if (st != AEB_OK) return st;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2; ++i) {
        if (eb->pin[i]) continue;
        void *h = nullptr;
        e = cudaHostAlloc(&h, sizeof(double) * AEB_NFIELDS * kSampledChunk, cudaHostAllocDefault);
        if (e != cudaSuccess) return cuda_fail(e, "cudaHostAlloc(sampling staging)");
        eb->pin[i] = static_cast<double *>(h);
    }
    const EvalLayout lay = eval_layout(*eb);
    ParamsDev pd;
    check_params(&lay.params, &pd);
    if (n > 0) {
        aeb_outputs want = lay.out;
        want.x_raw = nullptr;
        want.t_end = nullptr;
        want.n_onset = nullptr;
        const OutDev od = out_dev(&want);
        // the copies start after the work already queued on the caller's stream
        e = cudaEventRecord(eb->start, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(eb->copy, eb->start, 0);
        if (e != cudaSuccess) return cuda_fail(e, "aeb_evaluate_scenario: stream order");
        const uint64_t chunks = (n + kSampledChunk - 1) / kSampledChunk;
        for (uint64_t k = 0; k < chunks; ++k) {
            const uint64_t off = k * kSampledChunk;
            const uint64_t len = n - off < kSampledChunk ? n - off : kSampledChunk;
            const int b = (int)(k % 2);
            if (k >= 2) {  // the upload of chunk k - 2 from this buffer has ended
                e = cudaEventSynchronize(eb->uploaded[b]);
                if (e != cudaSuccess) return cuda_fail(e, "aeb_evaluate_scenario: staging");
            }
            aeb_params hp;
            double **hc[AEB_NFIELDS] = {&hp.v0, &hp.d0, &hp.mu, &hp.gs, &hp.gc,
                                        &hp.mass, &hp.cd, &hp.tau, &hp.t_delay, &hp.noise};
            for (int j = 0; j < AEB_NFIELDS; ++j) *hc[j] = eb->pin[b] + (size_t)j * kSampledChunk;
            st = aeb_sample_params(model, scenario, first + off, len, &hp, n_threads);
            if (st != AEB_OK) return st;
            ParamsDev pk = pd;
            for (int j = 0; j < AEB_NFIELDS; ++j) {
                e = cudaMemcpyAsync(const_cast<double *>(pd.col[j]) + off, *hc[j], 8 * len,
                                    cudaMemcpyHostToDevice, eb->copy);
                if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(params)");
                pk.col[j] = pd.col[j] + off;
            }
            cudaStream_t cs = eb->comp[b];
            e = cudaEventRecord(eb->uploaded[b], eb->copy);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, eb->uploaded[b], 0);
            if (e != cudaSuccess) return cuda_fail(e, "aeb_evaluate_scenario: chunk order");
            st = rollout_impl(md, pk, len, precision, offset_out(od, off), cs, off);
            if (st != AEB_OK) return st;
        }
        for (int i = 0; i < 2; ++i) {
            e = cudaEventRecord(eb->done[i], eb->comp[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, eb->done[i], 0);
            if (e != cudaSuccess) return cuda_fail(e, "aeb_evaluate_scenario: join");
        }
    }
    st = reduce_impl(&lay.out, n, *hist, lay.stats, s);
    if (st != AEB_OK) return st;
    e = cudaMemcpyAsync(host_stats, lay.stats, sizeof(aeb_stats), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(stats)");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return AEB_OK;
}
