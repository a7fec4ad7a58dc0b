// serve.cpp -- serving engine: continuous batching of scenario requests.
//
// A request is (scenario, n).  Its life:
//   pending  -> admitted: rows [r0, r0 + n) of the device arena (and of the
//               pinned staging) are granted first-fit, FIFO; requests wait
//               for rows to be freed when the arena is full
//   sampling -> uploading: the host sampler (Sec. IV-C) fills the staging rows,
//               ten column copies move them to the device rows on a copy stream
//   ready    -> the request is cut into fixed chunks of chunk_samples; chunks
//               of all ready requests are queued FIFO
//   waves    -> the scheduler takes queued chunks up to wave_samples, builds a
//               (chunk, tile) table and launches one persistent rollout over it
//               plus a per-chunk fixed-order reduction; waves alternate over
//               streams so a wave's tail overlaps the next wave's start
//   done     -> when every chunk of a request is reduced, the chunk statistics
//               are combined in chunk order, the rows are freed and pollers wake.
// Because chunks are fixed pieces of a request and each is reduced in a fixed
// order, a request's statistics are the same bits whatever it shares waves
// with.  The GPU never waits on the host: every wave is a bounded launch.
//
// Failures.  A request fails when its rows cannot be granted (AEB_ENOMEM),
// its sampling or upload fails, a wave holding one of its chunks fails to
// launch or completes with an error (AEB_ECUDA), or such a wave has not
// completed wave_timeout_ms after its launch (the watchdog: AEB_ETIMEOUT).
// A failed request's queued chunks are dropped, and its rows return to the
// arena once none of its chunks is on the GPU any more (a timed-out wave keeps
// its rows until it completes), so that no later request's upload or rollout
// can overlap work still writing those rows.  Other requests carry on.
// Failures can be injected on the host (aeb_serve_inject_faults) to test
// these paths without any GPU fault.
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "aeb_internal.h"
#include "host_util.h"

namespace aeb {
namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// First-fit allocator of row ranges inside [0, cap).
class RowArena {
    std::map<uint64_t, uint64_t> free_;  // start -> length

  public:
    void init(uint64_t cap)
    {
        free_.clear();
        if (cap) free_[0] = cap;
    }
    bool alloc(uint64_t n, uint64_t *start)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const uint64_t s = it->first, rem = it->second - n;
            free_.erase(it);
            if (rem) free_[s + n] = rem;
            *start = s;
            return true;
        }
        return false;
    }
    void release(uint64_t s, uint64_t n)
    {
        auto it = free_.emplace(s, n).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
};

enum class RState { Pending, Sampling, Uploading, Ready, Done, Cancelled, Failed };

struct Req {
    uint64_t ticket = 0;
    aeb_scenario sc{};
    uint64_t n = 0;
    RState state = RState::Pending;
    bool cancel = false;
    bool rows_held = false;    // rows [row0, row0 + n) granted and not yet returned
    uint64_t row0 = 0;
    uint32_t n_chunks = 0, chunks_done = 0;
    uint32_t inflight = 0;     // chunks in waves the GPU has not finished
    std::vector<aeb_job_stats> chunk;
    cudaEvent_t up_evt = nullptr;
    Clock::time_point t_submit, t_admit, t_ready, t_done;
    aeb_job_stats result{};
    aeb_status err = AEB_OK;
};

using ReqP = std::shared_ptr<Req>;

struct ChunkRef {
    ReqP req;
    uint32_t index;
    uint64_t first, n;
};

struct Wave {
    void *dmem = nullptr, *hmem = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    bool timed_out = false;       // the watchdog has failed this wave's requests
    bool inject_error = false;    // report this wave's completion as a CUDA error
    Clock::time_point t_launch;
    std::vector<ChunkRef> chunks;
    // device and pinned sub-buffers
    unsigned long long *counter = nullptr;
    JobDev *djobs = nullptr, *hjobs = nullptr;
    TileDesc *dtiles = nullptr, *htiles = nullptr, *dred = nullptr, *hred = nullptr;
    uint32_t *dfirst = nullptr, *hfirst = nullptr;
    RedPartial *dpart = nullptr;
    aeb_job_stats *dstats = nullptr, *hstats = nullptr;
};

constexpr uint32_t kMaxJobsPerWave = 4096;
constexpr int32_t kDefaultWaveTimeoutMs = 10000;

// Host-side fault injection (tests of the failure paths): the k-th admission,
// wave launch or wave completion counted from the injection fails; a delay
// holds every wave's completion back.
struct Faults {
    uint64_t admissions = 0, launches = 0, completions = 0;       // counts so far
    uint64_t admission_at = 0, launch_at = 0, completion_at = 0;  // 0: none
    int32_t delay_ms = 0;
};

void combine(aeb_job_stats &acc, const aeb_job_stats &c)
{
    acc.n += c.n;
    acc.n_stop += c.n_stop;
    acc.n_contact += c.n_contact;
    acc.n_horizon += c.n_horizon;
    acc.n_invalid += c.n_invalid;
    acc.steps += c.steps;
    acc.sum_d += c.sum_d;
    acc.sumsq_d += c.sumsq_d;
    acc.sum_v += c.sum_v;
    acc.sumsq_v += c.sumsq_v;
    acc.min_d = std::fmin(acc.min_d, c.min_d);
    acc.max_d = std::fmax(acc.max_d, c.max_d);
    acc.min_v = std::fmin(acc.min_v, c.min_v);
    acc.max_v = std::fmax(acc.max_v, c.max_v);
}

}  // namespace
}  // namespace aeb

using namespace aeb;

struct aeb_server {
    aeb_serve_cfg cfg{};
    aeb_model model{};
    ModelDev md{};
    LaunchCfg lcfg{};
    // device arena: 10 parameter columns + 4 output columns of arena_rows rows
    void *arena = nullptr;
    double *dcol[AEB_NFIELDS] = {};
    uint8_t *dstatus = nullptr;
    double *dxref = nullptr, *dvimp = nullptr;
    int32_t *dnsteps = nullptr;
    double *hcol[AEB_NFIELDS] = {};  // pinned staging columns
    void *staging = nullptr;
    RowArena rows;
    cudaStream_t copy_stream = nullptr;
    std::vector<Wave> waves;
    size_t next_wave = 0;

    std::mutex mu;
    std::condition_variable cv_feed;   // pending requests / freed rows
    std::condition_variable cv_done;   // request completions
    std::condition_variable cv_sched;  // work for the scheduler
    std::deque<ReqP> pending;
    std::vector<ReqP> uploading;
    std::deque<ChunkRef> ready;
    std::map<uint64_t, ReqP> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    bool feeder_done = false;  // the feeder has left its loop (nothing more to upload)
    aeb_serve_counters counters{};
    uint64_t rows_free = 0;
    int32_t wave_timeout_ms = kDefaultWaveTimeoutMs;  // < 0: no watchdog
    Faults faults;
    std::thread feeder, scheduler;

    void run_feeder();
    void run_scheduler();
    bool launch_wave(Wave &w);
    void finish_wave(Wave &w, bool ok);
    void retire_chunk(const ChunkRef &c, const aeb_job_stats *st, Clock::time_point now);
    void finish_request(const ReqP &r, Clock::time_point now);
    void fail_request(const ReqP &r, aeb_status code);
    void release_rows(const ReqP &r);
};

// Return a request's rows to the arena (once).
void aeb_server::release_rows(const ReqP &r)
{
    if (!r->rows_held) return;
    rows.release(r->row0, r->n);
    rows_free += r->n;
    r->rows_held = false;
    cv_feed.notify_all();
}

// End a request with an error (once): its queued chunks are dropped; its rows
// return now if none of its chunks is on the GPU, else when the last retires.
void aeb_server::fail_request(const ReqP &r, aeb_status code)
{
    if (r->state == RState::Done || r->state == RState::Cancelled || r->state == RState::Failed)
        return;
    r->state = RState::Failed;
    r->err = code;
    counters.failed++;
    if (code == AEB_ETIMEOUT) counters.timed_out++;
    for (auto it = ready.begin(); it != ready.end();)
        it = (it->req == r) ? ready.erase(it) : std::next(it);
    if (r->inflight == 0) release_rows(r);
    cv_done.notify_all();
}

// A chunk's wave has finished on the GPU (st: its statistics, or NULL if the
// wave failed).
void aeb_server::retire_chunk(const ChunkRef &c, const aeb_job_stats *st, Clock::time_point now)
{
    const ReqP &r = c.req;
    r->inflight--;
    if (r->state == RState::Ready) {
        if (!st) {
            fail_request(r, AEB_ECUDA);
            return;
        }
        r->chunk[c.index] = *st;
        if (++r->chunks_done == r->n_chunks) finish_request(r, now);
    } else if (r->state == RState::Failed && r->inflight == 0) {
        release_rows(r);
    }
}

void aeb_server::finish_request(const ReqP &r, Clock::time_point now)
{
    aeb_job_stats acc{};
    acc.min_d = acc.min_v = INFINITY;
    acc.max_d = acc.max_v = -INFINITY;
    for (const auto &c : r->chunk) combine(acc, c);  // chunk order: fixed
    r->result = acc;
    r->t_done = now;
    r->state = r->cancel ? RState::Cancelled : RState::Done;
    release_rows(r);
    if (r->cancel)
        counters.cancelled++;
    else
        counters.completed++;
    counters.rollouts += r->n;
    cv_done.notify_all();
}

void aeb_server::run_feeder()
{
    cudaSetDevice(cfg.device);
    for (;;) {
        ReqP r;
        {
            std::unique_lock<std::mutex> lk(mu);
            for (;;) {
                if (stop) {
                    feeder_done = true;
                    cv_sched.notify_all();
                    return;
                }
                while (!pending.empty() && pending.front()->cancel) {
                    ReqP c = pending.front();
                    pending.pop_front();
                    c->state = RState::Cancelled;
                    counters.cancelled++;
                    cv_done.notify_all();
                }
                if (!pending.empty()) {
                    uint64_t r0 = 0;
                    if (rows.alloc(pending.front()->n, &r0)) {
                        r = pending.front();
                        pending.pop_front();
                        r->row0 = r0;
                        r->rows_held = true;
                        rows_free -= r->n;
                        r->t_admit = Clock::now();
                        if (++faults.admissions == faults.admission_at) {
                            // injected: the grant fails as if the memory were gone
                            faults.admission_at = 0;
                            release_rows(r);
                            fail_request(r, AEB_ENOMEM);
                            r.reset();
                            continue;
                        }
                        r->state = RState::Sampling;
                        break;
                    }
                }
                cv_feed.wait(lk);  // new request, freed rows or stop
            }
        }
        aeb_params host{};
        double **hp[AEB_NFIELDS] = {&host.v0, &host.d0, &host.mu, &host.gs, &host.gc,
                                    &host.mass, &host.cd, &host.tau, &host.t_delay, &host.noise};
        for (int f = 0; f < AEB_NFIELDS; ++f) *hp[f] = hcol[f] + r->row0;
        aeb_status st = aeb_sample_params(&model, &r->sc, 0, r->n, &host, cfg.sampler_threads);
        cudaError_t e = cudaSuccess;
        for (int f = 0; f < AEB_NFIELDS && st == AEB_OK && e == cudaSuccess; ++f)
            e = cudaMemcpyAsync(dcol[f] + r->row0, hcol[f] + r->row0, 8 * r->n,
                                cudaMemcpyHostToDevice, copy_stream);
        if (e == cudaSuccess && st == AEB_OK) e = cudaEventCreateWithFlags(&r->up_evt, cudaEventDisableTiming);
        if (e == cudaSuccess && st == AEB_OK) e = cudaEventRecord(r->up_evt, copy_stream);
        std::lock_guard<std::mutex> lk(mu);
        if (st != AEB_OK || e != cudaSuccess) {
            if (r->up_evt) {
                cudaEventDestroy(r->up_evt);
                r->up_evt = nullptr;
            }
            // the copies already queued must end before the rows are reused
            cudaStreamSynchronize(copy_stream);
            fail_request(r, st != AEB_OK ? st : AEB_ECUDA);
            continue;
        }
        r->state = RState::Uploading;
        uploading.push_back(r);
        cv_sched.notify_all();
    }
}

bool aeb_server::launch_wave(Wave &w)
{
    // take queued chunks FIFO up to wave_samples (always at least one)
    uint64_t total = 0;
    w.chunks.clear();
    while (!ready.empty() && w.chunks.size() < kMaxJobsPerWave) {
        const ChunkRef &c = ready.front();
        if (!w.chunks.empty() && total + c.n > cfg.wave_samples) break;
        total += c.n;
        w.chunks.push_back(c);
        ready.pop_front();
    }
    if (w.chunks.empty()) return false;
    for (auto &c : w.chunks) c.req->inflight++;
    const uint32_t T = (uint32_t)lcfg.tile;
    const uint32_t nj = (uint32_t)w.chunks.size();
    uint32_t nt = 0, nr = 0;
    for (uint32_t j = 0; j < nj; ++j) {
        const ChunkRef &c = w.chunks[j];
        const uint64_t row = c.req->row0 + c.first;
        // readings keyed by the sample's index in its request, so a request's
        // results do not depend on where it sits in the arena
        w.hjobs[j] = JobDev{row, row, c.n, model.ttc_thr, c.first};
        for (uint64_t f = 0; f < c.n; f += T)
            w.htiles[nt++] = TileDesc{f, j, (uint32_t)std::min<uint64_t>(T, c.n - f)};
        w.hfirst[j] = nr;
        for (uint64_t f = 0; f < c.n; f += kRedSegment)
            w.hred[nr++] = TileDesc{f, j, (uint32_t)std::min<uint64_t>(kRedSegment, c.n - f)};
    }
    w.hfirst[nj] = nr;
    cudaError_t e = cudaSuccess;
    if (++faults.launches == faults.launch_at) {  // injected: the launch reports an error
        faults.launch_at = 0;
        e = cudaErrorLaunchFailure;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w.djobs, w.hjobs, sizeof(JobDev) * nj, cudaMemcpyHostToDevice, w.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w.dtiles, w.htiles, sizeof(TileDesc) * nt, cudaMemcpyHostToDevice, w.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w.dred, w.hred, sizeof(TileDesc) * nr, cudaMemcpyHostToDevice, w.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w.dfirst, w.hfirst, sizeof(uint32_t) * (nj + 1), cudaMemcpyHostToDevice,
                            w.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.counter, 0, sizeof(unsigned long long), w.stream);
    if (e == cudaSuccess) {
        ParamsDev pd;
        for (int f = 0; f < AEB_NFIELDS; ++f) pd.col[f] = dcol[f];
        OutDev od{};
        od.status = dstatus;
        od.x_ref = dxref;
        od.v_imp = dvimp;
        od.n_steps = dnsteps;
        WorkDev wd{total, T, w.counter, w.dtiles, nt, w.djobs, 0};
        e = (cfg.precision == AEB_FP64_PLAIN) ? launch_rollout_fp64(md, pd, od, wd, lcfg, w.stream)
                                              : launch_rollout_fp32(md, pd, od, wd, lcfg, w.stream);
    }
    if (e == cudaSuccess)
        e = launch_reduce_jobs(dstatus, dxref, dvimp, dnsteps, w.dred, nr, w.dfirst, w.djobs, nj,
                               w.dpart, w.dstats, w.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w.hstats, w.dstats, sizeof(aeb_job_stats) * nj, cudaMemcpyDeviceToHost,
                            w.stream);
    if (e == cudaSuccess) e = cudaEventRecord(w.done, w.stream);
    if (e != cudaSuccess) {
        // whatever part of the wave was queued ends before its rows are reused
        cudaStreamSynchronize(w.stream);
        finish_wave(w, false);
        return false;
    }
    w.busy = true;
    w.timed_out = false;
    w.inject_error = (++faults.completions == faults.completion_at);
    if (w.inject_error) faults.completion_at = 0;
    w.t_launch = Clock::now();
    counters.waves++;
    return true;
}

// The GPU has finished wave w (ok: without error): retire its chunks.
void aeb_server::finish_wave(Wave &w, bool ok)
{
    const Clock::time_point now = Clock::now();
    for (size_t j = 0; j < w.chunks.size(); ++j) retire_chunk(w.chunks[j], ok ? &w.hstats[j] : nullptr, now);
    w.chunks.clear();
    w.busy = false;
    w.timed_out = false;
    w.inject_error = false;
}

void aeb_server::run_scheduler()
{
    cudaSetDevice(cfg.device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool progress = false;
        for (size_t k = 0; k < uploading.size();) {
            const cudaError_t q = cudaEventQuery(uploading[k]->up_evt);
            if (q == cudaErrorNotReady) {
                ++k;
                continue;
            }
            ReqP r = uploading[k];
            uploading.erase(uploading.begin() + k);
            cudaEventDestroy(r->up_evt);
            r->up_evt = nullptr;
            progress = true;
            if (q != cudaSuccess) {
                fail_request(r, AEB_ECUDA);
                continue;
            }
            if (r->state != RState::Uploading) {  // failed meanwhile
                release_rows(r);
                continue;
            }
            r->state = RState::Ready;
            r->t_ready = Clock::now();
            const uint64_t C = cfg.chunk_samples;
            r->n_chunks = (uint32_t)((r->n + C - 1) / C);
            r->chunk.assign(r->n_chunks, aeb_job_stats{});
            for (uint32_t c = 0; c < r->n_chunks; ++c)
                ready.push_back(ChunkRef{r, c, c * C, std::min<uint64_t>(C, r->n - c * C)});
        }
        bool any_busy = false;
        const Clock::time_point now = Clock::now();
        for (auto &w : waves) {
            if (!w.busy) continue;
            cudaError_t q = cudaEventQuery(w.done);
            if (q == cudaSuccess && faults.delay_ms > 0 &&
                now < w.t_launch + std::chrono::milliseconds(faults.delay_ms))
                q = cudaErrorNotReady;  // injected: completion held back
            if (q == cudaSuccess && w.inject_error) q = cudaErrorLaunchFailure;
            if (q == cudaErrorNotReady) {
                any_busy = true;
                if (!w.timed_out && wave_timeout_ms >= 0 &&
                    now > w.t_launch + std::chrono::milliseconds(wave_timeout_ms)) {
                    // watchdog: the wave's requests stop waiting; the rows stay
                    // held until the GPU finishes the wave
                    w.timed_out = true;
                    for (auto &c : w.chunks) fail_request(c.req, AEB_ETIMEOUT);
                    progress = true;
                }
                continue;
            }
            finish_wave(w, q == cudaSuccess);
            progress = true;
        }
        while (!ready.empty()) {
            Wave *free_w = nullptr;
            for (size_t k = 0; k < waves.size(); ++k) {
                Wave &w = waves[(next_wave + k) % waves.size()];
                if (!w.busy) {
                    free_w = &w;
                    next_wave = (next_wave + k + 1) % waves.size();
                    break;
                }
            }
            if (!free_w || !launch_wave(*free_w)) break;
            any_busy = true;
            progress = true;
        }
        if (stop && feeder_done && uploading.empty() && !any_busy && ready.empty()) return;
        if (!progress) {
            if (any_busy || !uploading.empty())
                cv_sched.wait_for(lk, std::chrono::microseconds(50));  // GPU work in flight: poll
            else
                cv_sched.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
}

namespace aeb {
namespace {

void free_server(aeb_server *s)
{
    if (!s) return;
    cudaSetDevice(s->cfg.device);
    for (auto &w : s->waves) {
        if (w.done) cudaEventDestroy(w.done);
        if (w.stream) cudaStreamDestroy(w.stream);
        if (w.dmem) cudaFree(w.dmem);
        if (w.hmem) cudaFreeHost(w.hmem);
    }
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->arena) cudaFree(s->arena);
    if (s->staging) cudaFreeHost(s->staging);
    delete s;
}

}  // namespace
}  // namespace aeb

extern "C" aeb_status aeb_serve_create(const aeb_serve_cfg *cfg, const aeb_model *model,
                                       aeb_server **out)
{
    clear_error();
    if (!cfg || !model || !out) return fail(AEB_EINVAL, "aeb_serve_create: NULL argument");
    *out = nullptr;
    ModelDev md;
    aeb_status st = check_model(model, &md);
    if (st != AEB_OK) return st;
    if (cfg->precision != AEB_FP64_PLAIN && cfg->precision != AEB_FP32_COMP)
        return fail(AEB_EINVAL, "aeb_serve_create: unknown precision");
    if (cfg->arena_rows == 0 || cfg->chunk_samples == 0 || cfg->chunk_samples % 64 ||
        cfg->wave_samples < cfg->chunk_samples || cfg->max_waves_in_flight < 1 ||
        cfg->max_waves_in_flight > 4 || cfg->max_request_samples == 0 ||
        cfg->max_request_samples > cfg->arena_rows || cfg->reserved != 0)
        return fail(AEB_EINVAL, "aeb_serve_create: invalid configuration");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev)
        return fail(AEB_EDEVICE, "aeb_serve_create: no such device");
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");

    aeb_server *s = new aeb_server;
    s->cfg = *cfg;
    s->model = *model;
    s->md = md;
    s->lcfg = launch_cfg(cfg->precision);
    const uint64_t R = cfg->arena_rows;
    const size_t col = a256(8 * R);
    const size_t bytes = AEB_NFIELDS * col + a256(R) + 2 * col + a256(4 * R);
    e = cudaMalloc(&s->arena, bytes);
    if (e != cudaSuccess) {
        free_server(s);
        return cuda_fail(e, "aeb_serve_create: device arena");
    }
    char *p = static_cast<char *>(s->arena);
    for (int f = 0; f < AEB_NFIELDS; ++f, p += col) s->dcol[f] = reinterpret_cast<double *>(p);
    s->dstatus = reinterpret_cast<uint8_t *>(p);
    p += a256(R);
    s->dxref = reinterpret_cast<double *>(p);
    p += col;
    s->dvimp = reinterpret_cast<double *>(p);
    p += col;
    s->dnsteps = reinterpret_cast<int32_t *>(p);
    e = cudaHostAlloc(&s->staging, AEB_NFIELDS * col, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        free_server(s);
        return cuda_fail(e, "aeb_serve_create: pinned staging");
    }
    for (int f = 0; f < AEB_NFIELDS; ++f)
        s->hcol[f] = reinterpret_cast<double *>(static_cast<char *>(s->staging) + f * col);
    s->rows.init(R);
    s->rows_free = R;
    s->wave_timeout_ms = cfg->wave_timeout_ms == 0 ? kDefaultWaveTimeoutMs : cfg->wave_timeout_ms;
    e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
    // wave slots
    const uint64_t T = (uint64_t)s->lcfg.tile;
    const uint64_t max_tiles = cfg->wave_samples / T + kMaxJobsPerWave;
    const uint64_t max_red = cfg->wave_samples / kRedSegment + kMaxJobsPerWave;
    const size_t sz_jobs = a256(sizeof(JobDev) * kMaxJobsPerWave);
    const size_t sz_tiles = a256(sizeof(TileDesc) * max_tiles);
    const size_t sz_red = a256(sizeof(TileDesc) * max_red);
    const size_t sz_first = a256(sizeof(uint32_t) * (kMaxJobsPerWave + 1));
    const size_t sz_part = a256(sizeof(RedPartial) * max_red);
    const size_t sz_stats = a256(sizeof(aeb_job_stats) * kMaxJobsPerWave);
    s->waves.resize(cfg->max_waves_in_flight);
    for (auto &w : s->waves) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaMalloc(&w.dmem, 256 + sz_jobs + sz_tiles + sz_red + sz_first + sz_part + sz_stats);
        if (e == cudaSuccess)
            e = cudaHostAlloc(&w.hmem, sz_jobs + sz_tiles + sz_red + sz_first + sz_stats,
                              cudaHostAllocDefault);
        if (e != cudaSuccess) break;
        char *d = static_cast<char *>(w.dmem);
        w.counter = reinterpret_cast<unsigned long long *>(d);
        d += 256;
        w.djobs = reinterpret_cast<JobDev *>(d);
        d += sz_jobs;
        w.dtiles = reinterpret_cast<TileDesc *>(d);
        d += sz_tiles;
        w.dred = reinterpret_cast<TileDesc *>(d);
        d += sz_red;
        w.dfirst = reinterpret_cast<uint32_t *>(d);
        d += sz_first;
        w.dpart = reinterpret_cast<RedPartial *>(d);
        d += sz_part;
        w.dstats = reinterpret_cast<aeb_job_stats *>(d);
        char *h = static_cast<char *>(w.hmem);
        w.hjobs = reinterpret_cast<JobDev *>(h);
        h += sz_jobs;
        w.htiles = reinterpret_cast<TileDesc *>(h);
        h += sz_tiles;
        w.hred = reinterpret_cast<TileDesc *>(h);
        h += sz_red;
        w.hfirst = reinterpret_cast<uint32_t *>(h);
        h += sz_first;
        w.hstats = reinterpret_cast<aeb_job_stats *>(h);
    }
    if (e != cudaSuccess) {
        free_server(s);
        return cuda_fail(e, "aeb_serve_create: wave buffers");
    }
    try {
        s->feeder = std::thread([s] { s->run_feeder(); });
        s->scheduler = std::thread([s] { s->run_scheduler(); });
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_feed.notify_all();
        s->cv_sched.notify_all();
        if (s->feeder.joinable()) s->feeder.join();
        if (s->scheduler.joinable()) s->scheduler.join();
        free_server(s);
        return fail(AEB_ENOMEM, "aeb_serve_create: could not start threads");
    }
    *out = s;
    return AEB_OK;
}

extern "C" aeb_status aeb_serve_submit(aeb_server *srv, const aeb_scenario *scenario, uint64_t n,
                                       uint64_t *ticket)
{
    clear_error();
    if (!srv || !scenario || !ticket) return fail(AEB_EINVAL, "aeb_serve_submit: NULL argument");
    if (n == 0 || n > srv->cfg.max_request_samples)
        return fail(AEB_EINVAL, "aeb_serve_submit: n must be in [1, max_request_samples]");
    // validate the scenario by sampling nothing
    aeb_params none{};
    double dummy = 0.0;
    double **cols[AEB_NFIELDS] = {&none.v0, &none.d0, &none.mu, &none.gs, &none.gc,
                                  &none.mass, &none.cd, &none.tau, &none.t_delay, &none.noise};
    for (auto c : cols) *c = &dummy;
    aeb_status st = aeb_sample_params(&srv->model, scenario, 0, 0, &none, 1);
    if (st != AEB_OK) return st;
    auto r = std::make_shared<Req>();
    r->sc = *scenario;
    r->n = n;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return fail(AEB_EINVAL, "aeb_serve_submit: engine is stopping");
        r->ticket = srv->next_ticket++;
        srv->reqs[r->ticket] = r;
        srv->pending.push_back(r);
        srv->counters.submitted++;
        *ticket = r->ticket;
    }
    srv->cv_feed.notify_all();
    return AEB_OK;
}

extern "C" aeb_status aeb_serve_poll(aeb_server *srv, uint64_t ticket, int32_t timeout_ms,
                                     aeb_job_stats *stats, aeb_latency *lat)
{
    clear_error();
    if (!srv) return fail(AEB_EINVAL, "aeb_serve_poll: NULL server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(AEB_EINVAL, "aeb_serve_poll: unknown ticket");
    ReqP r = it->second;
    auto finished = [&] {
        return r->state == RState::Done || r->state == RState::Cancelled ||
               r->state == RState::Failed;
    };
    if (!finished()) {
        if (timeout_ms == 0) return AEB_EAGAIN;
        if (timeout_ms < 0)
            srv->cv_done.wait(lk, finished);
        else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished))
            return fail(AEB_ETIMEOUT, "aeb_serve_poll: request still running");
    }
    srv->reqs.erase(r->ticket);
    if (r->state == RState::Cancelled) return fail(AEB_ECANCELLED, "aeb_serve_poll: cancelled");
    if (r->state == RState::Failed)
        return fail(r->err, r->err == AEB_ETIMEOUT
                                ? "aeb_serve_poll: a wave of the request did not complete "
                                  "within wave_timeout_ms"
                                : (r->err == AEB_ENOMEM ? "aeb_serve_poll: no arena rows for "
                                                          "the request"
                                                        : "aeb_serve_poll: request failed"));
    if (stats) *stats = r->result;
    if (lat) {
        lat->queue_ms = ms_between(r->t_submit, r->t_admit);
        lat->sample_ms = ms_between(r->t_admit, r->t_ready);
        lat->gpu_ms = ms_between(r->t_ready, r->t_done);
        lat->total_ms = ms_between(r->t_submit, r->t_done);
    }
    return AEB_OK;
}

extern "C" aeb_status aeb_serve_cancel(aeb_server *srv, uint64_t ticket)
{
    clear_error();
    if (!srv) return fail(AEB_EINVAL, "aeb_serve_cancel: NULL server");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(AEB_EINVAL, "aeb_serve_cancel: unknown ticket");
    it->second->cancel = true;
    srv->cv_feed.notify_all();
    return AEB_OK;
}

extern "C" aeb_status aeb_serve_counters_get(aeb_server *srv, aeb_serve_counters *out)
{
    clear_error();
    if (!srv || !out) return fail(AEB_EINVAL, "aeb_serve_counters_get: NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->counters;
    out->rows_free = srv->rows_free;
    return AEB_OK;
}

extern "C" aeb_status aeb_serve_inject_faults(aeb_server *srv, const aeb_serve_faults *f)
{
    clear_error();
    if (!srv || !f) return fail(AEB_EINVAL, "aeb_serve_inject_faults: NULL argument");
    if (f->hold_waves_ms < 0 || f->reserved != 0)
        return fail(AEB_EINVAL, "aeb_serve_inject_faults: hold_waves_ms < 0 or reserved != 0");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        Faults &F = srv->faults;
        F.admission_at = f->fail_admission ? F.admissions + f->fail_admission : 0;
        F.launch_at = f->fail_wave_launch ? F.launches + f->fail_wave_launch : 0;
        F.completion_at = f->fail_wave_completion ? F.completions + f->fail_wave_completion : 0;
        F.delay_ms = f->hold_waves_ms;
    }
    srv->cv_sched.notify_all();
    return AEB_OK;
}

extern "C" void aeb_serve_destroy(aeb_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        for (auto &r : srv->pending) {
            r->state = RState::Cancelled;
            srv->counters.cancelled++;
        }
        srv->pending.clear();
    }
    srv->cv_feed.notify_all();
    srv->cv_sched.notify_all();
    srv->cv_done.notify_all();
    if (srv->feeder.joinable()) srv->feeder.join();
    if (srv->scheduler.joinable()) srv->scheduler.join();
    free_server(srv);
}
