// batch.cpp -- batched launches: many jobs (scenarios, thresholds) with uneven
// sample counts in one persistent rollout launch over a (job, tile) work table,
// followed by a per-job fixed-order reduction, captured once as a CUDA graph.
// Also the launch-shape configuration and its autotuner.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "aeb_internal.h"
#include "host_util.h"

struct aeb_batch {
    int device = 0;
    uint32_t n_jobs = 0;
    void *mem = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace aeb {
namespace {

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

bool valid_precision(aeb_precision p) { return p == AEB_FP64_PLAIN || p == AEB_FP32_COMP; }

aeb_status check_cfg(aeb_precision precision, const aeb_launch_config &c)
{
    if (!valid_precision(precision)) return fail(AEB_EINVAL, "unknown precision");
    if (c.tile < 32 || c.tile > 256 || c.tile % 32)
        return fail(AEB_EINVAL, "launch config: tile must be a multiple of 32 in [32, 256]");
    if (c.blocks_per_sm < 0 || c.blocks_per_sm > 32)
        return fail(AEB_EINVAL, "launch config: blocks_per_sm must be in [0, 32]");
    return AEB_OK;
}

void destroy_plan(aeb_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->mem) cudaFree(b->mem);  // waits for work still using it
    delete b;
}

}  // namespace
}  // namespace aeb

using namespace aeb;

extern "C" aeb_status aeb_batch_create(const aeb_model *model, const aeb_job *jobs, uint32_t n_jobs,
                                       const aeb_params *params, aeb_precision precision,
                                       const aeb_outputs *out, aeb_job_stats *stats,
                                       aeb_batch **plan)
{
    clear_error();
    if (!plan) return fail(AEB_EINVAL, "aeb_batch_create: plan is NULL");
    *plan = nullptr;
    if (!jobs || n_jobs == 0 || !stats || !out)
        return fail(AEB_EINVAL, "aeb_batch_create: NULL argument or no jobs");
    ModelDev md;
    ParamsDev pd;
    aeb_status st = check_model(model, &md);
    if (st != AEB_OK) return st;
    st = check_params(params, &pd);
    if (st != AEB_OK) return st;
    if (!valid_precision(precision)) return fail(AEB_EINVAL, "unknown precision");
    if (!out->status || !out->x_ref || !out->v_imp || !out->n_steps)
        return fail(AEB_EINVAL, "aeb_batch_create: status, x_ref, v_imp and n_steps are required");
    if (reinterpret_cast<uintptr_t>(stats) % 8 != 0)
        return fail(AEB_EINVAL, "aeb_batch_create: stats is not 8-byte aligned");

    const LaunchCfg cfg = launch_cfg(precision);
    const uint32_t T = (uint32_t)cfg.tile;
    std::vector<JobDev> hj(n_jobs);
    std::vector<TileDesc> tiles, red;
    std::vector<uint32_t> first(n_jobs + 1);
    uint64_t total = 0;
    for (uint32_t j = 0; j < n_jobs; ++j) {
        const aeb_job &jb = jobs[j];
        if (!std::isfinite(jb.ttc_thr)) return fail(AEB_EINVAL, "aeb_batch_create: ttc_thr not finite");
        hj[j] = JobDev{jb.param_offset, jb.out_offset, jb.n, jb.ttc_thr, jb.key_offset};
        for (uint64_t f = 0; f < jb.n; f += T)
            tiles.push_back(TileDesc{f, j, (uint32_t)std::min<uint64_t>(T, jb.n - f)});
        first[j] = (uint32_t)red.size();
        for (uint64_t f = 0; f < jb.n; f += kRedSegment)
            red.push_back(TileDesc{f, j, (uint32_t)std::min<uint64_t>(kRedSegment, jb.n - f)});
        if (red.size() > 0xffffffffull)
            return fail(AEB_EINVAL, "aeb_batch_create: too many reduction segments");
        total += jb.n;
    }
    first[n_jobs] = (uint32_t)red.size();

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    const size_t o_counter = 0;
    const size_t o_jobs = a256(sizeof(unsigned long long));
    const size_t o_tiles = o_jobs + a256(sizeof(JobDev) * n_jobs);
    const size_t o_red = o_tiles + a256(sizeof(TileDesc) * tiles.size());
    const size_t o_first = o_red + a256(sizeof(TileDesc) * red.size());
    const size_t o_part = o_first + a256(sizeof(uint32_t) * first.size());
    const size_t bytes = o_part + a256(sizeof(RedPartial) * (red.size() + 1));

    aeb_batch *b = new aeb_batch;
    b->device = dev;
    b->n_jobs = n_jobs;
    e = cudaMalloc(&b->mem, bytes);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "cudaMalloc(batch plan)");
    }
    char *base = static_cast<char *>(b->mem);
    auto *counter = reinterpret_cast<unsigned long long *>(base + o_counter);
    auto *djobs = reinterpret_cast<JobDev *>(base + o_jobs);
    auto *dtiles = reinterpret_cast<TileDesc *>(base + o_tiles);
    auto *dred = reinterpret_cast<TileDesc *>(base + o_red);
    auto *dfirst = reinterpret_cast<uint32_t *>(base + o_first);
    auto *dpart = reinterpret_cast<RedPartial *>(base + o_part);
    struct {
        void *d;
        const void *h;
        size_t n;
    } up[] = {{djobs, hj.data(), sizeof(JobDev) * hj.size()},
              {dtiles, tiles.data(), sizeof(TileDesc) * tiles.size()},
              {dred, red.data(), sizeof(TileDesc) * red.size()},
              {dfirst, first.data(), sizeof(uint32_t) * first.size()}};
    for (auto &u : up) {
        if (!u.n) continue;
        e = cudaMemcpy(u.d, u.h, u.n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            destroy_plan(b);
            return cuda_fail(e, "cudaMemcpy(batch tables)");
        }
    }

    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        destroy_plan(b);
        return cuda_fail(e, "cudaStreamCreate");
    }
    const OutDev od = out_dev(out);
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), cs);
        if (le == cudaSuccess && !tiles.empty()) {
            WorkDev w{total, T, counter, dtiles, (uint64_t)tiles.size(), djobs, 0};
            le = (precision == AEB_FP64_PLAIN) ? launch_rollout_fp64(md, pd, od, w, cfg, cs)
                                               : launch_rollout_fp32(md, pd, od, w, cfg, cs);
        }
        if (le == cudaSuccess)
            le = launch_reduce_jobs(out->status, out->x_ref, out->v_imp, out->n_steps, dred,
                                    (uint32_t)red.size(), dfirst, djobs, n_jobs, dpart, stats, cs);
        e = cudaStreamEndCapture(cs, &b->graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        destroy_plan(b);
        return cuda_fail(e, "batch graph capture");
    }
    *plan = b;
    return AEB_OK;
}

extern "C" aeb_status aeb_batch_run(aeb_batch *plan, void *stream)
{
    clear_error();
    if (!plan) return fail(AEB_EINVAL, "aeb_batch_run: plan is NULL");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != plan->device) return fail(AEB_EINVAL, "aeb_batch_run: plan belongs to another device");
    e = cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return AEB_OK;
}

extern "C" void aeb_batch_destroy(aeb_batch *plan) { destroy_plan(plan); }

extern "C" aeb_status aeb_rollout_batched(const aeb_model *model, const aeb_job *jobs,
                                          uint32_t n_jobs, const aeb_params *params,
                                          aeb_precision precision, const aeb_outputs *out,
                                          aeb_job_stats *stats, void *stream)
{
    aeb_batch *b = nullptr;
    aeb_status st = aeb_batch_create(model, jobs, n_jobs, params, precision, out, stats, &b);
    if (st != AEB_OK) return st;
    st = aeb_batch_run(b, stream);
    if (st == AEB_OK) {
        const cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
    }
    destroy_plan(b);
    return st;
}

extern "C" aeb_status aeb_get_launch_config(aeb_precision precision, aeb_launch_config *cfg)
{
    clear_error();
    if (!cfg) return fail(AEB_EINVAL, "aeb_get_launch_config: cfg is NULL");
    if (!valid_precision(precision)) return fail(AEB_EINVAL, "unknown precision");
    const LaunchCfg c = launch_cfg(precision);
    cfg->tile = c.tile;
    cfg->blocks_per_sm = c.blocks_per_sm;
    return AEB_OK;
}

extern "C" aeb_status aeb_set_launch_config(aeb_precision precision, const aeb_launch_config *cfg)
{
    clear_error();
    if (!cfg) return fail(AEB_EINVAL, "aeb_set_launch_config: cfg is NULL");
    const aeb_status st = check_cfg(precision, *cfg);
    if (st != AEB_OK) return st;
    LaunchCfg c = launch_cfg(precision);
    c.tile = cfg->tile;
    c.blocks_per_sm = cfg->blocks_per_sm;
    set_launch_cfg(precision, c);
    return AEB_OK;
}

namespace aeb {
namespace {

// Cache lines: "<key> <tile> <blocks_per_sm>", key = device|sms|precision|cap|trigger|lead.
std::string tune_key(const aeb_model &m, aeb_precision precision)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceProp prop;
    std::string name = "unknown";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char &c : name)
        if (c == ' ') c = '_';
    std::ostringstream k;
    k << name << "|" << sms << "|" << precision << "|" << m.cap_mode << "|" << m.trigger << "|"
      << m.lead;
    return k.str();
}

bool cache_lookup(const char *path, const std::string &key, aeb_launch_config *out)
{
    std::ifstream f(path);
    std::string k;
    int t, b;
    while (f >> k >> t >> b)
        if (k == key) {
            out->tile = t;
            out->blocks_per_sm = b;
            return true;
        }
    return false;
}

void cache_store(const char *path, const std::string &key, const aeb_launch_config &c)
{
    std::vector<std::string> lines;
    {
        std::ifstream f(path);
        std::string line;
        while (std::getline(f, line))
            if (line.compare(0, key.size() + 1, key + " ") != 0 && !line.empty()) lines.push_back(line);
    }
    std::ofstream f(path, std::ios::trunc);
    for (const auto &l : lines) f << l << "\n";
    f << key << " " << c.tile << " " << c.blocks_per_sm << "\n";
}

}  // namespace
}  // namespace aeb

extern "C" aeb_status aeb_autotune(const aeb_model *model, const aeb_params *params, uint64_t n,
                                   aeb_precision precision, const aeb_outputs *out, void *stream,
                                   const char *cache_path, aeb_launch_config *best)
{
    clear_error();
    if (!best || !out || n == 0) return fail(AEB_EINVAL, "aeb_autotune: NULL argument or n == 0");
    if (!valid_precision(precision)) return fail(AEB_EINVAL, "unknown precision");
    ModelDev md;
    aeb_status st = check_model(model, &md);
    if (st != AEB_OK) return st;
    const std::string key = tune_key(*model, precision);
    if (cache_path && cache_lookup(cache_path, key, best) && check_cfg(precision, *best) == AEB_OK)
        return aeb_set_launch_config(precision, best);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(AEB_ECUDA, "aeb_autotune: cudaEventCreate failed");
    const LaunchCfg saved = launch_cfg(precision);
    const int tiles64[] = {64, 128, 256}, tiles32[] = {32, 64, 128};
    const int *tl = precision == AEB_FP64_PLAIN ? tiles64 : tiles32;
    float best_ms = 1e30f;
    aeb_launch_config win{saved.tile, saved.blocks_per_sm};
    for (int ti = 0; ti < 3 && st == AEB_OK; ++ti) {
        for (int bps = 3; bps <= 8 && st == AEB_OK; ++bps) {
            LaunchCfg c = saved;
            c.tile = tl[ti];
            c.blocks_per_sm = bps;
            set_launch_cfg(precision, c);
            float ms = 0.0f;
            for (int rep = 0; rep < 2 && st == AEB_OK; ++rep) {  // warm-up, then timed
                cudaEventRecord(e0, s);
                st = aeb_rollout(model, params, n, precision, out, stream);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(AEB_ECUDA, "aeb_autotune: sync");
                cudaEventElapsedTime(&ms, e0, e1);
            }
            if (st == AEB_OK && ms < best_ms) {
                best_ms = ms;
                win = aeb_launch_config{c.tile, c.blocks_per_sm};
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    set_launch_cfg(precision, saved);
    if (st != AEB_OK) return st;
    *best = win;
    if (cache_path) cache_store(cache_path, key, win);
    return aeb_set_launch_config(precision, &win);
}
