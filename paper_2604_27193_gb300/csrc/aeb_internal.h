// aeb_internal.h -- declarations shared by the library's translation units.
// Nothing here is part of the C ABI (that is include/aeb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/aeb.h"

namespace aeb {

// Model constants as the kernels consume them.  hl, h2, h6 and n_max are
// taken once on the host, in binary64, in the operation order the plain
// definition uses: hl = h / L, h2 = 0.5 * dt, h6 = dt / 6, n_max = smallest n
// with n * dt >= t_max.
struct ModelDev {
    double g, rho, area, hl, beta, phi_f, a_cmd, dt, h2, h6, ttc_thr;
    // moving lead: initial speed, deceleration, stop time v/b (inf if b = 0),
    // stop position (v t_s) / 2 (the same binary64 expressions as the oracle)
    double lead_v0, lead_decel, lead_ts, lead_xs;
    // per-step perception of the TTC trigger: noise scale, dropout
    // probability, latency in steps, stream key; perc = any of them set
    double perc_sigma, perc_drop;
    uint64_t perc_seed;
    int32_t perc_lat, perc;
    int32_t n_max, cap_mode, trigger, lead;
    int32_t lead_moving;  // lead && lead_v0 > 0
};

enum Field { kV0 = 0, kD0, kMu, kGs, kGc, kMass, kCd, kTau, kTdelay, kNoise };

struct ParamsDev {
    const double *col[AEB_NFIELDS];
};

struct OutDev {
    uint8_t *status;
    double *x_raw, *x_ref, *v_imp, *t_end;
    int32_t *n_steps, *n_onset;
};

// A job: `n` samples whose parameters start at row `param_offset` of the
// columns and whose outputs start at row `out_offset`; `ttc_thr` is its TTC
// threshold (TTC trigger mode).
struct JobDev {
    uint64_t param_offset, out_offset, n;
    double ttc_thr;
    uint64_t key_offset;  // row of the job's first sample in the perception stream
};

// A tile: `count` consecutive samples of job `job`, from its sample `first`.
struct TileDesc {
    uint64_t first;
    uint32_t job, count;
};

// Work split, handed to warps through one 64-bit counter that must be zero at
// launch.  Flat mode (tiles == nullptr): samples [0, n) of one job in tiles of
// `tile` samples, parameters and outputs at the same row, the model's TTC
// threshold.  Table mode: tile t is tiles[t] of job jobs[tiles[t].job].
struct WorkDev {
    uint64_t n;
    uint32_t tile;
    unsigned long long *counter;
    const TileDesc *tiles;
    uint64_t n_tiles;
    const JobDev *jobs;
    uint64_t key_base;  // flat launches: perception-key row of sample 0
};

struct LaunchCfg {
    int block;          // threads per block (multiple of 32)
    int blocks_per_sm;  // resident blocks per SM requested (0: occupancy max)
    int tile;           // samples per tile (multiple of 32)
};

// Launchers (asynchronous on `stream`; return a cudaError_t of the launch).
cudaError_t launch_rollout_fp64(const ModelDev &m, const ParamsDev &p, const OutDev &o,
                                const WorkDev &w, const LaunchCfg &cfg, cudaStream_t stream);
cudaError_t launch_rollout_fp32(const ModelDev &m, const ParamsDev &p, const OutDev &o,
                                const WorkDev &w, const LaunchCfg &cfg, cudaStream_t stream);

// Reduction: partial sums per block in fixed order, then one block finishes.
struct RedPartial {
    unsigned long long n_stop, n_contact, n_horizon, n_invalid, steps;
    double sum_d, sumsq_d, min_d, max_d, sum_v, sumsq_v, min_v, max_v;
};
int reduce_blocks_for(uint64_t n);
cudaError_t launch_reduce(const uint8_t *status, const double *x_ref, const double *v_imp,
                          const int32_t *n_steps, uint64_t n, const aeb_hist_spec &h,
                          RedPartial *partials, aeb_stats *stats, cudaStream_t stream);

// Per-job reduction: partials over the segments `blocks` (8192 rows at most,
// each inside one job), then job j adds partials [first[j], first[j+1]).
constexpr uint32_t kRedSegment = 8192;
cudaError_t launch_reduce_jobs(const uint8_t *status, const double *x_ref, const double *v_imp,
                               const int32_t *n_steps, const TileDesc *blocks, uint32_t n_blocks,
                               const uint32_t *first, const JobDev *jobs, uint32_t n_jobs,
                               RedPartial *partials, aeb_job_stats *stats, cudaStream_t s);

// Host-side helpers shared by the C-ABI glue.
int64_t steps_to_reach_host(double t, double dt);
LaunchCfg launch_cfg(aeb_precision precision);
void set_launch_cfg(aeb_precision precision, const LaunchCfg &cfg);
aeb_status check_model(const aeb_model *m, ModelDev *out);
aeb_status check_params(const aeb_params *p, ParamsDev *out);
// A histogram spec: finite origins, widths positive powers of two (AEB_EINVAL
// with a message otherwise); shared by every reduction entry point.
aeb_status check_hist(const aeb_hist_spec *h);
OutDev out_dev(const aeb_outputs *o);
aeb_status cuda_fail(cudaError_t e, const char *what);

// Weighted event sums for importance sampling (reduce_weighted.cu): at most
// kWMaxBlocks partials in `partials` (weighted_partial_bytes() bytes).
constexpr int kWMaxBlocks = 1024;
size_t weighted_partial_bytes();
cudaError_t launch_reduce_weighted(const uint8_t *status, const double *x_ref, const double *w,
                                   uint64_t n, double x_thr, void *partials, aeb_wstats *stats,
                                   cudaStream_t s);

}  // namespace aeb
