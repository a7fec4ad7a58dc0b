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
    int32_t n_max, cap_mode, trigger, lead;
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

// Work split: samples [0, n) in tiles of `tile` consecutive samples, handed
// to warps through one 64-bit counter that must be zero at launch.
struct WorkDev {
    uint64_t n;
    uint32_t tile;
    unsigned long long *counter;
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

// Host-side helpers shared by the C-ABI glue.
int64_t steps_to_reach_host(double t, double dt);

}  // namespace aeb
