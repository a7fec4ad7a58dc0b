// rollout_common.cuh -- pieces shared by the FP64 and FP32-compensated rollout
// kernels: the warp work queue (lane refill), the per-sample validity test, the
// step-count rule and the output store.
#pragma once

#include "aeb_internal.h"

namespace aeb {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kNone = ~0ull;

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// A warp's cursor into the sample tiles.  All 32 lanes call take() together
// with the same `need` mask (the lanes whose rollout just ended).  Each lane
// in `need` receives the next unclaimed sample index of the warp's tile; when
// the tile is used up the warp claims the next tile from the global counter.
// Lanes get kNone once every tile has been claimed.  Sample order inside a
// warp depends only on when its lanes finish, never on other warps, but which
// tiles a warp owns depends on timing: per-sample results never do.
struct WarpQueue {
    uint64_t cur = 0, end = 0;  // warp-uniform
    bool dry = false;

    __device__ __forceinline__ uint64_t take(unsigned need, const WorkDev &w)
    {
        const unsigned lane = threadIdx.x & 31u;
        uint64_t mine = kNone;
        while (need && !dry) {
            if (cur >= end) {
                unsigned long long t = 0;
                if (lane == 0) t = atomicAdd(w.counter, 1ull);
                t = __shfl_sync(kFull, t, 0);
                uint64_t start = (uint64_t)t * w.tile;
                if (start >= w.n) { dry = true; break; }
                cur = start;
                end = (start + w.tile < w.n) ? start + w.tile : w.n;
            }
            uint64_t avail = end - cur;
            unsigned rank = __popc(need & lanemask_lt());
            bool got = ((need >> lane) & 1u) && rank < avail;
            if (got) mine = cur + rank;
            unsigned taken = __ballot_sync(kFull, got);
            cur += __popc(taken);
            need &= ~taken;
        }
        return mine;
    }
};

// A sample is invalid if any field is not finite, mass <= 0, or tau, mu, C_d
// or the delay is negative.
__device__ __forceinline__ bool sample_valid(const double f[AEB_NFIELDS])
{
#pragma unroll
    for (int j = 0; j < AEB_NFIELDS; ++j)
        if (!isfinite(f[j])) return false;
    if (!(f[kMass] > 0.0) || f[kTau] < 0.0 || f[kMu] < 0.0 || f[kCd] < 0.0 || f[kTdelay] < 0.0)
        return false;
    return true;
}

// Smallest n >= 0 with (double)n * dt >= t (clamped to 2^31 - 1).  The
// adjustment loops make the result independent of how the first guess rounds.
__device__ __forceinline__ int32_t steps_to_reach_dev(double t, double dt)
{
    if (!(t > 0.0)) return 0;
    double q = ceil(t / dt);
    if (!(q <= 2147483647.0)) return 2147483647;
    long long n = (long long)q;
    while (n > 0 && (double)(n - 1) * dt >= t) --n;
    while ((double)n * dt < t) ++n;
    return (int32_t)n;
}

__device__ __forceinline__ void store_out(const OutDev &o, uint64_t i, uint8_t status,
                                          double x_raw, double x_ref, double v_imp,
                                          double t_end, int32_t n_steps, int32_t n_onset)
{
    if (o.status) o.status[i] = status;
    if (o.x_raw) o.x_raw[i] = x_raw;
    if (o.x_ref) o.x_ref[i] = x_ref;
    if (o.v_imp) o.v_imp[i] = v_imp;
    if (o.t_end) o.t_end[i] = t_end;
    if (o.n_steps) o.n_steps[i] = n_steps;
    if (o.n_onset) o.n_onset[i] = n_onset;
}

__device__ __forceinline__ void load_fields(const ParamsDev &p, uint64_t i, double f[AEB_NFIELDS])
{
#pragma unroll
    for (int j = 0; j < AEB_NFIELDS; ++j) f[j] = __ldg(p.col[j] + i);
}

}  // namespace aeb

namespace aeb {

// The per-warp driver shared by both precisions.  `Lane` provides
//   bool init(M, X, P, O, i)  -- load sample i; true if it already ended (stored)
//   bool step(M, X, P, O, i)  -- one RK4 step; true if the rollout ended (stored)
// where X holds precision-specific constants (kernel parameters, so the
// compiler reads them from the parameter bank rather than registers).
// Each lane owns one rollout at a time (Sec. V-A, one thread per sample); a
// lane whose rollout ends takes the next sample of its warp's tile, so a warp
// keeps all 32 lanes busy until the tiles run out instead of idling until its
// slowest rollout ends.  There is no wait on other warps or on the host: the
// loop ends when no lane holds a rollout.
template <class Lane, class X>
__device__ __forceinline__ void rollout_driver(const ModelDev &M, const X &Xc, const ParamsDev &P,
                                               const OutDev &O, const WorkDev &W)
{
    const unsigned lane = threadIdx.x & 31u;
    WarpQueue q;
    Lane L;
    uint64_t idx = 0;
    bool active = false;
    unsigned need = kFull;
    for (;;) {
        while (need) {
            uint64_t got = q.take(need, W);
            bool ended = false;
            if ((need >> lane) & 1u) {
                active = (got != kNone);
                if (active) {
                    idx = got;
                    ended = L.init(M, Xc, P, O, idx);
                }
            }
            need = __ballot_sync(kFull, ended);
        }
        if (!__any_sync(kFull, active)) return;
        bool ended = false;
        if (active) ended = L.step(M, Xc, P, O, idx);
        need = __ballot_sync(kFull, ended);
    }
}

}  // namespace aeb
