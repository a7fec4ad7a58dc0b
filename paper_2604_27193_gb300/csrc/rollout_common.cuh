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

// A claimed tile: `count` samples with parameters at rows p0.. and outputs at
// rows o0.., and the TTC threshold of their job.  Warp-uniform.
struct Tile {
    uint64_t p0, o0, k0;  // parameter, output and perception-key rows of the first sample
    int count;
    double thr;
    bool ok;
};

// Claim the next tile (all 32 lanes call together; lane 0 takes the ticket).
__device__ __forceinline__ Tile claim_tile(const WorkDev &w, uint32_t tile_size, double model_thr)
{
    unsigned long long t = 0;
    if ((threadIdx.x & 31u) == 0) t = atomicAdd(w.counter, 1ull);
    t = __shfl_sync(kFull, t, 0);
    Tile r;
    if (!w.tiles) {
        const uint64_t start = (uint64_t)t * tile_size;
        r.ok = start < w.n;
        r.p0 = r.o0 = start;
        r.k0 = w.key_base + start;
        r.count = r.ok ? (int)((w.n - start < (uint64_t)tile_size) ? w.n - start : tile_size) : 0;
        r.thr = model_thr;
    } else {
        r.ok = t < w.n_tiles;
        r.count = 0;
        r.p0 = r.o0 = r.k0 = 0;
        r.thr = model_thr;
        if (r.ok) {
            const TileDesc d = w.tiles[t];
            const JobDev j = w.jobs[d.job];
            r.p0 = j.param_offset + d.first;
            r.o0 = j.out_offset + d.first;
            r.k0 = j.key_offset + d.first;
            r.count = (int)d.count;
            r.thr = j.ttc_thr;
        }
    }
    return r;
}

// Number of tiles a launch walks.
__host__ __forceinline__ uint64_t tiles_of(const WorkDev &w, uint32_t tile_size)
{
    return w.tiles ? w.n_tiles : (w.n + tile_size - 1) / tile_size;
}

// A warp's cursor into the sample tiles.  All 32 lanes call take() together
// with the same `need` mask (the lanes whose rollout just ended).  Each lane
// in `need` receives the next unclaimed sample of the warp's tile (its
// parameter row, output row and TTC threshold); when the tile is used up the
// warp claims the next tile.  Lanes get false once every tile has been
// claimed.  Per-sample results never depend on which warp runs a sample.
struct WarpQueue {
    Tile cur{};
    int used = 0;
    bool dry = false;

    __device__ __forceinline__ bool take(unsigned need, const WorkDev &w, uint32_t tile_size,
                                         double model_thr, uint64_t &pidx, uint64_t &oidx,
                                         uint64_t &kidx, double &thr)
    {
        const unsigned lane = threadIdx.x & 31u;
        bool mine = false;
        while (need && !dry) {
            if (used >= cur.count) {
                cur = claim_tile(w, tile_size, model_thr);
                used = 0;
                if (!cur.ok) {
                    dry = true;
                    break;
                }
            }
            const unsigned rank = __popc(need & lanemask_lt());
            const bool got = ((need >> lane) & 1u) && (int)rank < cur.count - used;
            if (got) {
                mine = true;
                pidx = cur.p0 + used + rank;
                oidx = cur.o0 + used + rank;
                kidx = cur.k0 + used + rank;
                thr = cur.thr;
            }
            const unsigned taken = __ballot_sync(kFull, got);
            used += __popc(taken);
            need &= ~taken;
        }
        return mine;
    }
};

// Philox-4x64-10 (Salmon, Moraes, Dror, Shaw, SC 2011): the block of counter
// c under key (k0, k1), in place.  Used for the per-step perception readings
// of the TTC trigger, two readings per block: counter (parameter row,
// floor(k / 2), 0, 0), key (seed, kPercKey1) (see perc_halves).
constexpr uint64_t kPercKey1 = 0x5045524345505431ull;  // "PERCEPT1"
__device__ __forceinline__ void philox_block(uint64_t c[4], uint64_t k0, uint64_t k1)
{
    constexpr uint64_t kM0 = 0xD2E7470EE14C6C93ull, kM1 = 0xCA5A826395121157ull;
    constexpr uint64_t kW0 = 0x9E3779B97F4A7C15ull, kW1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t h0 = __umul64hi(kM0, c[0]), l0 = kM0 * c[0];
        const uint64_t h1 = __umul64hi(kM1, c[2]), l1 = kM1 * c[2];
        const uint64_t n0 = h1 ^ c[1] ^ k0, n2 = h0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = l1;
        c[2] = n2;
        c[3] = l0;
        k0 += kW0;
        k1 += kW1;
    }
}

// The four 32-bit words h_j of reading k (taken at step k) of parameter row
// `row`: the high halves of the block's words for even k, the low halves for
// odd k.  Uniforms u_j = h_j 2^-32; the reading is missing if u_4 is below
// the dropout probability.
__device__ __forceinline__ void perc_halves(uint64_t row, uint64_t k, uint64_t seed, uint32_t h[4])
{
    uint64_t c[4] = {row, k >> 1, 0, 0};
    philox_block(c, seed, kPercKey1);
    const int sh = (k & 1) ? 0 : 32;
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = (uint32_t)(c[j] >> sh);
}

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
//   bool init(M, X, P, O, p, o, k, thr) -- load parameter row p (output row o,
//                                perception key row k); true if it already ended
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
                                               const OutDev &O, const WorkDev &W, uint32_t tile_size)
{
    const unsigned lane = threadIdx.x & 31u;
    WarpQueue q;
    Lane L;
    uint64_t pidx = 0, oidx = 0, kidx = 0;
    double thr = M.ttc_thr;
    bool active = false;
    unsigned need = kFull;
    for (;;) {
        while (need) {
            const bool got = q.take(need, W, tile_size, M.ttc_thr, pidx, oidx, kidx, thr);
            bool ended = false;
            if ((need >> lane) & 1u) {
                active = got;
                if (active) ended = L.init(M, Xc, P, O, pidx, oidx, kidx, thr);
            }
            need = __ballot_sync(kFull, ended);
        }
        if (!__any_sync(kFull, active)) return;
        bool ended = false;
        if (active) ended = L.step(M, Xc, P, O, oidx);
        need = __ballot_sync(kFull, ended);
    }
}

}  // namespace aeb
