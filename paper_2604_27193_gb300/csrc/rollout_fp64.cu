// rollout_fp64.cu -- binary64 rollout kernel, bit-identical to the plain
// definition of the method.
//
// Build: -fmad=false, so no multiply and add pair is ever fused; every
// expression below is evaluated in the order written, with IEEE round-to-
// nearest division.  The per-sample constants, the RK4 stages (Sec. IV-D,
// Eq. 7-9), the realised deceleration (Eq. 4-5 / per-axle caps), the command
// schedule, the termination tests (Sec. V-D) and the refinement are written
// in the same operation order as the binary64 definition, so each output is
// the same bits (Sec. V-D: same samples, same integrator, same precision,
// same termination, no fused or approximate operations).
#include <climits>

#include "rollout_common.cuh"

namespace aeb {
namespace {

__device__ __forceinline__ double dmin(double a, double b) { return (b < a) ? b : a; }

struct NoExtra {};

template <int CAP, bool LEAD, bool TTC>
struct Lane64 {
    double x, v, a;
    double d0, gs, noise, k, it, thr;
    double mg, f0, f1, r0, r1, cap;
    int32_t n, n_b, n_delay;
    bool trig, lagged;

    // Realised deceleration r for demand D = -a (Eq. 5 as printed, or the
    // per-axle fixed point min(min(D, mu gc), min(f0 + f1 D, r0 + r1 D))),
    // then dv/dt = -r - k v^2 - g sin(theta) (Eq. 4).
    __device__ __forceinline__ double accel(double vv, double aa) const
    {
        double D = -aa;
        double r;
        if (CAP == AEB_CAP_LUMPED) {
            r = dmin(D, cap);
        } else {
            double lf = f0 + f1 * D;
            double lr = r0 + r1 * D;
            r = dmin(dmin(D, mg), dmin(lf, lr));
        }
        return ((-r) - (k * vv) * vv) - gs;
    }

    __device__ __forceinline__ int32_t onset() const
    {
        return TTC ? (trig ? n_b : -1) : n_delay;
    }

    __device__ __forceinline__ bool init(const ModelDev &M, const NoExtra &, const ParamsDev &P,
                                         const OutDev &O, uint64_t pi, uint64_t i, double thr_job)
    {
        double f[AEB_NFIELDS];
        load_fields(P, pi, f);
        thr = thr_job;
        if (!sample_valid(f)) {
            const double nan = __longlong_as_double(0x7ff8000000000000ll);
            store_out(O, i, AEB_INVALID, nan, nan, nan, nan, 0, -1);
            return true;
        }
        d0 = f[kD0];
        gs = f[kGs];
        noise = f[kNoise];
        k = ((M.rho * f[kCd]) * M.area) / (2.0 * f[kMass]);
        lagged = f[kTau] > 0.0;
        it = lagged ? 1.0 / f[kTau] : 0.0;
        const double mu = f[kMu], gc = f[kGc];
        const double mh = mu * M.hl;
        if (CAP == AEB_CAP_LUMPED) {
            cap = (mu * M.g) / (1.0 + mh);
        } else {
            mg = mu * gc;
            f0 = (mg * M.phi_f) / (1.0 - mh);
            f1 = (1.0 - M.beta) / (1.0 - mh);
            r0 = (mg * (1.0 - M.phi_f)) / (1.0 + mh);
            r1 = M.beta / (1.0 + mh);
        }
        n_delay = steps_to_reach_dev(f[kTdelay], M.dt);
        trig = !TTC;
        n_b = n_delay;
        const int32_t on = TTC ? -1 : n_delay;
        if (LEAD && d0 <= 0.0) {
            store_out(O, i, AEB_CONTACT, 0.0, 0.0, f[kV0], 0.0, 0, on);
            return true;
        }
        if (f[kV0] <= 0.0) {
            store_out(O, i, AEB_STOP, 0.0, 0.0, 0.0, 0.0, 0, on);
            return true;
        }
        if (M.n_max == 0) {
            store_out(O, i, AEB_HORIZON, 0.0, 0.0, 0.0, 0.0, 0, on);
            return true;
        }
        x = 0.0;
        v = f[kV0];
        a = 0.0;
        n = 0;
        return false;
    }

    __device__ __forceinline__ bool step(const ModelDev &M, const NoExtra &, const ParamsDev &,
                                         const OutDev &O, uint64_t i)
    {
        const double dt = M.dt, h2 = M.h2, h6 = M.h6;
        if (TTC && !trig) {
            double gap_meas = (d0 - x) + noise;
            if (gap_meas <= thr * v) {
                trig = true;
                long long nb = (long long)n + n_delay;
                n_b = nb > INT_MAX ? INT_MAX : (int32_t)nb;
            }
        }
        const double u = (trig && n >= n_b) ? M.a_cmd : 0.0;

        double a1, a2, a3, a4, ka1 = 0.0, ka2 = 0.0, ka3 = 0.0, ka4 = 0.0;
        if (lagged) {
            a1 = a;
            ka1 = (u - a1) * it;
            a2 = a + h2 * ka1;
            ka2 = (u - a2) * it;
            a3 = a + h2 * ka2;
            ka3 = (u - a3) * it;
            a4 = a + dt * ka3;
            ka4 = (u - a4) * it;
        } else {
            a1 = a2 = a3 = a4 = u;
        }
        const double kv1 = accel(v, a1);
        const double v2 = v + h2 * kv1;
        const double kv2 = accel(v2, a2);
        const double v3 = v + h2 * kv2;
        const double kv3 = accel(v3, a3);
        const double v4 = v + dt * kv3;
        const double kv4 = accel(v4, a4);

        const double xn = x + h6 * (((v + 2.0 * v2) + 2.0 * v3) + v4);
        const double vn = v + h6 * (((kv1 + 2.0 * kv2) + 2.0 * kv3) + kv4);
        const double an = lagged ? a + h6 * (((ka1 + 2.0 * ka2) + 2.0 * ka3) + ka4) : u;

        if (LEAD && xn >= d0) {
            const double s = (d0 - x) / (xn - x);
            store_out(O, i, AEB_CONTACT, xn, d0, v + s * (vn - v), ((double)n + s) * dt, n + 1,
                      onset());
            return true;
        }
        if (vn <= 0.0) {
            const double s = v / (v - vn);
            store_out(O, i, AEB_STOP, xn, x + s * (xn - x), 0.0, ((double)n + s) * dt, n + 1,
                      onset());
            return true;
        }
        if (n + 1 >= M.n_max) {
            store_out(O, i, AEB_HORIZON, xn, xn, 0.0, (double)(n + 1) * dt, n + 1, onset());
            return true;
        }
        x = xn;
        v = vn;
        a = an;
        n = n + 1;
        return false;
    }
};

template <int CAP, bool LEAD, bool TTC>
__global__ void __launch_bounds__(128) k_rollout_fp64(ModelDev M, ParamsDev P, OutDev O, WorkDev W)
{
    rollout_driver<Lane64<CAP, LEAD, TTC>>(M, NoExtra{}, P, O, W, W.tile);
}

template <int CAP, bool LEAD, bool TTC>
cudaError_t launch_t(const ModelDev &m, const ParamsDev &p, const OutDev &o, const WorkDev &w,
                     const LaunchCfg &cfg, cudaStream_t s)
{
    auto kern = k_rollout_fp64<CAP, LEAD, TTC>;
    int dev = 0, sms = 0, per_sm = cfg.blocks_per_sm;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm <= 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    const uint64_t tiles = tiles_of(w, w.tile);
    uint64_t blocks = (uint64_t)sms * per_sm;
    uint64_t need_blocks = (tiles + 3) / 4;  // one tile per warp at least
    if (need_blocks < blocks) blocks = need_blocks;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, 128, 0, s>>>(m, p, o, w);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rollout_fp64(const ModelDev &m, const ParamsDev &p, const OutDev &o,
                                const WorkDev &w, const LaunchCfg &cfg, cudaStream_t s)
{
    const bool lead = m.lead != 0, ttc = m.trigger == AEB_TRIGGER_TTC;
    if (m.cap_mode == AEB_CAP_LUMPED) {
        if (lead) return ttc ? launch_t<AEB_CAP_LUMPED, true, true>(m, p, o, w, cfg, s)
                             : launch_t<AEB_CAP_LUMPED, true, false>(m, p, o, w, cfg, s);
        return ttc ? launch_t<AEB_CAP_LUMPED, false, true>(m, p, o, w, cfg, s)
                   : launch_t<AEB_CAP_LUMPED, false, false>(m, p, o, w, cfg, s);
    }
    if (lead) return ttc ? launch_t<AEB_CAP_PER_AXLE, true, true>(m, p, o, w, cfg, s)
                         : launch_t<AEB_CAP_PER_AXLE, true, false>(m, p, o, w, cfg, s);
    return ttc ? launch_t<AEB_CAP_PER_AXLE, false, true>(m, p, o, w, cfg, s)
               : launch_t<AEB_CAP_PER_AXLE, false, false>(m, p, o, w, cfg, s);
}

}  // namespace aeb
