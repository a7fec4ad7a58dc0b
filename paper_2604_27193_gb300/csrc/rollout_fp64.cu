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
//
// The realised deceleration is the minimum of lines (D, mu g cos(theta) and
// the two axle lines, or D and the Eq. 5 cap), and a minimum returns one of
// its arguments unchanged.  So a lane keeps the line that is the strict
// minimum over an interval [dlo, dhi] of demand, shrunk at each end by a band
// of 1e-12 relative (far above the few-ulp rounding of a line value, so no
// rounding can change which line is smallest inside it); while a step's
// stage demands lie in the interval (the first stage has the smallest demand
// and the fourth the largest when dt / tau <= 2), each stage evaluates only
// that line, with the same expression as the full minimum, and the result
// is the same bits.  Other steps evaluate the full minimum and re-select.
#include <climits>

#include "rollout_common.cuh"

namespace aeb {
namespace {

__device__ __forceinline__ double dmin(double a, double b) { return (b < a) ? b : a; }

// The per-step comparisons as integer comparisons of the bit patterns (the
// binary64 pipe is the narrow one here): each gives the same truth value as
// the binary64 comparison it replaces.

// x <= 0.0 (false for a NaN).
__device__ __forceinline__ bool le_zero(double x)
{
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const unsigned mag = (unsigned)hi & 0x7fffffffu;
    const bool nan = mag > 0x7ff00000u || (mag == 0x7ff00000u && lo != 0);
    return !nan && (hi < 0 || (mag | (unsigned)lo) == 0u);
}

// x >= y for a finite y > 0 (false for a NaN x): non-negative doubles order
// as their bit patterns, and every negative x (-0 included) has the sign bit.
__device__ __forceinline__ bool ge_pos(double x, double y)
{
    const long long bx = __double_as_longlong(x), by = __double_as_longlong(y);
    return bx >= by && bx <= 0x7ff0000000000000ll;
}

// Order key of a non-NaN double: a signed integer that increases with the
// value and is equal for -0 and +0; okey(-x) = -okey(x).
__device__ __forceinline__ long long okey(double x)
{
    const long long b = __double_as_longlong(x);
    return b < 0 ? -(b & 0x7fffffffffffffffll) : b;
}

struct NoExtra {};

__device__ __forceinline__ double dinf() { return __longlong_as_double(0x7ff0000000000000ll); }

// Moving lead (extension): the lead brakes from lead_v0 at lead_decel until it
// stops (stop time lead_ts, stop position lead_xs), in closed form.
__device__ __forceinline__ double lead_pos(const ModelDev &M, double t)
{
    if (M.lead_decel > 0.0 && t >= M.lead_ts) return M.lead_xs;
    return t * (M.lead_v0 - (0.5 * M.lead_decel) * t);
}

__device__ __forceinline__ double lead_speed(const ModelDev &M, double t)
{
    if (M.lead_decel > 0.0 && t >= M.lead_ts) return 0.0;
    return M.lead_v0 - M.lead_decel * t;
}

template <int CAP, bool LEAD, bool TTC>
struct Lane64 {
    double x, v, a;
    double d0, gs, noise, k, it, thr;
    double mg, f0, f1, r0, r1, cap;
    double pa, pb;                // current line pa + pb D (piece 1, 2)
    long long klo, khi;           // its demand interval [dlo, dhi] as order keys
    uint64_t row;                 // perception key row (counter of the readings)
    int32_t n, n_b, n_delay;
    int piece;                    // 0: D, 1, 2: an axle line, 3: the constant cap; -1: none
    bool trig, lagged, ordered;

    // Select the line that is the strict minimum at demand D and the demand
    // interval, shrunk by the band, on which it stays so (piece -1 if D is
    // inside a band, lines are nearly parallel, or the stage demands are not
    // ordered).
    __device__ void select_piece(double D)
    {
        piece = -1;
        if (!ordered) return;
        double A[4], S[4];
        int nl;
        if (CAP == AEB_CAP_LUMPED) {
            A[0] = 0.0; S[0] = 1.0; A[1] = cap; S[1] = 0.0;
            nl = 2;
        } else {
            A[0] = 0.0; S[0] = 1.0; A[1] = f0; S[1] = f1; A[2] = r0; S[2] = r1; A[3] = mg; S[3] = 0.0;
            nl = 4;
        }
        double val[4];
        int cur = 0;
        for (int j = 0; j < nl; ++j) {
            val[j] = (j == 0) ? D : A[j] + S[j] * D;
            if (val[j] < val[cur]) cur = j;
        }
        double lo = -dinf(), hi = dinf();
        for (int j = 0; j < nl; ++j) {
            if (j == cur) continue;
            const double ds = S[cur] - S[j];
            if (!(fabs(ds) >= 1e-6) || !(val[j] > val[cur])) return;
            const double B = (A[j] - A[cur]) / ds;  // line j meets the current line
            const double band = 1e-12 * (1.0 + fabs(A[j]) + fabs(A[cur]) + fabs(B)) / fabs(ds);
            if (ds > 0.0) hi = fmin(hi, B - band);  // line j is below beyond B
            else lo = fmax(lo, B + band);
        }
        if (!(lo <= D && D <= hi)) return;
        klo = okey(lo);
        khi = okey(hi);
        if (CAP == AEB_CAP_LUMPED) {
            piece = (cur == 0) ? 0 : 3;
        } else {
            piece = cur;
            pa = A[cur];
            pb = S[cur];
        }
    }

    // dv/dt on the current piece: the same value as `accel` for D in the
    // piece's interval.  `lines`: some lane of the warp is on an axle line.
    __device__ __forceinline__ double accel_piece(double vv, double aa, bool lines) const
    {
        const double D = -aa;
        const double c = (CAP == AEB_CAP_LUMPED) ? cap : mg;
        double r = (piece == 0) ? D : c;
        if (CAP != AEB_CAP_LUMPED && lines && (piece == 1 || piece == 2)) r = pa + pb * D;
        return ((-r) - (k * vv) * vv) - gs;
    }

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
                                         const OutDev &O, uint64_t pi, uint64_t i, uint64_t ki,
                                         double thr_job)
    {
        double f[AEB_NFIELDS];
        load_fields(P, pi, f);
        thr = thr_job;
        if (!sample_valid(f)) {
            const double nan = __longlong_as_double(0x7ff8000000000000ll);
            store_out(O, i, AEB_INVALID, nan, nan, nan, nan, 0, -1);
            return true;
        }
        row = ki;
        d0 = f[kD0];
        gs = f[kGs];
        noise = f[kNoise];
        k = ((M.rho * f[kCd]) * M.area) / (2.0 * f[kMass]);
        lagged = f[kTau] > 0.0;
        it = lagged ? 1.0 / f[kTau] : 0.0;
        ordered = !lagged || M.dt * it <= 2.0;
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
        select_piece(-a);
        return false;
    }

    __device__ __forceinline__ bool step(const ModelDev &M, const NoExtra &, const ParamsDev &,
                                         const OutDev &O, uint64_t i)
    {
        const double dt = M.dt, h2 = M.h2, h6 = M.h6;
        if (TTC && !trig) {
            double gap_meas, closing;
            if (M.lead_moving) {  // gap and closing speed to the moving lead
                const double t = (double)n * dt;
                gap_meas = ((d0 + lead_pos(M, t)) - x) + noise;
                closing = v - lead_speed(M, t);
            } else {
                gap_meas = (d0 - x) + noise;
                closing = v;
            }
            bool reading = true;
            if (M.perc) {  // the reading of step n + L describes step n
                uint32_t h[4];
                perc_halves(row, (uint64_t)((long long)n + M.perc_lat), M.perc_seed, h);
                const double s32 = 1.0 / 4294967296.0;  // 2^-32
                const double u1 = (double)h[0] * s32, u2 = (double)h[1] * s32;
                const double u3 = (double)h[2] * s32, u4 = (double)h[3] * s32;
                if (u4 < M.perc_drop) reading = false;
                else gap_meas = gap_meas + M.perc_sigma * (2.0 * (((u1 + u2) + u3) - 1.5));
            }
            if (reading && gap_meas <= thr * closing) {
                trig = true;
                long long nb = ((long long)n + M.perc_lat) + n_delay;
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
        // With dt / tau <= 2 the stage demands lie between the first and the
        // fourth (-a1 smallest when the command is a deceleration, so that
        // a - u >= 0 from the start, -a4 smallest otherwise): two tests for
        // the step.
        // (A piece exists only when dt / tau <= 2, where the lag is stable and
        // the stage actuator values are finite, so order keys compare them.)
        const bool dec = M.a_cmd <= 0.0;
        const long long kfirst = -okey(dec ? a1 : a4), klast = -okey(dec ? a4 : a1);
        const bool pw = piece >= 0 && kfirst >= klo && klast <= khi;
        const bool lines = __any_sync(__activemask(), pw && (piece == 1 || piece == 2));
        double kv1, kv2, kv3, kv4, v2, v3, v4;
        if (pw) {
            kv1 = accel_piece(v, a1, lines);
            v2 = v + h2 * kv1;
            kv2 = accel_piece(v2, a2, lines);
            v3 = v + h2 * kv2;
            kv3 = accel_piece(v3, a3, lines);
            v4 = v + dt * kv3;
            kv4 = accel_piece(v4, a4, lines);
        } else {
            kv1 = accel(v, a1);
            v2 = v + h2 * kv1;
            kv2 = accel(v2, a2);
            v3 = v + h2 * kv2;
            kv3 = accel(v3, a3);
            v4 = v + dt * kv3;
            kv4 = accel(v4, a4);
        }

        const double xn = x + h6 * (((v + 2.0 * v2) + 2.0 * v3) + v4);
        const double vn = v + h6 * (((kv1 + 2.0 * kv2) + 2.0 * kv3) + kv4);
        const double an = lagged ? a + h6 * (((ka1 + 2.0 * ka2) + 2.0 * ka3) + ka4) : u;

        if (LEAD && M.lead_moving) {
            const double t0 = (double)n * dt, t1 = (double)(n + 1) * dt;
            const double g1 = (d0 + lead_pos(M, t1)) - xn;
            if (g1 <= 0.0) {
                const double g0 = (d0 + lead_pos(M, t0)) - x;
                const double c0 = v - lead_speed(M, t0), c1 = vn - lead_speed(M, t1);
                const double s = g0 / (g0 - g1);
                store_out(O, i, AEB_CONTACT, xn, x + s * (xn - x), c0 + s * (c1 - c0),
                          ((double)n + s) * dt, n + 1, onset());
                return true;
            }
        } else if (LEAD && ge_pos(xn, d0)) {  // d0 > 0 and finite here
            const double s = (d0 - x) / (xn - x);
            store_out(O, i, AEB_CONTACT, xn, d0, v + s * (vn - v), ((double)n + s) * dt, n + 1,
                      onset());
            return true;
        }
        if (le_zero(vn)) {
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
        if (!pw) select_piece(-a);
        return false;
    }
};

#ifndef AEB_FP64_MIN_BLOCKS
#define AEB_FP64_MIN_BLOCKS 1  // resident blocks per SM the register budget must allow
#endif

template <int CAP, bool LEAD, bool TTC>
__global__ void __launch_bounds__(128, AEB_FP64_MIN_BLOCKS)
k_rollout_fp64(ModelDev M, ParamsDev P, OutDev O, WorkDev W)
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
