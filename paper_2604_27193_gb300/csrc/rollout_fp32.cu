// rollout_fp32.cu -- binary32 rollout kernel with compensated state.
//
// The RK4 stages of Eq. 7-9 (Sec. IV-D) run in binary32 with fused
// multiply-add, in scaled units: the lane carries w = s v with s = sqrt(k)
// (k = rho C_d A / (2 m)), so the drag term k v^2 of a stage is w^2 and a
// stage costs one FMA for drag plus one for the actuator term, and the gap
// G = sigma (d0 - x) with sigma = s / h6 (h6 the binary32 step factor of the
// speed update), so the position increment of a step is the plain weighted
// sum of the stage speeds, with no multiply.  (s is rounded to binary32, so
// the drag coefficient in effect is s^2, within 2e-7 relative of k.)
// Speed and gap are carried as
// unevaluated double-float pairs (hi + lo), so 1e4-1e5 increments of 1e-3-1e-4
// relative size do not lose the ~1e-7 relative precision of a binary32 stage.
// Within a window of steps the high words stay fixed and every increment is
// added to the low word; the stages start from v1 = vh + vl, so they see the
// current speed without bias, and a slow car's step, far below half an ulp of
// the gap, still counts.  At the end of each window Fast2Sum folds the low
// words back (|lo| <= ulp(hi)/2 again).  Contact is g <= 0 on the pair; the
// TTC margin (g + noise) - thr v is formed with the exact error of thr v.
//
// Actuator (Eq. 6).  The lag is linear with the command u held over a step, so
// the lane carries e = a - u: RK4's stage values are u + p_j e with p1 = 1,
// p2 = 1 - z/2, p3 = 1 - z/2 + z^2/4, p4 = 1 - z + z^2/2 - z^3/4 (z = dt/tau),
// and one step maps e to e - mP e with mP = z - z^2/2 + z^3/6 - z^4/24: the
// four RK4 stages of Eq. 6, written so that the decay keeps binary32 relative
// precision (a binary32 `a` would stall ~ulp(a)/(2z) short of the command).
// tau = 0 (instantaneous actuator) is p_j = 0, mP = 1.
//
// Realised deceleration (Eq. 4-5 / per-axle caps).  r(D) is the minimum of the
// lines D, f0 + f1 D, r0 + r1 D and mu g cos(theta) (Eq. 5 as printed: D and
// mu g / (1 + mu h/L)).  After brake onset the demand D = -a only grows, so the
// lane keeps the line that is the minimum at the step's smallest demand and the
// threshold on e beyond which the step's largest demand would pass the next
// breakpoint.  Inside a piece every stage costs one FMA:
//     r_j + g sin(theta) = C + e a_j,  a_j = -slope p_j,
//     C = intercept - slope u + g sin(theta).
// A step that crosses a breakpoint evaluates the full minimum for its four
// stages, then moves to the next piece.
//
// Binary64 runs at 1/64 of the binary32 rate on GB300, so it is kept out of the
// step loop and done at full SIMT width: when a warp claims a tile of
// samples, all 32 lanes prepare the tile's binary32 constants together into
// shared memory (brake-onset step by the binary64 rule, hi/lo splits of the
// scaled v0 and d0, scaled step factors, cap coefficients, actuator
// multipliers, the scaled TTC threshold and range noise).  Lanes whose rollout
// ends refill from that tile (the whole warp copies their records' rarely read
// part into their shared-memory columns).  The binary64 refinement of the last step (linear
// stop/contact interpolation from the hi + lo pairs) is also batched: an ending
// lane queues its terminal state in the warp's shared slab, and the warp refines
// 32 queued rollouts at once.
//
// Steps run in windows of up to K = 32 with no test in between.  A lane's
// window ends before its next event (brake onset, the last step before the
// horizon, a step that crosses a breakpoint of r(D), and before a TTC trigger
// the next step at which the trigger could fire); lanes of a warp with
// shorter windows run the same window code masked, so a lane close to an event
// does not hold up the others.  Brake onset is a change of state between two
// steps (new command, new piece); only the breakpoint-crossing step and the
// last step take a slow path that evaluates the full minimum per stage.
#include <climits>
#include <cmath>

#include "rollout_common.cuh"

namespace aeb {
namespace {

constexpr int kTileDefault = 32;  // samples per warp tile unless configured
constexpr int kTileMax = 256;
constexpr int kWarps = 4;      // warps per block
constexpr int kThreads = 32 * kWarps;
#ifndef AEB_FP32_WINDOW
#define AEB_FP32_WINDOW 32     // steps a lane runs without termination tests
#endif
#ifndef AEB_FP32_MIN_BLOCKS
#define AEB_FP32_MIN_BLOCKS 6  // resident blocks per SM the register budget must allow
#endif

// A prepared per-sample record in the warp's tile, sample-major: the fields
// the lane that takes the sample loads into registers (R_*), then the block it
// keeps in its shared-memory column (C_*, copied by the whole warp when lanes
// refill).  Integer fields are stored as their bits.  The TTC fields exist only
// in the TTC-trigger kernel; -s dt = 2 (-s dt/2) exactly, p4 = -np4, np1 = -1
// when tau > 0 (else 0) and (1 - mP)^(K-1) are derived where needed.
enum { R_W0H, R_W0L, R_G0H, R_G0L, R_NH2S, R_NH6S, R_NMP, R_KIND, R_C0 };
enum {
    C_NDELAY, C_GS, C_S, C_SIGMA, C_F0, C_F1, C_R0, C_R1, C_MG, C_NP2, C_NP3, C_NP4,
    C_NBASE,                               // fields of every kernel
    C_NZ = C_NBASE, C_THRH, C_THRL, C_NTTC  // TTC trigger only
};
template <bool TTC>
__host__ __device__ constexpr int copy_fields() { return TTC ? C_NTTC : C_NBASE; }
// Words per record: odd, so that 32 lanes reading one field of 32 records, or
// one lane's record read by 32 lanes, hit 32 different banks.
template <bool TTC>
__host__ __device__ constexpr int rec_stride() { return (R_C0 + copy_fields<TTC>()) | 1; }
enum { K_RUN = 0, K_INVALID, K_CONTACT0, K_STOP0, K_HORIZON0 };

// The lead vehicle, a template parameter of the kernel (so that a stationary
// lead pays nothing for the moving one).
enum { kNoLead = 0, kLeadStationary = 1, kLeadMoving = 2 };

struct ModelF32 {
    float acmd;
    // binary32 copies of the constants the tile preparation forms binary32
    // per-sample values from
    float rho, area, hl, g, phi_f, beta;
    // moving lead: step, initial speed, deceleration, half of it, stop time,
    // stop position (binary32 copies of the model's values)
    float dt, lv0, lb, lhb, lts, lxs;
    float idt;  // 1 / dt (first guess of the onset step)
    // per-step perception of the TTC trigger (see the model): noise scale,
    // dropout threshold on a reading's h_4 (ceil(perc_drop 2^32): h_4 below it
    // is exactly u_4 < perc_drop), latency in steps, stream key, any of them set
    float psig;
    uint64_t pdrop_h;
    uint64_t pseed;
    int plat, perc;
};

__device__ __forceinline__ float finf() { return __int_as_float(0x7f800000); }

static_assert(AEB_FP32_WINDOW >= 2 && AEB_FP32_WINDOW <= 32,
              "window lengths are found from five binary digits (<= 31 steps)");

// Relative margin on the actuator threshold of a window: covers the rounding
// of K - 1 binary32 decays of e and of the power and quotient that form the
// threshold.
constexpr float kMargin = 1.00001f;

// Before its TTC trigger a lane tests the trigger only at steps where it could
// fire: one test bounds how fast the trigger margin can fall over up to
// kTtcSpan steps (speed bound over the span, see ttc_check) and sets the step
// of the next test.
constexpr int kTtcSpan = 512;

// q^P by repeated squaring (P < 32, a compile-time constant).
template <int P>
__device__ __forceinline__ float powi(float q)
{
    float r = 1.0f, b = q;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        if ((P >> i) & 1) r *= b;
        if ((P >> (i + 1)) != 0) b *= b;
    }
    return r;
}

// Smallest n >= 0 with (double)n * dt >= t (clamped to 2^31 - 1), the rule of
// steps_to_reach_dev, from a binary32 first guess t * (1/dt) instead of a
// binary64 division (slow here); the adjustment loops make the result exact
// whatever the guess.
__device__ __forceinline__ int32_t steps_to_reach_f32(double t, double dt, float idt)
{
    if (!(t > 0.0)) return 0;
    const float qf = ceilf(__double2float_rn(t) * idt);
    if (!(qf < 1.0e9f)) return steps_to_reach_dev(t, dt);
    long long n = (long long)qf;
    while (n > 0 && (double)(n - 1) * dt >= t) --n;
    while ((double)n * dt < t) ++n;
    return (int32_t)n;
}

// Prepare samples [start, start + cnt) of a tile (TTC threshold thr) into the
// warp's records (sample-major, rec_stride words each).  Kept out of line: it
// runs once per tile, and its binary64 code inlined into the kernel cost the
// step loop ~3 % (measured on the single-scenario workload).
template <int LEAD, bool TTC>
__device__ __noinline__ void prep_tile(const ModelDev &M, const ModelF32 &F, const ParamsDev &P,
                                          uint64_t start, int cnt, double thr, float *tf)
{
    constexpr int RS = rec_stride<TTC>();
    for (int j = threadIdx.x & 31; j < cnt; j += 32) {
        const uint64_t i = start + j;
        float *rc = tf + j * RS;
        float *cp = rc + R_C0;
        double f[AEB_NFIELDS];
        load_fields(P, i, f);
        int kind = K_RUN, nd = 0;
        if (!sample_valid(f)) {
            kind = K_INVALID;
        } else {
            nd = steps_to_reach_f32(f[kTdelay], M.dt, F.idt);
            if (LEAD && f[kD0] <= 0.0) kind = K_CONTACT0;
            else if (f[kV0] <= 0.0) kind = K_STOP0;
            else if (M.n_max == 0) kind = K_HORIZON0;
        }
        cp[C_NDELAY] = __int_as_float(nd);
        rc[R_KIND] = __int_as_float(kind);
        if (kind != K_RUN) continue;
        // speed scale s = sqrt(k), bounded below so that a drag-free sample
        // keeps its scaled state in the normal binary32 range.  The constants
        // that end up in binary32 (k, the cap lines, the actuator multipliers)
        // are formed in binary32 (a few ulps; binary64 division is slow here);
        // the scales that tie the pairs to metres (sigma, w0, g0) stay binary64.
        const float k32 = ((F.rho * __double2float_rn(f[kCd])) * F.area) /
                          (2.0f * __double2float_rn(f[kMass]));
        const float sc = fmaxf(sqrtf(k32), 1e-18f);
        const double sd = (double)sc;
        const float nh6s = __double2float_rn(-(sd * M.h6));
        // gap scale sigma = s^2 / (-nh6s) = s / h6: 1 / (-nh6s) from the
        // binary32 reciprocal and one binary64 Newton step (relative error
        // ~4e-15, where a binary64 division would be slow)
        const double x6 = -(double)nh6s;
        const double r0 = (double)__frcp_rn(-nh6s);
        const double r6 = fma(r0, fma(-x6, r0, 1.0), r0);
        const double sigma = (sd * sd) * r6;
        const double w0 = sd * f[kV0], g0 = sigma * f[kD0];
        const float w0h = __double2float_rn(w0), g0h = __double2float_rn(g0);
        rc[R_W0H] = w0h;
        rc[R_W0L] = __double2float_rn(w0 - (double)w0h);
        rc[R_G0H] = g0h;
        rc[R_G0L] = __double2float_rn(g0 - (double)g0h);
        rc[R_NH2S] = __double2float_rn(-(sd * M.h2));
        rc[R_NH6S] = nh6s;
        cp[C_GS] = __double2float_rn(f[kGs]);
        cp[C_S] = sc;
        cp[C_SIGMA] = __double2float_rn(sigma);
        const float mu = __double2float_rn(f[kMu]), mh = mu * F.hl;
        if (M.cap_mode == AEB_CAP_LUMPED) {
            cp[C_F0] = finf();
            cp[C_F1] = 0.0f;
            cp[C_R0] = finf();
            cp[C_R1] = 0.0f;
            cp[C_MG] = (mu * F.g) / (1.0f + mh);
        } else {
            const float mg = mu * __double2float_rn(f[kGc]);
            const float im = 1.0f / (1.0f - mh), ip = 1.0f / (1.0f + mh);
            cp[C_F0] = (mg * F.phi_f) * im;
            cp[C_F1] = (1.0f - F.beta) * im;
            cp[C_R0] = (mg * (1.0f - F.phi_f)) * ip;
            cp[C_R1] = F.beta * ip;
            cp[C_MG] = mg;
        }
        float nmp = -1.0f;
        if (f[kTau] > 0.0) {
            const float z = F.dt / __double2float_rn(f[kTau]);
            cp[C_NP2] = -(1.0f - 0.5f * z);
            cp[C_NP3] = -(1.0f - 0.5f * z + 0.25f * z * z);
            cp[C_NP4] = -(1.0f - z + 0.5f * z * z - 0.25f * z * z * z);
            nmp = -(z * (1.0f + z * (-0.5f + z * (1.0f / 6.0f - z / 24.0f))));
        } else {
            cp[C_NP2] = 0.0f;
            cp[C_NP3] = 0.0f;
            cp[C_NP4] = 0.0f;
        }
        rc[R_NMP] = nmp;
        if (TTC) {  // (g + noise) - thr v scaled by sigma: G + sigma noise - (sigma thr / s) w
            const double ts = thr * (sd * r6);  // sigma / s
            const float tsh = __double2float_rn(ts);
            cp[C_NZ] = __double2float_rn(sigma * f[kNoise]);
            cp[C_THRH] = tsh;
            cp[C_THRL] = __double2float_rn(ts - (double)tsh);
        }
    }
}

// Per-lane values read only on rare paths (piece changes, slow steps, the TTC
// test, records) live in a column of the warp's shared slab, to keep the step
// loop's register budget small: the lane's own fields, its rows, then the
// record block C_* (both written by the whole warp at refill).  Lane-major
// with an odd stride, so that 32 lanes reading one field, or 32 lanes writing
// one lane's column, hit 32 different banks.
enum {
    L_U, L_ETHK, L_NB, L_NCHK, L_NP1, L_QF,                       // the lane's (NCHK: TTC)
    L_PIDXLO, L_PIDXHI, L_IDXLO, L_IDXHI, L_KIDXLO, L_KIDXHI,     // rows (two words each)
    L_C0,                                                         // the record block
    L_NDELAY = L_C0 + C_NDELAY, L_GS = L_C0 + C_GS, L_S = L_C0 + C_S,
    L_SIGMA = L_C0 + C_SIGMA, L_F0 = L_C0 + C_F0, L_F1 = L_C0 + C_F1, L_R0 = L_C0 + C_R0,
    L_R1 = L_C0 + C_R1, L_MG = L_C0 + C_MG, L_NP2 = L_C0 + C_NP2, L_NP3 = L_C0 + C_NP3,
    L_NP4 = L_C0 + C_NP4, L_NZ = L_C0 + C_NZ, L_THRH = L_C0 + C_THRH, L_THRL = L_C0 + C_THRL
};
template <bool TTC>
__host__ __device__ constexpr int cold_stride() { return (L_C0 + copy_fields<TTC>()) | 1; }
static_assert(L_C0 - L_PIDXLO + C_NTTC <= 32, "a column's rows and record block fit one warp");

template <int LEAD, bool TTC, bool PERC>
struct Lane32 {
    float vh, vl, gh, gl, e;      // state: scaled speed w = s v, scaled gap G = sigma (d0 - x),
                                  // actuator deviation a - u
    float C, eth;                 // current piece of r(D), its threshold on e
    float nh2s, ndts, nh6s;       // scaled step factors -s dt/2, -s dt, -s dt/6
    float a1, a2, a3, a4;         // slope of the piece times -p_j
    float nmP;
    int32_t n, ev;                // step, next slow step
    bool trig;
    float *cold;                  // this lane's column: cold[field]

    __device__ __forceinline__ float cf(int f) const { return cold[f]; }
    __device__ __forceinline__ void set_cf(int f, float x) { cold[f] = x; }
    __device__ __forceinline__ int ci(int f) const { return __float_as_int(cold[f]); }
    __device__ __forceinline__ void set_ci(int f, int x) { cold[f] = __int_as_float(x); }
    __device__ __forceinline__ float np1() const { return cf(L_NP1); }  // -p1
    __device__ __forceinline__ uint64_t pidx() const
    {
        return (uint64_t)(uint32_t)ci(L_PIDXLO) | ((uint64_t)(uint32_t)ci(L_PIDXHI) << 32);
    }

    // Select the line of r(D) that is the minimum at demand D (ties: the
    // flatter line, which stays the minimum to the right), its next breakpoint
    // B, and the threshold on e beyond which a step's largest demand
    // D4 = -(u + p4 e) exceeds B.
    __device__ __forceinline__ void set_piece(float D)
    {
        const float u = cf(L_U), p4 = -cf(L_NP4);
        const float a_[4] = {0.0f, cf(L_F0), cf(L_R0), cf(L_MG)};
        const float b_[4] = {1.0f, cf(L_F1), cf(L_R1), 0.0f};
        float ab = 0.0f, bb = 1.0f, bv = D;
#pragma unroll
        for (int j = 1; j < 4; ++j) {
            const float vj = fmaf(b_[j], D, a_[j]);
            if (vj < bv || (vj == bv && b_[j] < bb)) {
                bv = vj;
                ab = a_[j];
                bb = b_[j];
            }
        }
        // The breakpoint and the thresholds below only decide when a step
        // must take the full minimum, so they use the fast binary32 quotient
        // (error ~2 ulp, far inside the 1e-5 margin on e).
        float B = finf();
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (b_[j] < bb && a_[j] < finf()) B = fminf(B, __fdividef(a_[j] - ab, bb - b_[j]));
        a1 = bb * np1();
        a2 = bb * cf(L_NP2);
        a3 = bb * cf(L_NP3);
        a4 = bb * cf(L_NP4);
        C = (ab - bb * u) + cf(L_GS);
        eth = (p4 > 0.0f && B < finf()) ? __fdividef(-u - B, p4) : -finf();
        // e decays by (1 - mP) per step; a window of K steps stays inside the
        // piece if its last step does: e (1 - mP)^(K-1) >= eth (with margin)
        float ethK = eth;
        if (eth > 0.0f) {
            const float f = cf(L_QF);  // (1 - mP)^(K-1), taken once per sample
            ethK = (f > 0.0f) ? __fdividef(eth, f) * kMargin : finf();
        }
        set_cf(L_ETHK, ethK);
    }

    // r + g sin(theta) by the full minimum (slow steps)
    __device__ __forceinline__ float rg_full(float np) const
    {
        const float D = -fmaf(-np, e, cf(L_U));
        const float r = fminf(fminf(D, cf(L_MG)),
                              fminf(fmaf(cf(L_F1), D, cf(L_F0)), fmaf(cf(L_R1), D, cf(L_R0))));
        return r + cf(L_GS);
    }

    __device__ __forceinline__ int32_t onset() const
    {
        return TTC ? (trig ? ci(L_NB) : -1) : ci(L_NDELAY);
    }

    // Whether the next step must take the slow path: it crosses a breakpoint
    // of r(D) (the actuator deviation has reached the piece's threshold) or it
    // is the horizon's last step (a pending onset is a state change instead).
    __device__ __forceinline__ bool at_slow(int32_t n_last) const
    {
        return n >= n_last || e < eth;
    }

    // Next step that must take the slow path: the onset step (if still ahead,
    // possibly the current step) or the last step.
    __device__ __forceinline__ void next_event(int32_t n_last)
    {
        const int32_t n_b = ci(L_NB);
        ev = (trig && n_b >= n && n_b < n_last) ? n_b : n_last;
    }

    // One RK4 step inside the current piece of r(D) (one FMA per stage for r)
    // or, with FULL_MIN, with the full minimum per stage.  Within a window
    // the high words stay fixed and each step's increments are added to the
    // low words (`normalize` folds them in at the end of the window): the
    // stages start from v1 = vh + vl, so they see the current speed, and the
    // gap's low word collects position increments far below half an ulp of
    // the high word.  The gap scale sigma = s / h6 is built from the same
    // binary32 factor nh6s = -s h6 as the speed update, so distance and speed
    // advance with one step factor (independently rounded factors would scale
    // every stopping distance by their ratio, a systematic ~5e-8 relative
    // error), and the gap falls by the stage-speed sum v1 + 2 v2 + 2 v3 + v4,
    // formed as 6 v1 + s dt (q1 + q2 + q3) (the same sum in exact arithmetic,
    // one instruction fewer).  Returns the end-of-step low words and actuator
    // deviation.
    template <bool FULL_MIN>
    __device__ __forceinline__ void rk4_step(float &vl1, float &gl1, float &en) const
    {
        const float v1 = vh + vl;
        // the four actuator terms C + e a_j are independent of each other and
        // of the stage chain: two paired binary32 FMAs (per component the same
        // rounding as fmaf) cost two issue slots instead of four
        float2 X12, X34;
        if (FULL_MIN) {
            X12 = make_float2(rg_full(np1()), rg_full(cf(L_NP2)));
            X34 = make_float2(rg_full(cf(L_NP3)), rg_full(cf(L_NP4)));
        } else {
            const float2 ee = make_float2(e, e), cc = make_float2(C, C);
            X12 = __ffma2_rn(ee, make_float2(a1, a2), cc);
            X34 = __ffma2_rn(ee, make_float2(a3, a4), cc);
        }
        const float q1 = fmaf(v1, v1, X12.x);
        const float v2 = fmaf(nh2s, q1, v1);
        const float q2 = fmaf(v2, v2, X12.y);
        const float v3 = fmaf(nh2s, q2, v1);
        const float q3 = fmaf(v3, v3, X34.x);
        const float v4 = fmaf(ndts, q3, v1);
        const float q4 = fmaf(v4, v4, X34.y);
        // speed: q1 + 2 q2 + 2 q3 + q4; gap: the stage speeds sum to
        // v1 + 2 v2 + 2 v3 + v4 = 6 v1 + 2 (nh2s) (q1 + q2 + q3) (ndts = 2 nh2s)
        const float s23 = q2 + q3, s123 = s23 + q1;
        vl1 = fmaf(nh6s, fmaf(2.0f, s23, q1 + q4), vl);
        gl1 = fmaf(-ndts, s123, fmaf(-6.0f, v1, gl));
        en = fmaf(nmP, e, e);
    }

    // Fold the low words into the high words (Fast2Sum; the pairs stay exact).
    __device__ __forceinline__ void normalize()
    {
        const float sv = vh + vl;
        vl = vl - (sv - vh);
        vh = sv;
        const float sg = gh + gl;
        gl = gl - (sg - gh);
        gh = sg;
    }

    // Moving lead: the scaled distance sig x_L(m dt) the lead has covered by
    // the start of step m (sig: the lane's gap scale), and its scaled speed
    // sc v_L(m dt) (sc: the lane's speed scale), in binary32.
    static __device__ __forceinline__ float lead_gap(const ModelF32 &F, int32_t m, float sig)
    {
        const float t = (float)m * F.dt;
        const float x = (F.lb > 0.0f && t >= F.lts) ? F.lxs : t * fmaf(-F.lhb, t, F.lv0);
        return sig * x;
    }
    static __device__ __forceinline__ float lead_speed(const ModelF32 &F, int32_t m, float sc)
    {
        const float t = (float)m * F.dt;
        const float v = (F.lb > 0.0f && t >= F.lts) ? 0.0f : fmaf(-F.lb, t, F.lv0);
        return sc * v;
    }

    // Whether the gap (gh, gl1) at the end of step n has closed.
    __device__ __forceinline__ bool hits_lead(const ModelF32 &F, float gl1, float sig) const
    {
        if (!LEAD) return false;
        float g = gh + gl1;
        if (LEAD == kLeadMoving) g = g + lead_gap(F, n + 1, sig);
        return g <= 0.0f;
    }

    // Whether the state (vh, vl1), (gh, gl1) has stopped or reached the lead.
    __device__ __forceinline__ bool terminal(const ModelF32 &F, float vl1, float gl1,
                                             float sig) const
    {
        return hits_lead(F, gl1, sig) || vh + vl1 <= 0.0f;
    }

    __device__ __forceinline__ void commit(float vl1, float gl1, float en)
    {
        vl = vl1;
        gl = gl1;
        e = en;
        n = n + 1;
    }

    // A checked step inside the current piece; true if the rollout ended
    // (contact or stop) in this step, which is then not committed (its
    // end-of-step low words are returned).
    __device__ __forceinline__ bool step_fast(const ModelF32 &F, float &vl1, float &gl1,
                                              float sig)
    {
        float en;
        rk4_step<false>(vl1, gl1, en);
        const bool ended = terminal(F, vl1, gl1, sig);
        if (!ended) commit(vl1, gl1, en);
        return ended;
    }

    // An unchecked step inside the current piece (step counter not advanced).
    __device__ __forceinline__ void step_unchecked()
    {
        float vl1, gl1, en;
        rk4_step<false>(vl1, gl1, en);
        vl = vl1;
        gl = gl1;
        e = en;
    }

    // Whether the next K steps may run as one window with no event among
    // them (implies no onset and no slow step at this step).
    __device__ __forceinline__ bool full_window_ok(int tlen) const
    {
        return (!TTC || trig || tlen >= AEB_FP32_WINDOW) && n + AEB_FP32_WINDOW <= ev &&
               !(e < cf(L_ETHK));
    }

    // How many steps (1 .. K) may run as one window from here: none of them
    // a slow step, none a possible TTC trigger (tlen), and the piece of r(D)
    // valid for each (the actuator deviation e, which decays by the factor
    // q = 1 - mP per step, stays >= eth at the start of every step, with the
    // margin kMargin).
    __device__ __forceinline__ int window_len(int tlen) const
    {
        const int32_t room = ev - n;  // >= 1: a lane at its event takes the slow path
        int len = room < AEB_FP32_WINDOW ? (int)room : AEB_FP32_WINDOW;
        if (TTC && !trig && tlen < len) len = tlen;
        if (e < cf(L_ETHK)) {  // close to a breakpoint (eth > 0 here)
            // the largest k with e q^k >= m, from its binary digits: the
            // window runs steps 0 .. k, so the crossing step comes next
            const float q = 1.0f + nmP, m = eth * kMargin;
            int lb = 1;
            if (q > 0.0f && q < 1.0f) {
                const float q2 = q * q, q4 = q2 * q2, q8 = q4 * q4;
                float r = e;
                int k = 0;
                if (AEB_FP32_WINDOW > 16) {
                    const float q16 = q8 * q8;
                    if (r * q16 >= m) { r *= q16; k += 16; }
                }
                if (r * q8 >= m) { r *= q8; k += 8; }
                if (r * q4 >= m) { r *= q4; k += 4; }
                if (r * q2 >= m) { r *= q2; k += 2; }
                if (r * q >= m) k += 1;
                lb = k + 1;
            }
            len = len < lb ? len : lb;
        }
        return len;
    }

    // `len` fast steps (FULL: len = K) with no termination test in between.
    // Within a few milliseconds a stop leaves v <= 0 and a contact leaves
    // g <= 0 (a contact at near-zero speed turns into v <= 0), so the state
    // after the window shows whether the rollout ended inside it.  If so the
    // lane's state goes back to the window's start and the function returns
    // true: the warp queues the window and later replays it, one checked
    // step at a time, for 32 rollouts at once (`flush_batch`).  The replay
    // reproduces the same arithmetic (this file is compiled without FMA
    // contraction) and so finds the terminating step.  Lanes of a warp with
    // different lengths run the same window code, each masked off after its
    // own length (the short-window version is a rolled loop, to keep the
    // kernel's code small).
    template <bool FULL>
    __device__ __forceinline__ bool step_window(const ModelF32 &F, int len)
    {
        const float vh0 = vh, vl0 = vl, gh0 = gh, gl0 = gl, e0 = e;
        if (FULL) {
            len = AEB_FP32_WINDOW;
#pragma unroll
            for (int j = 0; j < AEB_FP32_WINDOW; ++j) step_unchecked();
        } else {
            // rolled (code size), two steps per trip, then the odd step
            int j = 0;
#pragma unroll 1
            for (; j + 2 <= len; j += 2) {
                step_unchecked();
                step_unchecked();
            }
            if (j < len) step_unchecked();
        }
        normalize();
        bool hit = vh <= 0.0f;
        if (LEAD == kLeadStationary) hit = hit || gh <= 0.0f;
        if (LEAD == kLeadMoving) hit = hit || gh + lead_gap(F, n + len, cf(L_SIGMA)) <= 0.0f;
        if (hit) {
            vh = vh0;
            vl = vl0;
            gh = gh0;
            gl = gl0;
            e = e0;
            return true;
        }
        n += len;
        return false;
    }

    // Brake onset (the command switches on at the start of step n_b): the
    // actuator deviation jumps by -a_cmd and the piece of r(D) is selected at
    // the step's first-stage demand; the step itself then runs as a fast step.
    __device__ __forceinline__ void onset_event(const ModelF32 &F, int32_t n_last)
    {
        set_cf(L_U, F.acmd);
        e = e - F.acmd;
        set_piece(-fmaf(-np1(), e, F.acmd));
        ev = n_last;
    }

    // A step crossing a breakpoint of r(D), or the last step before the
    // horizon (which may also be the onset step): full minimum for r, then
    // re-select the piece.
    __device__ __forceinline__ bool step_slow(const ModelF32 &F, int32_t n_last, float &vl1,
                                              float &gl1)
    {
        if (n == ci(L_NB)) {  // the command switches on at the start of this step
            set_cf(L_U, F.acmd);
            e = e - F.acmd;
        }
        float en;
        rk4_step<true>(vl1, gl1, en);
        const bool ended = terminal(F, vl1, gl1, cf(L_SIGMA)) || n >= n_last;
        if (!ended) {
            commit(vl1, gl1, en);
            normalize();
            set_piece(-fmaf(-np1(), e, cf(L_U)));
            next_event(n_last);
        }
        return ended;
    }

    // TTC trigger (while not yet triggered): (g + noise) - thr v <= 0, with the
    // exact rounding error of thr * vh; braking starts n_delay steps later.
    // Returns how many steps (1 .. kTtcSpan; whole windows from K up) may run
    // before the next test:
    // before the trigger the car coasts, the stage accelerations are
    // q = w^2 + C >= C, so over the span the scaled speed stays below
    // W = w + kTtcSpan s dt max(0, -C)
    // and the margin falls by at most 6 W + thr' s dt max(0, -C) per step
    // (the gap by the stage-speed sum, the speed term by the speed gain); the
    // first L - 1 steps after this one cannot trigger while (L - 1) times that
    // bound stays below the margin.  With a moving lead the margin is
    // (g + noise) - thr (v - v_L).
    // The trigger margin (g + noise) - thr v at the current state, scaled by
    // sigma, with the exact rounding error of thr * vh; a moving lead adds its
    // travel to the gap and takes its speed off the closing speed.
    __device__ __forceinline__ float ttc_margin(const ModelF32 &F) const
    {
        const float thr_h = cf(L_THRH);
        const float p = thr_h * vh;
        const float pe = fmaf(thr_h, vh, -p);
        const float hi = gh - p;
        const float lo = (gl + cf(L_NZ)) - (pe + fmaf(thr_h, vl, cf(L_THRL) * vh));
        float m = hi + lo;
        if (LEAD == kLeadMoving)
            m = m + fmaf(thr_h, lead_speed(F, n, cf(L_S)), lead_gap(F, n, cf(L_SIGMA)));
        return m;
    }

    // The noise of a reading with words h (perc_halves) in the margin's units
    // of a lane with gap scale sig, or +inf if the reading is missing: the
    // dropout decision is the exact integer form of u_4 < perc_drop, the
    // noise takes the top 24 bits of h_1 .. h_3.
    static __device__ __forceinline__ float reading_of(const ModelF32 &F, const uint32_t h[4],
                                                       float sig)
    {
        if ((uint64_t)h[3] < F.pdrop_h) return finf();
        const float s24 = 5.9604644775390625e-8f;  // 2^-24
        const float u1 = (float)(h[0] >> 8) * s24;
        const float u2 = (float)(h[1] >> 8) * s24;
        const float u3 = (float)(h[2] >> 8) * s24;
        return sig * (F.psig * (2.0f * (((u1 + u2) + u3) - 1.5f)));
    }

    // The reading of step k (taken at step k + L).
    static __device__ __forceinline__ float reading(const ModelF32 &F, uint64_t krow, int32_t k,
                                                    float sig)
    {
        uint32_t h[4];
        perc_halves(krow, (uint64_t)((long long)k + F.plat), F.pseed, h);
        return reading_of(F, h, sig);
    }

    // Readings 2b and 2b + 1 (one Philox block): ra, rb.
    static __device__ __forceinline__ void reading_pair(const ModelF32 &F, uint64_t krow,
                                                        uint64_t b, float sig, float &ra, float &rb)
    {
        uint64_t c[4] = {krow, b, 0, 0};
        philox_block(c, F.pseed, kPercKey1);
        uint32_t h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) h[j] = (uint32_t)(c[j] >> 32);
        ra = reading_of(F, h, sig);
#pragma unroll
        for (int j = 0; j < 4; ++j) h[j] = (uint32_t)c[j];
        rb = reading_of(F, h, sig);
    }

    __device__ __forceinline__ uint64_t krow() const
    {
        return (uint64_t)(uint32_t)ci(L_KIDXLO) | ((uint64_t)(uint32_t)ci(L_KIDXHI) << 32);
    }

    // The trigger fires at step k (its onset step n_b = k + L + n_delay); the
    // step stays in the test-step field, which is not read once triggered.
    __device__ __forceinline__ void fire(const ModelF32 &F, int32_t k, int32_t n_last)
    {
        trig = true;
        if (PERC) set_ci(L_NCHK, k);
        const long long nb = ((long long)k + F.plat) + ci(L_NDELAY);
        const int32_t n_b = nb > INT_MAX ? INT_MAX : (int32_t)nb;
        set_ci(L_NB, n_b);
        ev = (n_b < n_last) ? n_b : n_last;
    }

    // How many steps (1 .. kTtcSpan; whole windows from K up) may run before
    // the next trigger test, after the test of this step did not fire; 0 if
    // with per-step perception even this step's test cannot be ruled out by
    // the worst-case noise (the lane is in its noise band).
    // Before the trigger the car coasts, the stage accelerations are
    // q = w^2 + C >= C, so over the span the scaled speed stays below
    // W = w + kTtcSpan s dt max(0, -C)
    // and the margin falls by at most 6 W + thr' s dt max(0, -C) per step
    // (the gap by the stage-speed sum, the speed term by the speed gain); the
    // first L - 1 steps after this one cannot trigger while (L - 1) times that
    // bound stays below the margin.  With a moving lead the margin is
    // (g + noise) - thr (v - v_L).
    __device__ __forceinline__ int ttc_bound(const ModelF32 &F, float m) const
    {
        const float thr_h = cf(L_THRH);
        const float sdt = -ndts, acc = fmaxf(0.0f, -C);
        const float W = fmaf((float)kTtcSpan * sdt, acc, vh + vl);  // speed bound over the span
        // (a braking lead's speed term falls by thr' s dt b_L per step more;
        // its travel only widens the gap)
        const float d = fmaf(6.0f, W, thr_h * sdt * (acc + F.lb)) * 1.001f;
        // a reading's noise is at most 3 perc_sigma: only a margin beyond that
        // rules a trigger out whatever the readings of the skipped steps
        const float mw = PERC ? fmaf(-3.0f * F.psig, cf(L_SIGMA), m) : m;
        const float r = __fdividef(mw, d) * 0.999f;
        if (!(r > 0.0f)) return PERC ? 0 : 1;
        const int t = r >= (float)(kTtcSpan - 1) ? kTtcSpan : 1 + (int)r;
        // a span of whole windows (testing earlier is always safe), so that
        // far from the trigger the next test falls on a window boundary
        return t >= AEB_FP32_WINDOW ? t - t % AEB_FP32_WINDOW : t;
    }

    // TTC trigger test of this step (while not yet triggered): (g + noise) -
    // thr v <= 0 (with per-step perception: this step's reading, none if it is
    // missing); braking starts n_delay steps later.  Returns how many steps
    // (1 .. kTtcSpan) may run before the next test (K once triggered).
    __device__ __forceinline__ int ttc_check(const ModelF32 &F, int32_t n_last)
    {
        const float m = ttc_margin(F);
        const float pn = PERC ? reading(F, krow(), n, cf(L_SIGMA)) : 0.0f;
        if (m + pn <= 0.0f) {  // a missing reading (+inf) never fires
            fire(F, n, n_last);
            return AEB_FP32_WINDOW;
        }
        const int t = ttc_bound(F, m);
        return t > 0 ? t : 1;
    }

    // Per-step perception, the windows of a pass with lanes in their noise
    // band: `len` steps as step_window<false>; a band lane (state slot `st`)
    // also keeps the window's start (vh, gh, e at st[2K .. 2K + 2]) and, before
    // each step j, its low words gl (st[j]) and vl (st[K + j]), on which the
    // warp tests its trigger after the window (band_test).
    __device__ __forceinline__ bool step_window_st(const ModelF32 &F, int len, float *st)
    {
        const float vh0 = vh, vl0 = vl, gh0 = gh, gl0 = gl, e0 = e;
        if (st) {
            st[2 * AEB_FP32_WINDOW] = vh;
            st[2 * AEB_FP32_WINDOW + 1] = gh;
            st[2 * AEB_FP32_WINDOW + 2] = e;
        }
        int j = 0;
#pragma unroll 1
        for (; j + 2 <= len; j += 2) {
            if (st) {
                st[j] = gl;
                st[AEB_FP32_WINDOW + j] = vl;
            }
            step_unchecked();
            if (st) {
                st[j + 1] = gl;
                st[AEB_FP32_WINDOW + j + 1] = vl;
            }
            step_unchecked();
        }
        if (j < len) {
            if (st) {
                st[j] = gl;
                st[AEB_FP32_WINDOW + j] = vl;
            }
            step_unchecked();
        }
        normalize();
        bool hit = vh <= 0.0f;
        if (LEAD == kLeadStationary) hit = hit || gh <= 0.0f;
        if (LEAD == kLeadMoving) hit = hit || gh + lead_gap(F, n + len, cf(L_SIGMA)) <= 0.0f;
        if (hit) {
            vh = vh0;
            vl = vl0;
            gh = gh0;
            gl = gl0;
            e = e0;
            return true;
        }
        n += len;
        return false;
    }

    // The trigger margin of ttc_margin at a step of a window whose start had
    // the high words vh, gh, split into its window-constant part hk and the
    // scaled-threshold parts thr_h, c1 (the high words stay fixed in a window):
    // margin = (gl + hk) - fmaf(thr_h, vl, c1).
    __device__ __forceinline__ void band_consts(float &thr_h, float &c1, float &hk) const
    {
        thr_h = cf(L_THRH);
        const float p = thr_h * vh;
        const float pe = fmaf(thr_h, vh, -p);
        const float hi = gh - p;
        c1 = cf(L_THRL) * vh;
        hk = hi + (cf(L_NZ) - pe);
    }

    // Back to the start of the band window just run (its state slot st).
    __device__ __forceinline__ void band_rewind(const float *st, int32_t n0)
    {
        vh = st[2 * AEB_FP32_WINDOW];
        gh = st[2 * AEB_FP32_WINDOW + 1];
        e = st[2 * AEB_FP32_WINDOW + 2];
        gl = st[0];
        vl = st[AEB_FP32_WINDOW];
        n = n0;
    }

    // Take the prepared record rc (parameter row pi, output row i); true if
    // the sample ended at once (stored).  The record block and the rows reach
    // the lane's column from the whole warp afterwards (copy_records).
    __device__ __forceinline__ bool init(const ModelDev &M, const ParamsDev &P, const OutDev &O,
                                         uint64_t pi, uint64_t i, const float *rc)
    {
        const int kind = __float_as_int(rc[R_KIND]);
        const int32_t n_delay = __float_as_int(rc[R_C0 + C_NDELAY]);
        if (kind != K_RUN) {
            const int32_t on = TTC ? -1 : n_delay;
            if (kind == K_INVALID) {
                const double nan = __longlong_as_double(0x7ff8000000000000ll);
                store_out(O, i, AEB_INVALID, nan, nan, nan, nan, 0, -1);
            } else if (kind == K_CONTACT0) {
                store_out(O, i, AEB_CONTACT, 0.0, 0.0, __ldg(P.col[kV0] + pi), 0.0, 0, on);
            } else if (kind == K_STOP0) {
                store_out(O, i, AEB_STOP, 0.0, 0.0, 0.0, 0.0, 0, on);
            } else {
                store_out(O, i, AEB_HORIZON, 0.0, 0.0, 0.0, 0.0, 0, on);
            }
            return true;
        }
        vh = rc[R_W0H];
        vl = rc[R_W0L];
        gh = rc[R_G0H];
        gl = rc[R_G0L];
        nh2s = rc[R_NH2S];
        ndts = 2.0f * nh2s;
        nh6s = rc[R_NH6S];
        nmP = rc[R_NMP];
        // -p1 = -1 when tau > 0 (then np2 or np3 is nonzero), else 0
        set_cf(L_NP1, (rc[R_C0 + C_NP2] != 0.0f || rc[R_C0 + C_NP3] != 0.0f) ? -1.0f : 0.0f);
        // (1 - mP)^(K-1): the actuator decay over a window's last K-1 steps
        set_cf(L_QF, powi<AEB_FP32_WINDOW - 1>(1.0f + nmP));
        if (TTC) set_ci(L_NCHK, 0);  // test the trigger at the first step
        e = 0.0f;  // a = 0 and the command is 0 before onset
        set_cf(L_U, 0.0f);
        n = 0;
        trig = !TTC;
        set_ci(L_NB, TTC ? INT_MAX : n_delay);
        next_event(M.n_max - 1);
        // Before onset e = u = 0, so every stage's demand is D = 0, where the
        // realised deceleration min(D, f0 + f1 D, r0 + r1 D, mu g cos) is 0
        // (mu >= 0): the stage term r + g sin(theta) is g sin(theta), and no
        // breakpoint can be reached.  The piece is selected at onset.
        C = rc[R_C0 + C_GS];
        a1 = a2 = a3 = a4 = 0.0f;
        eth = -finf();
        set_cf(L_ETHK, -finf());
        return false;
    }
};

// After lanes took samples cursor, cursor + 1, ... of the tile (the lanes of
// `taken`, in lane order): the rows and the record block of those in `keep`
// reach their columns, written by the whole warp (lane t: word t of the
// column's rows-and-record part; consecutive words, so no bank conflicts),
// instead of ~20 loads and stores by each refilling lane alone.
template <bool TTC>
__device__ __forceinline__ void copy_records(float *coldw, const float *tf, const Tile &tile,
                                             int cursor, unsigned taken, unsigned keep)
{
    constexpr int NC = copy_fields<TTC>(), CS = cold_stride<TTC>(), RS = rec_stride<TTC>();
    const int t = (int)(threadIdx.x & 31u);
    const uint64_t base = t < 2 ? tile.p0 : t < 4 ? tile.o0 : tile.k0;  // rows (t < 6)
    int r = 0;
    for (unsigned tk = taken; tk; tk &= tk - 1, ++r) {
        const int l = __ffs(tk) - 1;
        if (!((keep >> l) & 1u)) continue;
        const int slot = cursor + r;
        float w = 0.0f;
        if (t < L_C0 - L_PIDXLO) {
            const uint64_t v = base + (uint64_t)slot;
            w = __int_as_float((int)(uint32_t)((t & 1) ? (v >> 32) : v));
        } else if (t < L_C0 - L_PIDXLO + NC) {
            w = tf[slot * RS + R_C0 + (t - (L_C0 - L_PIDXLO))];
        }
        if (t < L_C0 - L_PIDXLO + NC) coldw[l * CS + L_PIDXLO + t] = w;
    }
    __syncwarp();  // the columns are read by their lanes from here on
}

// Records of ended rollouts waiting for the warp's flush, per warp,
// field-major.  A window record (len > 0) holds the state at the start of the
// window that contained the end and the lane's step constants; a terminal
// record (len = 0, from a slow step) holds the last step's start and end pairs
// (end pairs in the B_A1 .. B_A4 slots) and its status.  Both keep the
// scales s (B_S) and -s h6 (B_NH6S) that undo the scaled units.
enum {
    B_VH, B_VL, B_GH, B_GL, B_E, B_NH2S, B_NH6S, B_A1, B_A2, B_A3, B_A4, B_NMP,
    B_C, B_S, B_SIGMA, B_NF
};
enum { B_G1H = B_A1, B_G1L = B_A2, B_W1H = B_A3, B_W1L = B_A4 };
enum { B_IDXLO, B_IDXHI, B_PIDXLO, B_PIDXHI, B_STATUS, B_N, B_LEN, B_ONSET, B_NI };
constexpr int kBatchWords = (B_NF + B_NI) * 32;
// Per-step perception: readings of up to kBandSlots lanes near their trigger,
// kBandCache steps each, in the margin's units (+inf: missing), and per slot
// the tag of what it holds: the reading row (two words), the first step and
// the count.
constexpr int kBandSlots = 3;
constexpr int kBandCache = 2 * AEB_FP32_WINDOW;
enum { G_KLO, G_KHI, G_STEP, G_CNT, G_NI };
// and per slot the band window's states (step_window_st): 2K low words, the
// window's start, one word of padding (slots in different banks)
constexpr int kBandState = 2 * AEB_FP32_WINDOW + 4;
template <bool TTC, bool PERC>
__host__ __device__ constexpr int warp_words(int T)
{
    return rec_stride<TTC>() * T + kBatchWords + cold_stride<TTC>() * 32 +
           (PERC ? kBandSlots * (kBandCache + G_NI + kBandState) : 0);
}
template <bool TTC, bool PERC>
__host__ __device__ constexpr size_t smem_per_block(int T)
{
    return sizeof(float) * warp_words<TTC, PERC>(T) * kWarps;
}

// For the warp's queued records, all 32 lanes at once: replay the windows that
// contained an end one checked step at a time, then the binary64 refinement
// of the last step (Sec. V-D termination; the refinement of the last step).
template <int LEAD, bool TTC, bool PERC>
__device__ __forceinline__ void flush_batch(const ModelDev &M, const ModelF32 &F,
                                            const ParamsDev &P, const OutDev &O,
                                            const float *bf, const int *bi, int count)
{
    __syncwarp();
    const int j = threadIdx.x & 31;
    if (j < count) {
        const uint64_t i = (uint64_t)(uint32_t)bi[B_IDXLO * 32 + j] |
                           ((uint64_t)(uint32_t)bi[B_IDXHI * 32 + j] << 32);
        const uint64_t pi = (uint64_t)(uint32_t)bi[B_PIDXLO * 32 + j] |
                            ((uint64_t)(uint32_t)bi[B_PIDXHI * 32 + j] << 32);
        const int len = bi[B_LEN * 32 + j] & 0xff;
        const int trel = (bi[B_LEN * 32 + j] >> 8) - 1;  // trigger step in the window (-1: none)
        int32_t on = bi[B_ONSET * 32 + j];
        int status;
        int32_t n1;
        float g0h, g0l, w0h, w0l, g1h, g1l, w1h, w1l;
        if (len > 0) {
            Lane32<LEAD, TTC, PERC> R;
            R.vh = bf[B_VH * 32 + j];
            R.vl = bf[B_VL * 32 + j];
            R.gh = bf[B_GH * 32 + j];
            R.gl = bf[B_GL * 32 + j];
            R.e = bf[B_E * 32 + j];
            R.nh2s = bf[B_NH2S * 32 + j];
            R.ndts = 2.0f * R.nh2s;
            R.nh6s = bf[B_NH6S * 32 + j];
            R.a1 = bf[B_A1 * 32 + j];
            R.a2 = bf[B_A2 * 32 + j];
            R.a3 = bf[B_A3 * 32 + j];
            R.a4 = bf[B_A4 * 32 + j];
            R.nmP = bf[B_NMP * 32 + j];
            R.C = bf[B_C * 32 + j];
            R.n = bi[B_N * 32 + j];
            const int32_t nstart = R.n;
            // ends within len steps: the window's last state is terminal
            float vl1, gl1;
            const float sig = bf[B_SIGMA * 32 + j];
            for (int s = 1; !R.step_fast(F, vl1, gl1, sig) && s < len; ++s) {
            }
            g0h = R.gh;
            g0l = R.gl;
            w0h = R.vh;
            w0l = R.vl;
            g1h = R.gh;
            g1l = gl1;
            w1h = R.vh;
            w1l = vl1;
            n1 = R.n + 1;
            status = R.hits_lead(F, gl1, sig) ? AEB_CONTACT : AEB_STOP;
            // a trigger tested inside the window after the rollout's last step
            // never happened
            if (trel >= 0 && nstart + trel > n1 - 1) on = -1;
        } else {
            g0h = bf[B_GH * 32 + j];
            g0l = bf[B_GL * 32 + j];
            w0h = bf[B_VH * 32 + j];
            w0l = bf[B_VL * 32 + j];
            g1h = bf[B_G1H * 32 + j];
            g1l = bf[B_G1L * 32 + j];
            w1h = bf[B_W1H * 32 + j];
            w1l = bf[B_W1L * 32 + j];
            n1 = bi[B_N * 32 + j];
            status = bi[B_STATUS * 32 + j];
        }
        const double d0 = __ldg(P.col[kD0] + pi);
        const double sd = (double)bf[B_S * 32 + j];
        // back to metres and metres per second: 1 / sigma = -h6 s / s^2 and
        // 1 / s, one binary64 division each (division is slow in binary64)
        const double isig = -(double)bf[B_NH6S * 32 + j] / (sd * sd);
        const double isd = 1.0 / sd;
        const double x0 = d0 - ((double)g0h + (double)g0l) * isig;
        const double x1 = d0 - ((double)g1h + (double)g1l) * isig;
        const double w0 = ((double)w0h + (double)w0l) * isd;
        const double w1 = ((double)w1h + (double)w1l) * isd;
        const double n = (double)(n1 - 1);
        if (status == AEB_CONTACT && LEAD == kLeadMoving) {
            // gaps and closing speeds to the moving lead at both ends of the step
            const double t0 = n * M.dt, t1 = (double)n1 * M.dt;
            const double l0 = (M.lead_decel > 0.0 && t0 >= M.lead_ts)
                                  ? M.lead_xs : t0 * (M.lead_v0 - (0.5 * M.lead_decel) * t0);
            const double l1 = (M.lead_decel > 0.0 && t1 >= M.lead_ts)
                                  ? M.lead_xs : t1 * (M.lead_v0 - (0.5 * M.lead_decel) * t1);
            const double u0 = (M.lead_decel > 0.0 && t0 >= M.lead_ts) ? 0.0
                                                                     : M.lead_v0 - M.lead_decel * t0;
            const double u1 = (M.lead_decel > 0.0 && t1 >= M.lead_ts) ? 0.0
                                                                     : M.lead_v0 - M.lead_decel * t1;
            const double q0 = (d0 + l0) - x0, q1 = (d0 + l1) - x1;
            const double s = q0 / (q0 - q1);
            const double c0 = w0 - u0, c1 = w1 - u1;
            store_out(O, i, AEB_CONTACT, x1, x0 + s * (x1 - x0), c0 + s * (c1 - c0),
                      (n + s) * M.dt, n1, on);
        } else if (status == AEB_CONTACT) {
            const double s = (d0 - x0) / (x1 - x0);
            store_out(O, i, AEB_CONTACT, x1, d0, w0 + s * (w1 - w0), (n + s) * M.dt, n1, on);
        } else if (status == AEB_STOP) {
            const double s = w0 / (w0 - w1);
            store_out(O, i, AEB_STOP, x1, x0 + s * (x1 - x0), 0.0, (n + s) * M.dt, n1, on);
        } else {
            store_out(O, i, AEB_HORIZON, x1, x1, 0.0, (double)n1 * M.dt, n1, on);
        }
    }
    __syncwarp();
}

// One warp walks tiles of kTile samples claimed from a global counter; see the
// file comment.  No wait on other warps or on the host: the loop ends when the
// tiles are used up and no lane holds a rollout.
template <int LEAD, bool TTC, bool PERC>
__global__ void __launch_bounds__(kThreads, PERC ? 5 : AEB_FP32_MIN_BLOCKS)
k_rollout_fp32(ModelDev M, ModelF32 F, ParamsDev P, OutDev O, WorkDev W)
{
    extern __shared__ float smem[];
    const unsigned lane = threadIdx.x & 31u;
    const int T = (int)W.tile;
    float *tf = smem + (threadIdx.x >> 5) * warp_words<TTC, PERC>(T);
    float *bf = tf + rec_stride<TTC>() * T;
    int *bi = reinterpret_cast<int *>(bf + B_NF * 32);
    float *coldw = bf + kBatchWords;
    float *rdg = coldw + cold_stride<TTC>() * 32;  // band readings (per-step perception)
    int *btag = reinterpret_cast<int *>(rdg + kBandSlots * kBandCache);
    float *sst = reinterpret_cast<float *>(btag + kBandSlots * G_NI);  // band window states
    if (PERC && (int)lane < kBandSlots) btag[lane * G_NI + G_CNT] = 0;  // nothing cached
    const int32_t n_last = M.n_max - 1;
    // A band window starting at step n runs up to K steps if the reading index
    // n + L is even, else K - 1 (a fresh batch of readings starts at the even
    // index below n + L): the length never depends on what the slot holds.
    auto band_len = [&](int32_t n) { return AEB_FP32_WINDOW - (int)((n + F.plat) & 1); };
    // where the readings of a band lane's step n are in its slot
    auto band_rd = [&](int sl, int32_t n) {
        return rdg + sl * kBandCache + (n - btag[sl * G_NI + G_STEP]);
    };

    Tile tile{};
    int cursor = 0, bcount = 0;
    bool dry = false;
    Lane32<LEAD, TTC, PERC> L;
    L.cold = coldw + lane * cold_stride<TTC>();
    bool active = false;
    unsigned need = kFull;
    for (;;) {
        if (need) {
            while (need) {
                if (cursor >= tile.count) {
                    if (dry) {
                        if ((need >> lane) & 1u) active = false;
                        break;
                    }
                    const Tile nt = claim_tile(W, (uint32_t)T, M.ttc_thr);
                    if (!nt.ok) {
                        dry = true;
                        continue;
                    }
                    tile = nt;
                    cursor = 0;
                    __syncwarp();  // every lane has read its record of the previous tile
                    prep_tile<LEAD, TTC>(M, F, P, tile.p0, tile.count, tile.thr, tf);
                    __syncwarp();
                }
                const unsigned rank = __popc(need & lanemask_lt());
                const bool got = ((need >> lane) & 1u) && (int)rank < tile.count - cursor;
                bool ended = false;
                if (got) {
                    const int slot = cursor + (int)rank;
                    active = true;
                    ended = L.init(M, P, O, tile.p0 + slot, tile.o0 + slot,
                                   tf + slot * rec_stride<TTC>());
                }
                const unsigned taken = __ballot_sync(kFull, got);
                const unsigned endm = __ballot_sync(kFull, ended);
                copy_records<TTC>(coldw, tf, tile, cursor, taken, taken & ~endm);
                cursor += __popc(taken);
                need = (need & ~taken) | endm;
            }
            if (!__any_sync(kFull, active)) {
                flush_batch<LEAD, TTC, PERC>(M, F, P, O, bf, bi, bcount);
                return;
            }
        }

        // ---- one window of up to K RK4 steps (Sec. IV-D) per lane ----
        bool ended = false;
        float vl1, gl1;  // end-of-step low words of a slow step that ended
        int tlen = AEB_FP32_WINDOW;  // steps before the next TTC test
        int slot = -1;               // per-step perception: the lane's band slot
        bool wait = false;           // per-step perception: a band lane waiting for a slot
        if (TTC && active && !L.trig) {
            tlen = L.ci(L_NCHK) - L.n;  // steps the last test still covers
            if (tlen <= 0) {
                if (PERC) {  // no reading needed unless the worst-case noise can trigger
                    tlen = L.ttc_bound(F, L.ttc_margin(F));
                    if (tlen > 0) L.set_ci(L_NCHK, L.n + tlen);
                } else {
                    tlen = L.ttc_check(F, n_last);
                    if (!L.trig) L.set_ci(L_NCHK, L.n + tlen);
                }
            }
        }
        if (PERC) {
            // Lanes in their noise band (every step needs its reading): up to
            // kBandSlots of them get a slot that holds their readings, and run
            // windows with the trigger tested inside; the others wait for a
            // later pass (so that a sample's windows, and its arithmetic, never
            // depend on the lanes it shares a warp with), and a lane at its
            // last step (no window) tests that step alone.  Readings are
            // generated at full warp width, two per Philox block per thread:
            // a slot whose tag does not cover the lane's next band window
            // (band_len) gets 2K readings from the whole warp if it is alone,
            // else K from a half-warp, starting at the lane's step (one
            // earlier if that step's reading index is odd: a block holds an
            // even and an odd reading).
            const bool band = active && !L.trig && tlen <= 0;
            const unsigned bm = __ballot_sync(kFull, band && !L.at_slow(n_last));
            if (bm) {
                const int rank = __popc(bm & lanemask_lt());
                if (((bm >> lane) & 1u) && rank < kBandSlots) slot = rank;
                const int klo = L.ci(L_KIDXLO), khi = L.ci(L_KIDXHI);
                bool miss = false;
                if (slot >= 0) {
                    const int *tg = btag + slot * G_NI;
                    miss = !(tg[G_KLO] == klo && tg[G_KHI] == khi && tg[G_STEP] <= L.n &&
                             L.n + band_len(L.n) <= tg[G_STEP] + tg[G_CNT]);
                }
                unsigned mm = __ballot_sync(kFull, miss);
                if (mm) {
                    __syncwarp();  // the last window's reads of the slots come first
                    const int g = __popc(mm);
                    const int par = (int)((L.n + F.plat) & 1);
                    if (miss) {  // the schedule below: pairs in rank order, a last single
                        const int iota = __popc(mm & lanemask_lt());
                        int *tg = btag + slot * G_NI;
                        tg[G_KLO] = klo;
                        tg[G_KHI] = khi;
                        tg[G_STEP] = L.n - par;
                        tg[G_CNT] = ((g & 1) && iota == g - 1) ? kBandCache : AEB_FP32_WINDOW;
                    }
                    const float sgl = L.cf(L_SIGMA);
                    const int hw = (int)(lane >> 4);
                    while (mm) {
                        const int sa = __ffs(mm) - 1;
                        mm &= mm - 1;
                        const bool pair = mm != 0;
                        const int sbb = pair ? __ffs(mm) - 1 : sa;
                        if (pair) mm &= mm - 1;
                        const int src = (pair && hw) ? sbb : sa;
                        const uint64_t kr = (uint64_t)(uint32_t)__shfl_sync(kFull, klo, src) |
                                            ((uint64_t)(uint32_t)__shfl_sync(kFull, khi, src) << 32);
                        const int32_t ns = __shfl_sync(kFull, L.n, src);
                        const float sig = __shfl_sync(kFull, sgl, src);
                        const int ss = __shfl_sync(kFull, slot, src);
                        // block q of this slot's batch: readings 2q, 2q + 1 of its cache
                        const int q = pair ? (int)(lane & 15u) : (int)lane;
                        const long long r0 = (long long)ns + F.plat;
                        float ra, rb;
                        L.reading_pair(F, kr, (uint64_t)(r0 >> 1) + (uint64_t)q, sig, ra, rb);
                        float *rs = rdg + ss * kBandCache;
                        rs[2 * q] = ra;
                        rs[2 * q + 1] = rb;
                    }
                }
                __syncwarp();
            }
            if (band && slot < 0) {
                if (L.at_slow(n_last)) {
                    tlen = L.ttc_check(F, n_last);
                    if (!L.trig) L.set_ci(L_NCHK, L.n + tlen);
                } else {
                    wait = true;
                }
            }
        }
        // Most passes: every active lane can run a full window (no event in
        // reach); one vote decides.  Otherwise handle onsets, slow steps and
        // window lengths lane by lane.
        bool full = __all_sync(kFull, !active || L.full_window_ok(tlen));
        int len = AEB_FP32_WINDOW;
        if (!full) {
            const bool onset = active && L.n == L.ev && L.n < n_last;
            if (__any_sync(kFull, onset)) {  // warp-uniform: once per rollout
                if (onset) L.onset_event(F, n_last);
            }
            // a lane already at a slow step runs no window in this pass
            if (active)
                len = (wait || L.at_slow(n_last)) ? 0 : L.window_len(slot >= 0 ? band_len(L.n) : tlen);
            // (a lane with readings tests its trigger in the band window, never
            // in the unrolled full one)
            full = __all_sync(kFull, len == AEB_FP32_WINDOW && slot < 0);
        }
        bool replay = false;
        if (full) {
            // (the perception kernels, whose readings and band code already
            // fill the instruction cache, run it through the rolled loop: the
            // unrolled copy costs them more in cache misses than it saves)
            if (active) replay = L.template step_window<!PERC>(F, len);
        } else if (PERC && __any_sync(kFull, slot >= 0)) {
            // Band lanes keep their window's states; then the warp tests each
            // band lane's trigger at all the window's steps at once (lane j:
            // step j, with the margin's window-constant parts and the
            // readings of the band lane).  The first step that fires is the
            // trigger; if its onset falls inside the window, the lane goes
            // back to the window's start and, triggered, runs up to the onset
            // in the next pass, the window the trigger test inside the loop
            // would have cut (the same steps, so the same arithmetic).
            float *st = (slot >= 0 && len > 0) ? sst + slot * kBandState : nullptr;
            float thr_h = 0.0f, c1 = 0.0f, hk = 0.0f;
            if (st) L.band_consts(thr_h, c1, hk);
            const int32_t n0 = L.n;
            if (active && len > 0) replay = L.step_window_st(F, len, st);
            __syncwarp();
            unsigned tm = __ballot_sync(kFull, st != nullptr);
            int tr = -1;
            const float sl = LEAD == kLeadMoving ? L.cf(L_S) : 0.0f;
            const float sg = LEAD == kLeadMoving ? L.cf(L_SIGMA) : 0.0f;
            while (tm) {
                const int src = __ffs(tm) - 1;
                tm &= tm - 1;
                const int ss = __shfl_sync(kFull, slot, src);
                const int ln = __shfl_sync(kFull, len, src);
                const int32_t m0 = __shfl_sync(kFull, n0, src);
                const float th = __shfl_sync(kFull, thr_h, src);
                const float cc = __shfl_sync(kFull, c1, src);
                const float hh = __shfl_sync(kFull, hk, src);
                const float ssl = __shfl_sync(kFull, sl, src);
                const float ssg = __shfl_sync(kFull, sg, src);
                bool f = false;
                if ((int)lane < ln) {
                    const float *sp = sst + ss * kBandState;
                    float m = (sp[lane] + hh) - fmaf(th, sp[AEB_FP32_WINDOW + lane], cc);
                    if (LEAD == kLeadMoving)
                        m = m + fmaf(th, L.lead_speed(F, m0 + (int32_t)lane, ssl),
                                     L.lead_gap(F, m0 + (int32_t)lane, ssg));
                    f = m + band_rd(ss, m0)[lane] <= 0.0f;  // a missing reading never fires
                }
                const unsigned fb = __ballot_sync(kFull, f);
                if ((int)lane == src && fb) tr = __ffs(fb) - 1;
            }
            if (tr >= 0) {
                L.fire(F, n0 + tr, n_last);
                if (L.ev - n0 < len) {  // the onset falls inside the window
                    L.band_rewind(st, n0);
                    replay = false;
                }
            }
        } else {
            if (active && len > 0) replay = L.template step_window<false>(F, len);
        }
        // Slow steps (breakpoint crossings, the horizon's last step) after the
        // windows: a window that stopped right before one takes it in the same
        // pass, so the lane does not sit out the next pass's window for one
        // step.  A lane before its TTC trigger takes one only if it ran no
        // window in this pass (its trigger test for this step came first).
        const bool slow = active && !replay && (!TTC || L.trig || len == 0) && L.at_slow(n_last);
        if (__any_sync(kFull, slow)) {  // warp-uniform: rare
            if (slow) ended = L.step_slow(F, n_last, vl1, gl1);
        }
        ended = ended || replay;
        const unsigned endm = __ballot_sync(kFull, ended);
        if (endm) {
            const int cnt = __popc(endm);
            if (bcount + cnt > 32) {
                flush_batch<LEAD, TTC, PERC>(M, F, P, O, bf, bi, bcount);
                bcount = 0;
            }
            if (ended) {
                const int j = bcount + __popc(endm & lanemask_lt());
                bf[B_VH * 32 + j] = L.vh;
                bf[B_VL * 32 + j] = L.vl;
                bf[B_GH * 32 + j] = L.gh;
                bf[B_GL * 32 + j] = L.gl;
                bf[B_NH6S * 32 + j] = L.nh6s;
                bf[B_S * 32 + j] = L.cf(L_S);
                bf[B_SIGMA * 32 + j] = L.cf(L_SIGMA);
                bi[B_IDXLO * 32 + j] = L.ci(L_IDXLO);
                bi[B_IDXHI * 32 + j] = L.ci(L_IDXHI);
                bi[B_PIDXLO * 32 + j] = L.ci(L_PIDXLO);
                bi[B_PIDXHI * 32 + j] = L.ci(L_PIDXHI);
                bi[B_ONSET * 32 + j] = L.onset();
                if (replay) {
                    bf[B_E * 32 + j] = L.e;
                    bf[B_NH2S * 32 + j] = L.nh2s;
                    bf[B_A1 * 32 + j] = L.a1;
                    bf[B_A2 * 32 + j] = L.a2;
                    bf[B_A3 * 32 + j] = L.a3;
                    bf[B_A4 * 32 + j] = L.a4;
                    bf[B_NMP * 32 + j] = L.nmP;
                    bf[B_C * 32 + j] = L.C;
                    bi[B_N * 32 + j] = L.n;
                    // + the step of a trigger inside the window (from the
                    // test-step field; the flush drops a trigger after the end)
                    const int trel = (PERC && L.trig && L.ci(L_NCHK) >= L.n) ? L.ci(L_NCHK) - L.n : -1;
                    bi[B_LEN * 32 + j] = len | ((trel + 1) << 8);
                } else {
                    bf[B_G1H * 32 + j] = L.gh;
                    bf[B_G1L * 32 + j] = gl1;
                    bf[B_W1H * 32 + j] = L.vh;
                    bf[B_W1L * 32 + j] = vl1;
                    bi[B_STATUS * 32 + j] = L.hits_lead(F, gl1, L.cf(L_SIGMA))
                                                ? AEB_CONTACT
                                                : (L.vh + vl1 <= 0.0f ? AEB_STOP : AEB_HORIZON);
                    bi[B_N * 32 + j] = L.n + 1;
                    bi[B_LEN * 32 + j] = 0;
                }
            }
            bcount += cnt;
            need = endm;
        }
    }
}

ModelF32 to_f32(const ModelDev &m)
{
    ModelF32 f;
    f.acmd = (float)m.a_cmd;
    f.rho = (float)m.rho;
    f.area = (float)m.area;
    f.hl = (float)m.hl;
    f.g = (float)m.g;
    f.phi_f = (float)m.phi_f;
    f.beta = (float)m.beta;
    f.dt = (float)m.dt;
    f.idt = (float)(1.0 / m.dt);
    f.lv0 = (float)m.lead_v0;
    f.lb = (float)m.lead_decel;
    f.lhb = (float)(0.5 * m.lead_decel);
    f.lts = (float)m.lead_ts;
    f.lxs = (float)m.lead_xs;
    f.psig = (float)m.perc_sigma;
    f.pdrop_h = (uint64_t)std::ceil(m.perc_drop * 4294967296.0);  // perc_drop in [0, 1]
    f.pseed = m.perc_seed;
    f.plat = m.perc_lat;
    f.perc = m.perc;
    return f;
}

template <int LEAD, bool TTC, bool PERC>
cudaError_t launch_t(const ModelDev &m, const ParamsDev &p, const OutDev &o, const WorkDev &w,
                     const LaunchCfg &cfg, cudaStream_t s)
{
    auto kern = k_rollout_fp32<LEAD, TTC, PERC>;
    const int T = w.tiles ? (int)w.tile : (cfg.tile > 0 ? cfg.tile : kTileDefault);
    if (T < 32 || T > kTileMax || T % 32) return cudaErrorInvalidValue;
    const size_t smem = smem_per_block<TTC, PERC>(T);
    int dev = 0, sms = 0, per_sm = cfg.blocks_per_sm;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (per_sm <= 0 || per_sm > occ) per_sm = occ;
    WorkDev wt = w;
    wt.tile = (uint32_t)T;
    const uint64_t tiles = tiles_of(wt, (uint32_t)T);
    uint64_t blocks = (uint64_t)sms * per_sm;
    const uint64_t need_blocks = (tiles + kWarps - 1) / kWarps;
    if (need_blocks < blocks) blocks = need_blocks;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, kThreads, smem, s>>>(m, to_f32(m), p, o, wt);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rollout_fp32(const ModelDev &m, const ParamsDev &p, const OutDev &o,
                                const WorkDev &w, const LaunchCfg &cfg, cudaStream_t s)
{
    const bool ttc = m.trigger == AEB_TRIGGER_TTC;
    // per-step perception readings (TTC trigger only) have their own kernels
    const bool perc = ttc && m.perc;
    if (m.lead_moving)
        return perc ? launch_t<kLeadMoving, true, true>(m, p, o, w, cfg, s)
                    : ttc ? launch_t<kLeadMoving, true, false>(m, p, o, w, cfg, s)
                          : launch_t<kLeadMoving, false, false>(m, p, o, w, cfg, s);
    if (m.lead)
        return perc ? launch_t<kLeadStationary, true, true>(m, p, o, w, cfg, s)
                    : ttc ? launch_t<kLeadStationary, true, false>(m, p, o, w, cfg, s)
                          : launch_t<kLeadStationary, false, false>(m, p, o, w, cfg, s);
    return perc ? launch_t<kNoLead, true, true>(m, p, o, w, cfg, s)
                : ttc ? launch_t<kNoLead, true, false>(m, p, o, w, cfg, s)
                      : launch_t<kNoLead, false, false>(m, p, o, w, cfg, s);
}

}  // namespace aeb
