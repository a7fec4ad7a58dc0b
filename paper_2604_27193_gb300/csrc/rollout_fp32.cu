// rollout_fp32.cu -- binary32 rollout kernel with compensated state.
//
// The RK4 stages of Eq. 7-9 (Sec. IV-D) run in binary32 with fused
// multiply-add.  Position and speed are carried as unevaluated double-float
// sums (hi + lo): each step's increment is added with Fast2Sum and its rounding
// error kept in lo, so 1e4-1e5 increments of 1e-3-1e-4 relative size do not
// lose the ~1e-7 relative precision of a binary32 stage.  The speed pair is
// renormalised every step because the stages read its high word.  The contact test compares the
// double-float position with a double-float d0, and the TTC trigger margin
// (gap - thr v) is formed with exact product and sum error terms.  Binary64 is
// used only once per sample: the brake-onset step (the same integer rule as the
// binary64 path, so the onset step is always identical) and the linear
// stop/contact refinement of the last step from the hi + lo pairs.
//
// The actuator lag (Eq. 6) is linear with the command u held over the step.
// The lane carries the deviation e = a - u instead of a: RK4's stage values
// are u + p_j e with p1 = 1, p2 = 1 - z/2, p3 = 1 - z/2 + z^2/4,
// p4 = 1 - z + z^2/2 - z^3/4 (z = dt / tau), and the step maps e to
// e - mP e with mP = z - z^2/2 + z^3/6 - z^4/24; this is what the four RK4
// stages of Eq. 6 evaluate.  Carried as a, the state would stall about
// ulp(a) / (2 z) short of the command in binary32; carried as e it decays with
// full relative precision.  When the command switches from 0 to a_cmd at the
// onset step, e drops by a_cmd.  tau = 0 (instantaneous actuator) is the case
// p_j = 0, mP = 1.
#include <climits>

#include "rollout_common.cuh"

namespace aeb {
namespace {

struct ModelF32 {
    float g, rho, area, hl, beta, phi_f;
    float dt, h6, nh2, nh6, ndt, acmd, thr_h, thr_l;
};

template <int CAP, bool LEAD, bool TTC>
struct Lane32 {
    float xh, xl, vh, vl, e;
    float d0h, d0l, gs, k;
    float mg, nf1, f0, nr1, r0, cap;
    float p1, p2, p3, p4, nmP;
    float nzh, nzl;
    int32_t n, n_b, n_delay;
    bool trig;

    // -(dv/dt) = r + g sin(theta) + k v^2 for actuator state a (Eq. 4-5).
    __device__ __forceinline__ float qacc(float vv, float aa) const
    {
        float r;
        if (CAP == AEB_CAP_LUMPED)
            r = fminf(-aa, cap);
        else
            r = fminf(fminf(-aa, mg), fminf(fmaf(nf1, aa, f0), fmaf(nr1, aa, r0)));
        return fmaf(k * vv, vv, r + gs);
    }

    __device__ __forceinline__ int32_t onset() const
    {
        return TTC ? (trig ? n_b : -1) : n_delay;
    }

    __device__ __forceinline__ bool init(const ModelDev &M, const ModelF32 &F, const ParamsDev &P,
                                         const OutDev &O, uint64_t i)
    {
        double f[AEB_NFIELDS];
        load_fields(P, i, f);
        if (!sample_valid(f)) {
            const double nan = __longlong_as_double(0x7ff8000000000000ll);
            store_out(O, i, AEB_INVALID, nan, nan, nan, nan, 0, -1);
            return true;
        }
        n_delay = steps_to_reach_dev(f[kTdelay], M.dt);
        trig = !TTC;
        n_b = n_delay;
        const int32_t on = TTC ? -1 : n_delay;
        const double d0 = f[kD0];
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
        d0h = __double2float_rn(d0);
        d0l = __double2float_rn(d0 - (double)d0h);
        gs = __double2float_rn(f[kGs]);
        k = ((F.rho * __double2float_rn(f[kCd])) * F.area) / (2.0f * __double2float_rn(f[kMass]));
        const float mu = __double2float_rn(f[kMu]);
        const float mh = mu * F.hl;
        if (CAP == AEB_CAP_LUMPED) {
            cap = (mu * F.g) / (1.0f + mh);
        } else {
            mg = mu * __double2float_rn(f[kGc]);
            const float im = 1.0f / (1.0f - mh), ip = 1.0f / (1.0f + mh);
            f0 = (mg * F.phi_f) * im;
            nf1 = -(1.0f - F.beta) * im;
            r0 = (mg * (1.0f - F.phi_f)) * ip;
            nr1 = -F.beta * ip;
        }
        const float tau = __double2float_rn(f[kTau]);
        if (f[kTau] > 0.0) {
            const double z = M.dt / f[kTau];
            p1 = 1.0f;
            p2 = __double2float_rn(1.0 - 0.5 * z);
            p3 = __double2float_rn(1.0 - 0.5 * z + 0.25 * z * z);
            p4 = __double2float_rn(1.0 - z + 0.5 * z * z - 0.25 * z * z * z);
            nmP = __double2float_rn(-(z * (1.0 + z * (-0.5 + z * (1.0 / 6.0 - z / 24.0)))));
        } else {
            p1 = p2 = p3 = p4 = 0.0f;
            nmP = -1.0f;
        }
        if (TTC) {
            nzh = __double2float_rn(f[kNoise]);
            nzl = __double2float_rn(f[kNoise] - (double)nzh);
        }
        xh = 0.0f;
        xl = 0.0f;
        vh = __double2float_rn(f[kV0]);
        vl = __double2float_rn(f[kV0] - (double)vh);
        e = 0.0f;  // a = 0 and the command before onset is 0
        n = 0;
        return false;
    }

    __device__ __forceinline__ bool step(const ModelDev &M, const ModelF32 &F, const ParamsDev &P,
                                         const OutDev &O, uint64_t i)
    {
        if (TTC && !trig) {
            // measured gap (d0 - x) + noise against thr * v, as double-float
            const float s = d0h - xh;
            const float bb = s - d0h;
            const float es = (d0h - (s - bb)) + (-xh - bb);
            const float p = F.thr_h * vh;
            const float pe = fmaf(F.thr_h, vh, -p);
            const float hi = s - p;
            const float lo = ((es + (d0l - xl)) + (nzh + nzl)) - ((pe + F.thr_h * vl) + F.thr_l * vh);
            if (hi + lo <= 0.0f) {
                trig = true;
                long long nb = (long long)n + n_delay;
                n_b = nb > INT_MAX ? INT_MAX : (int32_t)nb;
            }
        }
        const bool on = trig && n >= n_b;
        const float u = on ? F.acmd : 0.0f;
        const float ee = (trig && n == n_b) ? e - F.acmd : e;  // command switches on
        const float a1 = fmaf(ee, p1, u);
        const float a2 = fmaf(ee, p2, u);
        const float a3 = fmaf(ee, p3, u);
        const float a4 = fmaf(ee, p4, u);
        const float en = fmaf(nmP, ee, ee);

        const float q1 = qacc(vh, a1);
        const float v2 = fmaf(F.nh2, q1, vh);
        const float q2 = qacc(v2, a2);
        const float v3 = fmaf(F.nh2, q2, vh);
        const float q3 = qacc(v3, a3);
        const float v4 = fmaf(F.ndt, q3, vh);
        const float q4 = qacc(v4, a4);

        const float dv = F.nh6 * fmaf(2.0f, q2 + q3, q1 + q4);
        const float dx = fmaf(F.dt, vl, F.h6 * fmaf(2.0f, v2 + v3, vh + v4));
        // v: Fast2Sum of the increment, then renormalise so |vl| <= ulp(vh)/2.
        // Without the renormalisation a nearly constant increment leaves the
        // same rounding residual every step, vl grows linearly and the stages,
        // which read vh, see a biased speed.
        const float vs0 = vh + dv;
        const float tv = vl + (dv - (vs0 - vh));
        const float vs = vs0 + tv;
        const float vln = tv - (vs - vs0);
        // x: Fast2Sum only (no stage reads x)
        const float xs = xh + dx;
        const float xln = xl + (dx - (xs - xh));

        const bool contact = LEAD && ((xs - d0h) + (xln - d0l) >= 0.0f);
        const bool stop = vs <= 0.0f;
        if (contact || stop || n + 1 >= M.n_max) {
            const double x0 = (double)xh + (double)xl, x1 = (double)xs + (double)xln;
            const double w0 = (double)vh + (double)vl, w1 = (double)vs + (double)vln;
            const double dt = M.dt;
            if (contact) {
                const double d0 = __ldg(P.col[kD0] + i);
                const double s = (d0 - x0) / (x1 - x0);
                store_out(O, i, AEB_CONTACT, x1, d0, w0 + s * (w1 - w0), ((double)n + s) * dt,
                          n + 1, onset());
            } else if (stop) {
                const double s = w0 / (w0 - w1);
                store_out(O, i, AEB_STOP, x1, x0 + s * (x1 - x0), 0.0, ((double)n + s) * dt,
                          n + 1, onset());
            } else {
                store_out(O, i, AEB_HORIZON, x1, x1, 0.0, (double)(n + 1) * dt, n + 1, onset());
            }
            return true;
        }
        xh = xs;
        xl = xln;
        vh = vs;
        vl = vln;
        e = en;
        n = n + 1;
        return false;
    }
};

template <int CAP, bool LEAD, bool TTC>
__global__ void __launch_bounds__(128) k_rollout_fp32(ModelDev M, ModelF32 F, ParamsDev P,
                                                      OutDev O, WorkDev W)
{
    rollout_driver<Lane32<CAP, LEAD, TTC>>(M, F, P, O, W);
}

ModelF32 to_f32(const ModelDev &m)
{
    ModelF32 f;
    f.g = (float)m.g;
    f.rho = (float)m.rho;
    f.area = (float)m.area;
    f.hl = (float)m.hl;
    f.beta = (float)m.beta;
    f.phi_f = (float)m.phi_f;
    f.dt = (float)m.dt;
    f.h6 = (float)m.h6;
    f.nh2 = -(float)m.h2;
    f.nh6 = -(float)m.h6;
    f.ndt = -(float)m.dt;
    f.acmd = (float)m.a_cmd;
    f.thr_h = (float)m.ttc_thr;
    f.thr_l = (float)(m.ttc_thr - (double)f.thr_h);
    return f;
}

template <int CAP, bool LEAD, bool TTC>
cudaError_t launch_t(const ModelDev &m, const ParamsDev &p, const OutDev &o, const WorkDev &w,
                     const LaunchCfg &cfg, cudaStream_t s)
{
    auto kern = k_rollout_fp32<CAP, LEAD, TTC>;
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
    uint64_t tiles = (w.n + w.tile - 1) / w.tile;
    uint64_t blocks = (uint64_t)sms * per_sm;
    uint64_t need_blocks = (tiles + 3) / 4;
    if (need_blocks < blocks) blocks = need_blocks;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, 128, 0, s>>>(m, to_f32(m), p, o, w);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rollout_fp32(const ModelDev &m, const ParamsDev &p, const OutDev &o,
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
