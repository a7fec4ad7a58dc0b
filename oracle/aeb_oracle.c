/*
 * aeb_oracle.c -- plain FP64 CPU oracle for Monte Carlo AEB braking rollouts.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load it; the product library never does, and it
 * shares no source, header or generated table with the product.
 *
 * It is written to be read against the paper:
 *   Karjol & Alawneh, "Real-Time GPU-Accelerated Monte Carlo Evaluation of
 *   Safety-Critical AEB Systems Under Uncertainty".
 *   - state (x, v, a_brake,actual) and step command ............ Sec. III-A, Eq. 1-3
 *   - force balance with drag and grade ......................... Sec. III-B, Eq. 4
 *   - weight-transfer bound on realised deceleration ............ Sec. III-B, Eq. 5
 *   - first-order brake-actuator lag ............................ Sec. III-C, Eq. 6
 *   - complete ODE system ....................................... Sec. III-D, Eq. 7-9
 *   - fixed-step RK4, dt, horizon, termination v <= 0 ........... Sec. IV-B, IV-D, V-D
 *   - host-side seeded sampling ................................. Sec. IV-A, IV-C
 *   - collision probability P(D_stop > H0) ...................... Sec. VI-C, Eq. 19
 * The lead vehicle, reaction delay, range noise, per-axle friction caps and the
 * TTC trigger extend the paper; their reading is stated at each function.
 *
 * Arithmetic: IEEE binary64, every operation written out in the order it is
 * evaluated, no fused multiply-add (build with -ffp-contract=off), no fast-math.
 * Each function is the plain definition; there is no blocking or reordering.
 *
 * Parity status of each function (what pins it, see tests/test_oracle_*.py):
 *   om_philox4x64_10   pinned: numpy's Philox4x64-10 bit generator.
 *   om_sample          pinned: Kolmogorov-Smirnov / moment tests against scipy
 *                      distributions, clamping and counter-layout invariants.
 *   om_rollout_probe   pinned: equal to om_rollout without an override; the
 *                      recorded margins against the closed form of a car at
 *                      constant speed and against the trigger step it reports.
 *   om_rollout         pinned: closed forms (constant deceleration, constant
 *                      deceleration + quadratic drag, pure actuator lag, grade,
 *                      contact kinematics, TTC trigger step, moving-lead contact
 *                      and closing-speed trigger), RK4 order of
 *                      convergence, monotonicity sweeps, paper Table I / Sec. VI-C
 *                      statistics (statistical band).
 *   om_perception      pinned: numpy's Philox-4x64-10 per reading, the exact
 *                      Irwin-Hall CDF, dropout frequency; the trigger step of
 *                      coasting cars against a brute-force search, latency shift.
 *   om_sample_is       pinned: draws equal om_sample's from the proposal; weights
 *                      against scipy densities and tail masses; unbiasedness;
 *                      a rare event with an exact probability.
 *   om_axle_cap        pinned: brute-force fixed-point iteration of the per-axle
 *                      force balance.
 *   om_reduce          pinned: numpy / math.fsum brute force over the outputs.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Types (oracle-private; deliberately not shared with the product headers)   */
/* ------------------------------------------------------------------------- */

enum { OM_CAP_LUMPED = 0, OM_CAP_PER_AXLE = 1 };
enum { OM_TRIGGER_IMMEDIATE = 0, OM_TRIGGER_TTC = 1 };
enum { OM_STOP = 0, OM_CONTACT = 1, OM_HORIZON = 2, OM_INVALID = 255 };
enum { OM_DIST_CONST = 0, OM_DIST_UNIFORM = 1, OM_DIST_NORMAL = 2 };
enum { OM_NFIELDS = 10 };

typedef struct {
    double g;          /* gravitational acceleration [m/s^2]                  */
    double rho;        /* air density [kg/m^3]                                */
    double area;       /* frontal area A_f [m^2]                              */
    double h_cg;       /* centre-of-gravity height h [m]                      */
    double wheelbase;  /* wheelbase L [m]                                     */
    double beta;       /* front share of the demanded brake force             */
    double phi_f;      /* static front-axle share of the normal load          */
    double a_cmd;      /* commanded braking acceleration (negative) [m/s^2]   */
    double dt;         /* integration step [s]                                */
    double t_max;      /* horizon [s]                                         */
    double ttc_thr;    /* TTC trigger threshold [s]                           */
    int32_t cap_mode;  /* OM_CAP_*                                            */
    int32_t trigger;   /* OM_TRIGGER_*                                        */
    int32_t lead;      /* 1: lead vehicle, initially at distance d0           */
    int32_t pad_;
    double lead_v0;    /* initial speed of the lead [m/s] (0: stationary)     */
    double lead_decel; /* constant braking deceleration of the lead [m/s^2]   */
    double perc_sigma;   /* per-step perception noise scale [m] (TTC trigger)  */
    double perc_drop;    /* probability that a step's reading is missing        */
    double perc_latency; /* age of a reading when it is used [s]                */
    uint64_t perc_seed;  /* key of the per-step perception stream               */
} om_model;

/* Field order of a parameter set xi^(i) (structure-of-arrays columns). */
enum { F_V0 = 0, F_D0, F_MU, F_GS, F_GC, F_MASS, F_CD, F_TAU, F_TDELAY, F_NOISE };

typedef struct {
    int32_t kind;      /* OM_DIST_*                                           */
    int32_t pad_;
    double p0, p1;     /* const: p0 | uniform: [p0, p1) | normal: mean p0, sd p1 */
    double lo, hi;     /* result clamped to [lo, hi]                           */
} om_dist;

/* Distributions of the sampled quantities, in sampling-block order.        */
enum { S_V0 = 0, S_D0, S_MU, S_GRADE, S_MASS, S_CD, S_TAU, S_TDELAY, S_NOISE, S_COUNT };

typedef struct {
    om_dist dist[S_COUNT];
    uint64_t seed;
    uint64_t scenario_id;
} om_scenario;

typedef struct {
    uint64_t n, n_stop, n_contact, n_horizon, n_invalid, steps;
    double sum_d, sumsq_d, min_d, max_d;  /* over stopped samples, x_ref      */
    double sum_v, sumsq_v, min_v, max_v;  /* over contact samples, v_imp      */
} om_stats;

/* ------------------------------------------------------------------------- */
/* Philox-4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Counter-based: the output block depends only on */
/* (counter, key).  The paper fixes no generator (Sec. IV-C asks only for a   */
/* fixed seed); this is the reading used throughout.                          */
/* ------------------------------------------------------------------------- */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void om_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c0, &hi0, &lo0);
        mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* Sampling of xi^(i) (Sec. IV-A, IV-C).                                      */
/*   block b = 0..4 of sample i: counter (i, b, 0, 0), key (seed, scenario).  */
/*   quantity 2b uses words 0,1; quantity 2b+1 uses words 2,3.               */
/*   uniform draw: lo + (hi - lo) * U,  U = (w0 >> 11) * 2^-53 in [0, 1)      */
/*   normal draw:  mean + sd * sqrt(-2 ln U1) cos(2 pi U2)   (Box-Muller)     */
/*                 U1 = ((w0 >> 11) + 1) * 2^-53 in (0, 1], U2 from w1       */
/*   every draw is then clamped to [lo, hi].                                  */
/*   The grade angle is turned into g sin(theta), g cos(theta) here, on the   */
/*   host, like every other transcendental of the method.                     */
/* ------------------------------------------------------------------------- */

static double draw(const om_dist *d, uint64_t w0, uint64_t w1)
{
    const double two_m53 = 1.0 / 9007199254740992.0; /* 2^-53 */
    double x;
    if (d->kind == OM_DIST_UNIFORM) {
        double u = (double)(w0 >> 11) * two_m53;
        x = d->p0 + (d->p1 - d->p0) * u;
    } else if (d->kind == OM_DIST_NORMAL) {
        double u1 = (double)((w0 >> 11) + 1) * two_m53;
        double u2 = (double)(w1 >> 11) * two_m53;
        double radius = sqrt(-2.0 * log(u1));
        double z = radius * cos(6.283185307179586 * u2);
        x = d->p0 + d->p1 * z;
    } else {
        x = d->p0;
    }
    if (x < d->lo) x = d->lo;
    if (x > d->hi) x = d->hi;
    return x;
}

int om_sample(const om_model *m, const om_scenario *sc, uint64_t first, uint64_t n,
              double *const cols[OM_NFIELDS])
{
    const uint64_t key[2] = { sc->seed, sc->scenario_id };
    for (uint64_t j = 0; j < n; ++j) {
        uint64_t i = first + j;
        double q[S_COUNT + 1];
        for (int b = 0; b < 5; ++b) {
            uint64_t ctr[4] = { i, (uint64_t)b, 0, 0 }, w[4];
            om_philox4x64_10(ctr, key, w);
            int qa = 2 * b, qb = 2 * b + 1;
            q[qa] = draw(&sc->dist[qa], w[0], w[1]);
            if (qb < S_COUNT) q[qb] = draw(&sc->dist[qb], w[2], w[3]);
        }
        cols[F_V0][j] = q[S_V0];
        cols[F_D0][j] = q[S_D0];
        cols[F_MU][j] = q[S_MU];
        cols[F_GS][j] = m->g * sin(q[S_GRADE]);
        cols[F_GC][j] = m->g * cos(q[S_GRADE]);
        cols[F_MASS][j] = q[S_MASS];
        cols[F_CD][j] = q[S_CD];
        cols[F_TAU][j] = q[S_TAU];
        cols[F_TDELAY][j] = q[S_TDELAY];
        cols[F_NOISE][j] = q[S_NOISE];
    }
    return 0;
}

/*
 * Importance sampling (extension; Sec. VIII names rare-event estimation of
 * low collision probabilities as future work).  Parameter sets are drawn from
 * a proposal scenario q exactly as om_sample draws them, and each carries the
 * likelihood ratio w = p(xi) / q(xi) to the nominal scenario p, the product
 * over the nine quantities of one quantity's ratio for its clamped value x:
 *   constant: 1 (p and q must agree);
 *   an atom at a clamp bound (the bound holds probability mass under q):
 *     P_p(X <= lo) / P_q(X <= lo), or the upper tails at hi;
 *   otherwise the density ratio: uniform 1[a_p <= x < b_p] (b_q - a_q)/(b_p - a_p),
 *     normal (s_q / s_p) exp(z_q^2 / 2 - z_p^2 / 2), z = (x - mean) / sd.
 * p and q must have the same kind and clamp bounds per quantity, and a
 * uniform q must cover p's interval (else om_sample_is returns -1).  Then
 * E_q[w f(xi)] = E_p[f(xi)] for any outcome f.
 */
static double cdf_dist(const om_dist *d, double x) /* P(unclamped draw <= x) */
{
    if (d->kind == OM_DIST_UNIFORM) {
        double u = (x - d->p0) / (d->p1 - d->p0);
        return u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
    }
    return 0.5 * erfc(-((x - d->p0) / d->p1) / sqrt(2.0));
}

static double sf_dist(const om_dist *d, double x) /* P(unclamped draw > x) */
{
    if (d->kind == OM_DIST_UNIFORM) return 1.0 - cdf_dist(d, x);
    return 0.5 * erfc(((x - d->p0) / d->p1) / sqrt(2.0));
}

static double quantity_ratio(const om_dist *p, const om_dist *q, double x)
{
    if (q->kind == OM_DIST_CONST) return 1.0;
    if (x <= q->lo) {
        double mq = cdf_dist(q, q->lo);
        if (mq > 0.0) return cdf_dist(p, p->lo) / mq;
    }
    if (x >= q->hi) {
        double mq = sf_dist(q, q->hi);
        if (mq > 0.0) return sf_dist(p, p->hi) / mq;
    }
    if (q->kind == OM_DIST_UNIFORM) {
        if (!(x >= p->p0 && x < p->p1)) return 0.0;
        return (q->p1 - q->p0) / (p->p1 - p->p0);
    }
    double zp = (x - p->p0) / p->p1, zq = (x - q->p0) / q->p1;
    return (q->p1 / p->p1) * exp(0.5 * (zq * zq) - 0.5 * (zp * zp));
}

static int is_compatible(const om_dist *p, const om_dist *q)
{
    if (p->kind != q->kind || p->lo != q->lo || p->hi != q->hi) return 0;
    if (q->kind == OM_DIST_CONST) return p->p0 == q->p0;
    if (q->kind == OM_DIST_UNIFORM) return q->p0 <= p->p0 && p->p1 <= q->p1 && p->p1 > p->p0;
    return p->p1 > 0.0 && q->p1 > 0.0;
}

int om_sample_is(const om_model *m, const om_scenario *nominal, const om_scenario *proposal,
                 uint64_t first, uint64_t n, double *const cols[OM_NFIELDS], double *weights)
{
    for (int k = 0; k < S_COUNT; ++k)
        if (!is_compatible(&nominal->dist[k], &proposal->dist[k])) return -1;
    const uint64_t key[2] = { proposal->seed, proposal->scenario_id };
    for (uint64_t j = 0; j < n; ++j) {
        uint64_t i = first + j;
        double q[S_COUNT + 1];
        for (int b = 0; b < 5; ++b) {
            uint64_t ctr[4] = { i, (uint64_t)b, 0, 0 }, w[4];
            om_philox4x64_10(ctr, key, w);
            int qa = 2 * b, qb = 2 * b + 1;
            q[qa] = draw(&proposal->dist[qa], w[0], w[1]);
            if (qb < S_COUNT) q[qb] = draw(&proposal->dist[qb], w[2], w[3]);
        }
        double wt = 1.0;
        for (int k = 0; k < S_COUNT; ++k)
            wt *= quantity_ratio(&nominal->dist[k], &proposal->dist[k], q[k]);
        weights[j] = wt;
        cols[F_V0][j] = q[S_V0];
        cols[F_D0][j] = q[S_D0];
        cols[F_MU][j] = q[S_MU];
        cols[F_GS][j] = m->g * sin(q[S_GRADE]);
        cols[F_GC][j] = m->g * cos(q[S_GRADE]);
        cols[F_MASS][j] = q[S_MASS];
        cols[F_CD][j] = q[S_CD];
        cols[F_TAU][j] = q[S_TAU];
        cols[F_TDELAY][j] = q[S_TDELAY];
        cols[F_NOISE][j] = q[S_NOISE];
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Model pieces                                                               */
/* ------------------------------------------------------------------------- */

static double dmin(double a, double b) { return (b < a) ? b : a; }

/* Smallest integer n >= 0 with (double)n * dt >= t.  Used for the horizon    */
/* step count (T_max / dt, Sec. IV-B) and for the brake-onset delay.          */
int64_t om_steps_to_reach(double t, double dt)
{
    if (!(t > 0.0)) return 0;
    double q = ceil(t / dt);
    if (!(q <= 2147483647.0)) return 2147483647;  /* beyond any representable horizon */
    int64_t n = (int64_t)q;
    while (n > 0 && (double)(n - 1) * dt >= t) --n;
    while ((double)n * dt < t) ++n;
    return n;
}

/* Per-sample constants, each in the operation order stated. */
typedef struct {
    double v0, d0, gs, noise, tau;
    double k;            /* drag: (rho * C_d * A_f) / (2 m), Eq. 4             */
    double it;           /* 1 / tau, Eq. 6                                     */
    double mg;           /* mu * g cos(theta): both axles at their limit      */
    double f0, f1;       /* front-axle-limited line  r = f0 + f1 * D           */
    double r0, r1;       /* rear-axle-limited line   r = r0 + r1 * D           */
    double cap;          /* lumped bound of Eq. 5 solved for a                 */
    int64_t n_delay;
    int cap_mode;
} om_consts;

/* Coefficients of the realised-deceleration map below, once per sample. */
static void cap_coeffs(const om_model *m, double mu, double gc, om_consts *c)
{
    double hl = m->h_cg / m->wheelbase;
    double mh = mu * hl;
    c->mg = mu * gc;
    c->f0 = (c->mg * m->phi_f) / (1.0 - mh);
    c->f1 = (1.0 - m->beta) / (1.0 - mh);
    c->r0 = (c->mg * (1.0 - m->phi_f)) / (1.0 + mh);
    c->r1 = m->beta / (1.0 + mh);
    c->cap = (mu * m->g) / (1.0 + mh);
    c->cap_mode = m->cap_mode;
}

/*
 * Realised braking deceleration r for a demanded deceleration D = -a_brake,actual.
 *
 * Lumped (Eq. 5, as printed).  The bound a >= -mu g (1 + (h/L) a / g) is linear
 * in a; with a = -r it reads r <= mu g - mu (h/L) r, i.e. r <= mu g / (1 + mu h/L).
 * So r = min(D, mu g / (1 + mu h / L)).
 *
 * Per axle.  Front/rear demanded forces beta m D and (1-beta) m D are each
 * capped at mu N with N_f = m (g cos(theta) phi_f + r h / L) and
 * N_r = m (g cos(theta) (1 - phi_f) - r h / L).  Then
 *     r = min(beta D, mu N_f / m) + min((1 - beta) D, mu N_r / m),
 * a piecewise-affine equation whose four pieces have slopes 0, +mu h/L,
 * -mu h/L, 0 in r (all below 1).  Each piece's own fixed point is
 *     D,  (mu gc phi_f + (1-beta) D) / (1 - mu h/L),
 *     (beta D + mu gc (1-phi_f)) / (1 + mu h/L),  mu gc,
 * and the fixed point of the minimum of affine maps with slope < 1 is the
 * minimum of their fixed points.  The divisions are taken once per sample:
 *     r = min(min(D, mg), min(f0 + f1 D, r0 + r1 D)).
 */
static double om_axle_cap_c(const om_consts *c, double D)
{
    if (c->cap_mode == OM_CAP_LUMPED) return dmin(D, c->cap);
    double lf = c->f0 + c->f1 * D;
    double lr = c->r0 + c->r1 * D;
    return dmin(dmin(D, c->mg), dmin(lf, lr));
}

/* dv/dt of Eq. 4 with the realised deceleration r: -r - k v^2 - g sin(theta). */
static double accel(const om_consts *c, double v, double a)
{
    double D = -a;
    double r = om_axle_cap_c(c, D);
    return ((-r) - (c->k * v) * v) - c->gs;
}

static int make_consts(const om_model *m, const double *const cols[OM_NFIELDS], uint64_t i,
                       om_consts *c)
{
    double v0 = cols[F_V0][i], d0 = cols[F_D0][i], mu = cols[F_MU][i];
    double gs = cols[F_GS][i], gc = cols[F_GC][i], mass = cols[F_MASS][i];
    double cd = cols[F_CD][i], tau = cols[F_TAU][i], td = cols[F_TDELAY][i];
    double noise = cols[F_NOISE][i];
    /* A sample is invalid if any field is not finite or a physical quantity
       has the wrong sign. */
    if (!isfinite(v0) || !isfinite(d0) || !isfinite(mu) || !isfinite(gs) || !isfinite(gc) ||
        !isfinite(mass) || !isfinite(cd) || !isfinite(tau) || !isfinite(td) || !isfinite(noise))
        return 0;
    if (!(mass > 0.0) || tau < 0.0 || mu < 0.0 || cd < 0.0 || td < 0.0) return 0;

    c->v0 = v0; c->d0 = d0; c->gs = gs; c->noise = noise; c->tau = tau;
    c->k = ((m->rho * cd) * m->area) / (2.0 * mass);
    c->it = (tau > 0.0) ? 1.0 / tau : 0.0;
    cap_coeffs(m, mu, gc, c);
    c->n_delay = om_steps_to_reach(td, m->dt);
    return 1;
}

/* Exposed for the per-axle brute-force pin. */
double om_axle_cap(const om_model *m, double mu, double gc, double D)
{
    om_consts c;
    memset(&c, 0, sizeof c);
    cap_coeffs(m, mu, gc, &c);
    return om_axle_cap_c(&c, D);
}

/*
 * Moving lead (extension; Sec. VIII names other road users as future work).
 * The lead starts d0 ahead of the ego car at speed lead_v0 and brakes at the
 * constant deceleration lead_decel until it stops, then stays put:
 *   x_L(t) = t (v_L0 - (b_L / 2) t)   for t < t_s = v_L0 / b_L,
 *   x_L(t) = (v_L0 t_s) / 2           for t >= t_s,
 *   v_L(t) = v_L0 - b_L t, then 0      (b_L = 0: t_s = infinity).
 * This is exact (no integration); the gap is g = (d0 + x_L(t)) - x.
 */
static double lead_pos(const om_model *m, double t)
{
    const double vl = m->lead_v0, bl = m->lead_decel;
    if (bl > 0.0) {
        const double ts = vl / bl;
        if (t >= ts) return 0.5 * (vl * ts);
    }
    return t * (vl - (0.5 * bl) * t);
}

static double lead_speed(const om_model *m, double t)
{
    const double vl = m->lead_v0, bl = m->lead_decel;
    if (bl > 0.0 && t >= vl / bl) return 0.0;
    return vl - bl * t;
}

/*
 * Per-step perception (extension; Sec. VIII names noise, latency and dropout
 * of the perception chain as future work), TTC trigger only.  The reading
 * taken at step k = n + L describes the state of step n (L = smallest integer
 * with L dt >= perc_latency).  Two consecutive readings share one
 * Philox-4x64-10 block, of counter (sample row, floor(k / 2), 0, 0) under key
 * (perc_seed, "PERCEPT1"): reading k takes the high 32-bit halves h_j of the
 * block's four words if k is even, the low halves if k is odd.  With the
 * uniforms u_j = h_j 2^-32, the reading is missing if u_4 < perc_drop, else
 * its noise is perc_sigma * 2 ((u_1 + u_2) + u_3 - 1.5): zero mean (to
 * 2^-32 perc_sigma), unit variance (Irwin-Hall of three uniforms, bounded by
 * +-3 perc_sigma, close to normal), so no transcendental function enters the
 * trigger decision.  (The paper fixes no generator; sharing a block between
 * two readings halves the work of drawing them.)
 */
static const uint64_t PERC_KEY1 = 0x5045524345505431ULL; /* "PERCEPT1" */

/* Returns 0 if the reading of step k is missing, else 1 and its noise. */
static int perception(const om_model *m, uint64_t row, int64_t k, double *noise)
{
    const double two_m32 = 1.0 / 4294967296.0; /* 2^-32 */
    uint64_t ctr[4] = {row, (uint64_t)k >> 1, 0, 0}, key[2] = {m->perc_seed, PERC_KEY1}, w[4];
    om_philox4x64_10(ctr, key, w);
    const int sh = (k & 1) ? 0 : 32; /* even k: high halves; odd k: low halves */
    double u1 = (double)((w[0] >> sh) & 0xffffffffULL) * two_m32;
    double u2 = (double)((w[1] >> sh) & 0xffffffffULL) * two_m32;
    double u3 = (double)((w[2] >> sh) & 0xffffffffULL) * two_m32;
    double u4 = (double)((w[3] >> sh) & 0xffffffffULL) * two_m32;
    if (u4 < m->perc_drop) return 0;
    *noise = m->perc_sigma * (2.0 * (((u1 + u2) + u3) - 1.5));
    return 1;
}

/* Exposed for the perception pins: 1 and the noise, or 0 if missing. */
int om_perception(const om_model *m, uint64_t row, int64_t k, double *noise)
{
    *noise = 0.0;
    return perception(m, row, k, noise);
}

/*
 * Test hook of the TTC trigger, used only to check the binary32 kernel's
 * trigger decisions (which may differ from these where the trigger margin is
 * within rounding of zero).  With force >= 0 the trigger fires at step
 * `force` exactly, with force == -1 never, in place of the margin test; with
 * force == -2 nothing is overridden.  For each step n in [lo, hi) at which the
 * trigger is still tested, the position x_n, the measured gap (with the range
 * noise and the reading's noise) and ttc_thr times the closing speed are
 * recorded, and whether the reading is present (steps not tested are left as
 * the caller set them).
 */
typedef struct {
    int64_t force;
    int64_t lo, hi;
    double *x;
    double *gap_meas;
    double *thr_closing;
    int8_t *reading;
} om_probe;

/*
 * One rollout (Sec. IV-D): classic RK4 on Eq. 7-9 with the command held over
 * the step, until contact, stop (v <= 0, Sec. V-D) or the horizon.
 *
 * Command (Eq. 2): a_cmd from the brake-onset step n_b on, 0 before it (the
 * car coasts under drag and grade during the reaction delay).
 *   immediate trigger: n_b = n_delay (the paper's setting has no delay, n_b = 0)
 *   TTC trigger: at the start of step n, while not yet triggered, the measured
 *   gap ((d0 + x_L(t_n)) - x_n) + noise is compared with ttc_thr times the
 *   closing speed v_n - v_L(t_n); the first step n_t where gap <= thr * closing
 *   speed sets n_b = n_t + n_delay (stationary lead: x_L = v_L = 0, TTC = H0 / v
 *   of Sec. VI-C).  With per-step perception the test at step n uses the
 *   reading of step n + L (plus its noise; none if it is missing) and then
 *   n_b = (n_t + L) + n_delay.
 * Actuator (Eq. 6): tau == 0 means an instantaneous actuator (a == command at
 * every stage).
 *
 * Termination after step n -> n+1, in this order: contact if a lead is
 * present and the gap (d0 + x_L(t_{n+1})) - x_{n+1} <= 0 (stationary lead:
 * x_{n+1} >= d0); stop if v_{n+1} <= 0; horizon if n+1 == N_max.
 * Outputs: n_onset = n_b once the command is issued (immediate trigger: always
 *   n_delay; TTC trigger: -1 if it never fires), x_raw = x_{n+1} (the paper's
 *   D_stop = x(t_stop), Eq. 3);
 *   stop:    s = v_n / (v_n - v_{n+1}),  x_ref = x_n + s (x_{n+1} - x_n)
 *   contact, stationary lead: s = (d0 - x_n) / (x_{n+1} - x_n), x_ref = d0,
 *            v_imp = v_n + s (v_{n+1} - v_n)
 *   contact, moving lead: with the gaps g_n, g_{n+1} and the closing speeds
 *            c_n = v_n - v_L(t_n), c_{n+1}: s = g_n / (g_n - g_{n+1}),
 *            x_ref = x_n + s (x_{n+1} - x_n), v_imp = c_n + s (c_{n+1} - c_n)
 *   t_end = (n + s) dt;  horizon: s = 1, x_ref = x_{n+1}.
 */
static void rollout_one(const om_model *m, const om_consts *c, uint64_t row, uint8_t *status,
                        double *x_raw, double *x_ref, double *v_imp, double *t_end,
                        int32_t *n_steps, int32_t *n_onset, const om_probe *pr)
{
    const double dt = m->dt;
    const double h2 = 0.5 * dt;
    const double h6 = dt / 6.0;
    const int64_t n_max = om_steps_to_reach(m->t_max, dt);

    double x = 0.0, v = c->v0, a = 0.0;
    *v_imp = 0.0;
    *n_onset = (m->trigger == OM_TRIGGER_IMMEDIATE) ? (int32_t)c->n_delay : -1;
    if (m->lead && c->d0 <= 0.0) {
        *status = OM_CONTACT; *x_raw = 0.0; *x_ref = 0.0; *v_imp = v;
        *t_end = 0.0; *n_steps = 0; return;
    }
    if (v <= 0.0) {
        *status = OM_STOP; *x_raw = 0.0; *x_ref = 0.0; *t_end = 0.0; *n_steps = 0; return;
    }
    if (n_max == 0) {
        *status = OM_HORIZON; *x_raw = 0.0; *x_ref = 0.0; *t_end = 0.0; *n_steps = 0; return;
    }

    int triggered = (m->trigger == OM_TRIGGER_IMMEDIATE);
    const int moving = m->lead && m->lead_v0 > 0.0;
    const int perc = m->perc_sigma > 0.0 || m->perc_drop > 0.0 || m->perc_latency > 0.0;
    const int64_t lat = perc ? om_steps_to_reach(m->perc_latency, dt) : 0;
    int64_t n_b = c->n_delay;
    for (int64_t n = 0;; ++n) {
        if (!triggered) {
            double gap_meas, closing;
            if (moving) {
                const double t = (double)n * dt;
                gap_meas = ((c->d0 + lead_pos(m, t)) - x) + c->noise;
                closing = v - lead_speed(m, t);
            } else {
                gap_meas = (c->d0 - x) + c->noise;
                closing = v;
            }
            int reading = 1;
            if (perc) {
                double pn = 0.0;
                reading = perception(m, row, n + lat, &pn);
                gap_meas = gap_meas + pn;
            }
            int fire = reading && gap_meas <= m->ttc_thr * closing;
            if (pr) {
                if (n >= pr->lo && n < pr->hi) {
                    const int64_t j = n - pr->lo;
                    pr->x[j] = x;
                    pr->gap_meas[j] = gap_meas;
                    pr->thr_closing[j] = m->ttc_thr * closing;
                    pr->reading[j] = (int8_t)reading;
                }
                if (pr->force != -2) fire = (n == pr->force);
            }
            if (fire) {
                triggered = 1; n_b = (n + lat) + c->n_delay;
                *n_onset = (n_b > 2147483647) ? 2147483647 : (int32_t)n_b;
            }
        }
        double u = (triggered && n >= n_b) ? m->a_cmd : 0.0;

        double a1, a2, a3, a4, ka1 = 0, ka2 = 0, ka3 = 0, ka4 = 0;
        if (c->tau > 0.0) {
            a1 = a;
            ka1 = (u - a1) * c->it;
            a2 = a + h2 * ka1;
            ka2 = (u - a2) * c->it;
            a3 = a + h2 * ka2;
            ka3 = (u - a3) * c->it;
            a4 = a + dt * ka3;
            ka4 = (u - a4) * c->it;
        } else {
            a1 = a2 = a3 = a4 = u;
        }
        double kv1 = accel(c, v, a1);
        double v2 = v + h2 * kv1;
        double kv2 = accel(c, v2, a2);
        double v3 = v + h2 * kv2;
        double kv3 = accel(c, v3, a3);
        double v4 = v + dt * kv3;
        double kv4 = accel(c, v4, a4);

        double xn = x + h6 * (((v + 2.0 * v2) + 2.0 * v3) + v4);
        double vn = v + h6 * (((kv1 + 2.0 * kv2) + 2.0 * kv3) + kv4);
        double an = (c->tau > 0.0) ? a + h6 * (((ka1 + 2.0 * ka2) + 2.0 * ka3) + ka4) : u;

        if (moving) {
            const double t0 = (double)n * dt, t1 = (double)(n + 1) * dt;
            const double g1 = (c->d0 + lead_pos(m, t1)) - xn;
            if (g1 <= 0.0) {
                const double g0 = (c->d0 + lead_pos(m, t0)) - x;
                const double c0 = v - lead_speed(m, t0), c1 = vn - lead_speed(m, t1);
                double s = g0 / (g0 - g1);
                *status = OM_CONTACT; *x_raw = xn; *x_ref = x + s * (xn - x);
                *v_imp = c0 + s * (c1 - c0);
                *t_end = ((double)n + s) * dt; *n_steps = (int32_t)(n + 1); return;
            }
        } else if (m->lead && xn >= c->d0) {
            double s = (c->d0 - x) / (xn - x);
            *status = OM_CONTACT; *x_raw = xn; *x_ref = c->d0;
            *v_imp = v + s * (vn - v);
            *t_end = ((double)n + s) * dt; *n_steps = (int32_t)(n + 1); return;
        }
        if (vn <= 0.0) {
            double s = v / (v - vn);
            *status = OM_STOP; *x_raw = xn; *x_ref = x + s * (xn - x);
            *t_end = ((double)n + s) * dt; *n_steps = (int32_t)(n + 1); return;
        }
        if (n + 1 >= n_max) {
            *status = OM_HORIZON; *x_raw = xn; *x_ref = xn;
            *t_end = (double)(n + 1) * dt; *n_steps = (int32_t)(n + 1); return;
        }
        x = xn; v = vn; a = an;
    }
}

int om_rollout(const om_model *m, const double *const cols[OM_NFIELDS], uint64_t row0, uint64_t n,
               uint8_t *status, double *x_raw, double *x_ref, double *v_imp, double *t_end,
               int32_t *n_steps, int32_t *n_onset)
{
    for (uint64_t i = 0; i < n; ++i) {
        om_consts c;
        if (!make_consts(m, cols, i, &c)) {
            status[i] = OM_INVALID; x_raw[i] = NAN; x_ref[i] = NAN; v_imp[i] = NAN;
            t_end[i] = NAN; n_steps[i] = 0; n_onset[i] = -1;
            continue;
        }
        rollout_one(m, &c, row0 + i, &status[i], &x_raw[i], &x_ref[i], &v_imp[i], &t_end[i],
                    &n_steps[i], &n_onset[i], NULL);
    }
    return 0;
}

/* One sample (column index i, perception row `row`) with the TTC test hook
 * `pr`; returns 0 (outputs untouched) if the sample is invalid. */
int om_rollout_probe(const om_model *m, const double *const cols[OM_NFIELDS], uint64_t i,
                     uint64_t row, const om_probe *pr, uint8_t *status, double *x_raw,
                     double *x_ref, double *v_imp, double *t_end, int32_t *n_steps,
                     int32_t *n_onset)
{
    om_consts c;
    if (!make_consts(m, cols, i, &c)) return 0;
    rollout_one(m, &c, row, status, x_raw, x_ref, v_imp, t_end, n_steps, n_onset, pr);
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Reduction (Sec. VI-B, VI-C): counts, moments, extremes, fixed-bin          */
/* histograms.  Sums run in sample order.  Bin j of a histogram with origin   */
/* lo and width w holds floor((x - lo) / w) == j, with the index clamped to   */
/* [0, nbins - 1].                                                            */
/* ------------------------------------------------------------------------- */

static int64_t bin_of(double x, double lo, double w, int64_t nb)
{
    double q = floor((x - lo) / w);
    if (q < 0.0) return 0;
    if (q > (double)(nb - 1)) return nb - 1;
    return (int64_t)q;
}

int om_reduce(uint64_t n, const uint8_t *status, const double *x_ref, const double *v_imp,
              const int32_t *n_steps, om_stats *st,
              uint64_t *hist_d, double lo_d, double w_d,
              uint64_t *hist_v, double lo_v, double w_v, int64_t nbins)
{
    memset(st, 0, sizeof *st);
    st->min_d = INFINITY; st->max_d = -INFINITY;
    st->min_v = INFINITY; st->max_v = -INFINITY;
    for (int64_t j = 0; j < nbins; ++j) { hist_d[j] = 0; hist_v[j] = 0; }
    st->n = n;
    for (uint64_t i = 0; i < n; ++i) {
        st->steps += (uint64_t)n_steps[i];
        if (status[i] == OM_STOP) {
            double d = x_ref[i];
            st->n_stop++;
            st->sum_d += d;
            st->sumsq_d += d * d;
            if (d < st->min_d) st->min_d = d;
            if (d > st->max_d) st->max_d = d;
            hist_d[bin_of(d, lo_d, w_d, nbins)]++;
        } else if (status[i] == OM_CONTACT) {
            double vi = v_imp[i];
            st->n_contact++;
            st->sum_v += vi;
            st->sumsq_v += vi * vi;
            if (vi < st->min_v) st->min_v = vi;
            if (vi > st->max_v) st->max_v = vi;
            hist_v[bin_of(vi, lo_v, w_v, nbins)]++;
        } else if (status[i] == OM_HORIZON) {
            st->n_horizon++;
        } else {
            st->n_invalid++;
        }
    }
    return 0;
}
