/*
 * aeb.h -- C ABI of the GB300 Monte Carlo AEB braking library (libaeb.so).
 *
 * The library evaluates independent Monte Carlo emergency-braking rollouts of a
 * longitudinal vehicle model and reduces them to stopping, collision and
 * impact-speed statistics, after Karjol & Alawneh, "Real-Time GPU-Accelerated
 * Monte Carlo Evaluation of Safety-Critical AEB Systems Under Uncertainty":
 *   model ................ Sec. III, Eq. 1-9 (drag, grade, weight transfer, lag)
 *   sampling ............. Sec. IV-A..IV-C, Eq. 10-15 (seeded, on the host)
 *   integration .......... Sec. IV-D (fixed-step RK4), Sec. V-D (v <= 0)
 *   one rollout per lane . Sec. V-A..V-C
 *   statistics ........... Sec. VI-B (mean, std, range), Sec. VI-C, Eq. 19
 *                          (P(D_stop > H0), safe headways)
 * The lead vehicle, reaction delay, range noise, per-axle friction caps and
 * the TTC trigger extend the paper's model; each struct field says so.
 *
 * Conventions for every entry point:
 *   - Plain C types only; pointers are host or device as each argument says.
 *   - Buffers passed in are owned by the caller and never freed or retained by
 *     the library after the call's stream work completes.  Library-owned
 *     scratch is allocated on first use per device and reused.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls marked
 *     "asynchronous" only enqueue work on it; results are valid once the
 *     stream has reached that point.
 *   - Every call returns an aeb_status; on failure aeb_last_error() gives a
 *     message (thread-local, valid until the next call on the same thread).
 *     Invalid arguments never reach the GPU.
 */
#ifndef AEB_H
#define AEB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AEB_ABI_VERSION 6
#define AEB_NFIELDS 10   /* columns of a parameter set, see aeb_params       */
#define AEB_NBINS 4096   /* bins of each fixed histogram in aeb_stats         */

/* ---- status codes ------------------------------------------------------- */
typedef int32_t aeb_status;
enum {
    AEB_OK = 0,
    AEB_EINVAL = 1,      /* an argument is out of its documented domain       */
    AEB_ENOMEM = 2,      /* host or device allocation failed                   */
    AEB_ECUDA = 3,       /* a CUDA runtime call failed (message says which)   */
    AEB_ETIMEOUT = 4,    /* a bounded wait ran out                             */
    AEB_EAGAIN = 5,      /* result not ready yet                               */
    AEB_ECANCELLED = 6,  /* the request was cancelled                          */
    AEB_EDEVICE = 7      /* no usable CUDA device / wrong architecture         */
};

/* ---- enumerations ------------------------------------------------------- */
typedef int32_t aeb_precision;
enum {
    AEB_FP64_PLAIN = 0,  /* binary64, no fused multiply-add: bit-identical to
                            the plain CPU definition (Sec. V-D)               */
    AEB_FP32_COMP = 1    /* binary32 stages with compensated (double-float)
                            position and speed; FP64 stop/contact refinement  */
};
enum { AEB_CAP_LUMPED = 0, AEB_CAP_PER_AXLE = 1 };
enum { AEB_TRIGGER_IMMEDIATE = 0, AEB_TRIGGER_TTC = 1 };
enum { AEB_STOP = 0, AEB_CONTACT = 1, AEB_HORIZON = 2, AEB_INVALID = 255 };
enum { AEB_DIST_CONST = 0, AEB_DIST_UNIFORM = 1, AEB_DIST_NORMAL = 2 };
enum { AEB_HIST_D = 0, AEB_HIST_V = 1 };  /* stopping-distance / impact-speed histogram */

/* ---- model constants (Sec. III, Sec. IV-B) ------------------------------- */
typedef struct aeb_model {
    double g;          /* gravitational acceleration [m/s^2]                      */
    double rho;        /* air density [kg/m^3] (Eq. 4)                            */
    double area;       /* frontal area A_f [m^2] (Eq. 4)                          */
    double h_cg;       /* centre-of-gravity height h [m] (Eq. 5)                  */
    double wheelbase;  /* wheelbase L [m] (Eq. 5)                                 */
    double beta;       /* front share of the demanded brake force (per-axle caps) */
    double phi_f;      /* static front share of the normal load (per-axle caps)   */
    double a_cmd;      /* commanded braking acceleration, negative [m/s^2] (Eq. 2) */
    double dt;         /* RK4 step [s] (Sec. IV-B), > 0                            */
    double t_max;      /* horizon [s] (Sec. IV-B), >= 0                            */
    double ttc_thr;    /* TTC trigger threshold [s] (TTC = H0 / v, Sec. VI-C)     */
    int32_t cap_mode;  /* AEB_CAP_LUMPED: Eq. 5 as printed, r <= mu g/(1+mu h/L);
                          AEB_CAP_PER_AXLE: front/rear forces capped at mu N per
                          axle with weight transfer (extension)                  */
    int32_t trigger;   /* AEB_TRIGGER_IMMEDIATE: brake after the reaction delay;
                          AEB_TRIGGER_TTC: brake once the measured gap
                          (gap + noise) <= ttc_thr * closing speed, then the
                          delay (stationary lead: d0 - x + noise <= thr * v)    */
    int32_t lead;      /* 1: lead vehicle, initially d0 ahead (contact ends a run) */
    int32_t reserved;  /* must be 0                                             */
    /* Moving lead (extension; the paper's lead is stationary).  The lead starts
       at lead_v0 and brakes at the constant lead_decel until it stops:
       x_L(t) = t (v_L0 - lead_decel t / 2) up to t_s = v_L0 / lead_decel, then
       constant; the gap is (d0 + x_L(t)) - x and the impact speed reported for
       a contact is the closing speed v - v_L.  lead_v0 = 0: stationary lead.
       Both finite and >= 0, else AEB_EINVAL.                                   */
    double lead_v0;    /* initial speed of the lead [m/s]                       */
    double lead_decel; /* braking deceleration of the lead [m/s^2]              */
    /* Per-step perception of the TTC trigger's readings (extension).  The
       reading used at step n is taken L steps later (L = smallest integer with
       L dt >= perc_latency) and describes step n; it is missing with
       probability perc_drop (u4 < perc_drop), else carries the noise
       perc_sigma * 2 ((u1 + u2) + u3 - 1.5) (zero mean, unit variance, within
       +-3 perc_sigma), u_j = h_j 2^-32, h_j the high 32-bit halves (k = n + L
       even) or the low halves (k odd) of the four words of the Philox-4x64-10
       block of counter (parameter row, floor(k / 2), 0, 0) under key
       (perc_seed, 0x5045524345505431).
       A trigger at step n starts braking at n + L + n_delay.  All zero: the
       plain trigger.  perc_sigma, perc_latency finite and >= 0, perc_drop in
       [0, 1], else AEB_EINVAL.                                                 */
    double perc_sigma;   /* noise scale of a reading [m]                         */
    double perc_drop;    /* probability that a step's reading is missing         */
    double perc_latency; /* age of a reading when it is used [s]                 */
    uint64_t perc_seed;  /* key of the per-step reading stream                   */
} aeb_model;

/* ---- sampling description (Sec. IV-A, IV-C) ------------------------------ */
typedef struct aeb_dist {
    int32_t kind;      /* AEB_DIST_*                                             */
    int32_t reserved;  /* must be 0                                             */
    double p0, p1;     /* const: p0 | uniform: [p0, p1) | normal: mean p0, sd p1  */
    double lo, hi;     /* every draw is clamped to [lo, hi] (+-inf: no clamp)    */
} aeb_dist;

typedef struct aeb_scenario {
    aeb_dist v0;       /* initial speed [m/s]                 (Eq. 11)          */
    aeb_dist d0;       /* initial gap to the lead [m]         (extension)       */
    aeb_dist mu;       /* tyre-road friction coefficient      (Eq. 12)          */
    aeb_dist grade;    /* road grade angle [rad]              (Eq. 13)          */
    aeb_dist mass;     /* vehicle mass [kg]                   (Eq. 14)          */
    aeb_dist cd;       /* drag coefficient                    (Eq. 15)          */
    aeb_dist tau;      /* actuator time constant [s]          (Eq. 6)           */
    aeb_dist t_delay;  /* reaction delay before braking [s]   (extension)       */
    aeb_dist noise;    /* constant range-measurement bias [m] (extension)       */
    uint64_t seed;     /* Philox-4x64-10 key word 0                             */
    uint64_t scenario_id; /* Philox-4x64-10 key word 1                          */
} aeb_scenario;

/* Structure-of-arrays parameter sets xi^(i) (Eq. 10): ten float64 columns of
 * the same length, sample i at index i of each.  gs = g sin(theta) and
 * gc = g cos(theta) are taken on the host so the device never evaluates a
 * transcendental.  Columns are host or device memory as each call states;
 * each column must be 8-byte aligned. */
typedef struct aeb_params {
    double *v0, *d0, *mu, *gs, *gc, *mass, *cd, *tau, *t_delay, *noise;
} aeb_params;

/* Per-sample outputs, one entry per sample.  Any pointer may be NULL (that
 * output is not stored); aeb_reduce needs status, x_ref, v_imp, n_steps.
 *   status  AEB_STOP / AEB_CONTACT / AEB_HORIZON / AEB_INVALID
 *   x_raw   x at the end of the terminating step: the paper's D_stop (Eq. 3)
 *   x_ref   position at the refined stop or contact instant (contact: d0)
 *   v_imp   speed at contact (0 unless AEB_CONTACT)
 *   t_end   refined time of the stop / contact / horizon [s]
 *   n_steps RK4 steps executed
 *   n_onset first step with the braking command applied (-1: never issued)
 * Invalid samples (non-finite field, mass <= 0, tau/mu/cd/t_delay < 0) get
 * AEB_INVALID, NaN values and n_steps = 0. */
typedef struct aeb_outputs {
    uint8_t *status;
    double *x_raw, *x_ref, *v_imp, *t_end;
    int32_t *n_steps, *n_onset;
} aeb_outputs;

/* Fixed-bin histograms: bin j of D holds floor((x_ref - lo_d) / w_d) == j over
 * stopped samples, bin j of V the same for v_imp over contact samples, the
 * index clamped to [0, AEB_NBINS - 1].  Widths must be powers of two. */
typedef struct aeb_hist_spec {
    double lo_d, w_d, lo_v, w_v;
} aeb_hist_spec;

/* Reduction of a set of outputs (Sec. VI-B, VI-C). */
typedef struct aeb_stats {
    uint64_t n, n_stop, n_contact, n_horizon, n_invalid;
    uint64_t steps;                       /* sum of n_steps                    */
    double sum_d, sumsq_d, min_d, max_d;  /* x_ref over stopped samples        */
    double sum_v, sumsq_v, min_v, max_v;  /* v_imp over contact samples        */
    double lo_d, w_d, lo_v, w_v;          /* the histogram spec used           */
    uint64_t hist_d[AEB_NBINS];
    uint64_t hist_v[AEB_NBINS];
} aeb_stats;

/* One job of a batched launch (many scenarios with uneven sample counts in
 * one persistent launch): its parameters are rows
 * [param_offset, param_offset + n) of the device columns, its outputs rows
 * [out_offset, out_offset + n) of the output columns; ttc_thr is its own TTC
 * threshold (used when model.trigger is AEB_TRIGGER_TTC); sample j of the job
 * draws its per-step perception readings from row key_offset + j of the
 * reading stream (a plain aeb_rollout uses the parameter row). */
typedef struct aeb_job {
    uint64_t param_offset;
    uint64_t out_offset;
    uint64_t n;
    double ttc_thr;
    uint64_t key_offset;
} aeb_job;

/* Per-job reduction of a batched launch: aeb_stats without the histograms. */
typedef struct aeb_job_stats {
    uint64_t n, n_stop, n_contact, n_horizon, n_invalid, steps;
    double sum_d, sumsq_d, min_d, max_d;  /* x_ref over stopped samples */
    double sum_v, sumsq_v, min_v, max_v;  /* v_imp over contact samples */
} aeb_job_stats;

/* Launch shape of the rollout kernels (chosen by aeb_autotune or set). */
typedef struct aeb_launch_config {
    int32_t tile;           /* samples per warp tile: 32..256, multiple of 32   */
    int32_t blocks_per_sm;  /* resident blocks per SM (0: as many as fit)       */
} aeb_launch_config;

/* Opaque batched-launch plan (device tables + captured CUDA graph). */
typedef struct aeb_batch aeb_batch;

/* Serving engine configuration (continuous batching of requests; the 530 ms
 * budget of Sec. VI-F). */
typedef struct aeb_serve_cfg {
    aeb_precision precision;      /* rollout precision of every request               */
    int32_t device;               /* CUDA device ordinal                              */
    uint64_t arena_rows;          /* device rows for resident requests (admission
                                     budget; 101 B of device memory per row)          */
    uint64_t chunk_samples;       /* fixed chunk a request is cut into (multiple of 64) */
    uint64_t wave_samples;        /* samples launched per wave, at most               */
    int32_t max_waves_in_flight;  /* waves queued on the GPU at once (1..4)           */
    int32_t sampler_threads;      /* host sampling threads (<= 0: all)                */
    uint64_t max_request_samples; /* larger requests are rejected (<= arena_rows)     */
    int32_t wave_timeout_ms;      /* watchdog: a wave not complete this long after its
                                     launch fails its requests with AEB_ETIMEOUT
                                     (0: 10,000 ms; < 0: no watchdog)                 */
    int32_t reserved;             /* must be 0                                        */
} aeb_serve_cfg;

/* Per-request timing, milliseconds. */
typedef struct aeb_latency {
    double queue_ms;   /* submit -> admitted (arena rows granted)                */
    double sample_ms;  /* admitted -> parameters resident on the GPU            */
    double gpu_ms;     /* resident -> statistics ready on the host              */
    double total_ms;   /* submit -> statistics ready                            */
} aeb_latency;

/* Engine counters since creation. */
typedef struct aeb_serve_counters {
    uint64_t submitted, completed, cancelled, failed, rollouts, waves;
    uint64_t timed_out;   /* failed requests that the wave watchdog ended       */
    uint64_t rows_free;   /* arena rows not held by any request (now)           */
} aeb_serve_counters;

/* Host-side fault injection into a serving engine, for testing its failure
 * handling without any GPU fault (aeb_serve_inject_faults).  Counts are
 * 1-based from the call (0: no fault); each fires once. */
typedef struct aeb_serve_faults {
    uint64_t fail_admission;        /* the k-th admission finds no rows: AEB_ENOMEM     */
    uint64_t fail_wave_launch;      /* the k-th wave's launch reports a CUDA error      */
    uint64_t fail_wave_completion;  /* the k-th wave launched completes with an error   */
    int32_t hold_waves_ms;          /* every wave's completion is seen this late (>= 0) */
    int32_t reserved;               /* must be 0                                        */
} aeb_serve_faults;

/* Opaque serving engine. */
typedef struct aeb_server aeb_server;

/* Weighted event sums of an importance-sampled set (aeb_reduce_weighted). */
typedef struct aeb_wstats {
    uint64_t n, n_valid, n_event;  /* samples, valid samples, valid samples in E   */
    double sum_w, sumsq_w;         /* sum of w and of w^2 over valid samples       */
    double sum_we, sumsq_we;       /* sum of w 1[E] and of (w 1[E])^2              */
} aeb_wstats;

/* Summary of a reduction (Sec. VI-B, Table I: mean, standard deviation and
 * range of the stopping distance; the collision probability).  Means and
 * unbiased standard deviations come from the sums of the statistics:
 * m = s / k, sd = sqrt((ss - (k m) m) / (k - 1)) (negative variance from
 * cancellation clamped to 0).  Fields of an empty set are NaN; sd needs two
 * values. */
typedef struct aeb_summary {
    uint64_t n, n_valid;                   /* samples; n - n_invalid          */
    uint64_t n_stop, n_contact, n_horizon, n_invalid;
    uint64_t steps;                        /* RK4 steps executed in total     */
    double mean_steps;                     /* steps / n                       */
    double mean_d, std_d, min_d, max_d;    /* x_ref over stopped samples [m]  */
    double mean_v, std_v, min_v, max_v;    /* v_imp over contact samples [m/s] */
    double p_contact;                      /* n_contact / n_valid             */
    double p_contact_lo, p_contact_hi;     /* 95 % Wilson score interval      */
} aeb_summary;

/* A probability estimated from k events in n trials, with its 95 % Wilson
 * score interval. */
typedef struct aeb_prob {
    uint64_t k, n;
    double p;              /* k / n (NaN if n == 0)                          */
    double ci_lo, ci_hi;
} aeb_prob;

/* Importance-sampling estimate of an event probability under the nominal
 * scenario (aeb_is_estimate). */
typedef struct aeb_is_result {
    uint64_t n, n_event;   /* samples, valid samples in the event             */
    double p;              /* sum_we / n                                      */
    double se;             /* standard error (NaN below two samples)          */
    double ci_lo, ci_hi;   /* p -+ 1.959963984540054 se                       */
} aeb_is_result;

/* Collision probability at one TTC threshold, pooled over the scenarios
 * (Sec. VI-C, Eq. 19 with the TTC = H0 / v criterion). */
typedef struct aeb_sweep_result {
    double threshold;
    uint64_t n, n_contact, n_stop, n_horizon, n_invalid;
    double p_contact;      /* n_contact / (n - n_invalid)                       */
    double ci_lo, ci_hi;   /* 95 % Wilson score interval of p_contact           */
} aeb_sweep_result;

/* ---- entry points -------------------------------------------------------- */

/* ABI version of the loaded library (AEB_ABI_VERSION when it was built). */
int32_t aeb_abi_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char *aeb_last_error(void);

/*
 * aeb_sample_params -- draw parameter sets xi^(first) .. xi^(first+n-1)
 * (Sec. IV-A, IV-C: random numbers drawn on the host from a fixed seed).
 * Sample i, quantity q uses Philox-4x64-10 block (counter (i, q/2, 0, 0),
 * key (seed, scenario_id)), words 0-1 for even q and 2-3 for odd q, in the
 * quantity order of aeb_scenario.  Uniform: p0 + (p1 - p0) U, U = (w0>>11)
 * 2^-53.  Normal: p0 + p1 sqrt(-2 ln U1) cos(2 pi U2), U1 = ((w0>>11)+1) 2^-53,
 * U2 = (w1>>11) 2^-53.  Then clamp.  gs, gc = g sin(grade), g cos(grade).
 *   model    host; only model->g is read
 *   out      host columns (caller-owned, >= n doubles each)
 *   n_threads host threads to use (<= 0: all hardware threads)
 * Synchronous, host only.  Output is independent of n_threads.
 * AEB_EINVAL: NULL pointer, unknown distribution kind, non-finite parameter.
 */
aeb_status aeb_sample_params(const aeb_model *model, const aeb_scenario *scenario,
                             uint64_t first, uint64_t n, const aeb_params *out,
                             int32_t n_threads);

/*
 * aeb_sample_params_is -- importance sampling (extension: rare-event
 * estimation of low collision probabilities), first half: draw parameter sets
 * from `proposal` exactly as aeb_sample_params does and write each set's
 * likelihood ratio w = p(xi) / q(xi) to `nominal`: the product over the
 * quantities of, for the clamped value x, 1 for a constant, the ratio of the
 * probability masses the two laws put at a clamp bound if x sits on one that
 * holds mass under q, else the ratio of the densities (uniform:
 * 1[a_p <= x < b_p] (b_q - a_q) / (b_p - a_p); normal: (s_q / s_p)
 * exp((z_q^2 - z_p^2) / 2)).  Then E_q[w f] = E_p[f] for any outcome f.
 *   weights  host array of n doubles (caller-owned)
 * Synchronous, host only; independent of n_threads.  AEB_EINVAL: NULL pointer,
 * invalid distribution, or a proposal incompatible with `nominal` (per
 * quantity: same kind and clamp bounds, equal constants, a uniform proposal
 * covering the nominal interval, positive normal sds).
 */
aeb_status aeb_sample_params_is(const aeb_model *model, const aeb_scenario *nominal,
                                const aeb_scenario *proposal, uint64_t first, uint64_t n,
                                const aeb_params *out, double *weights, int32_t n_threads);

/*
 * aeb_reduce_weighted -- importance sampling, second half: over valid samples,
 * the sums of w, w^2, w 1[E] and (w 1[E])^2 for the event E = contact, or
 * x_ref > x_thr (P(D_stop > H0), Sec. VI-C; x_thr = +inf: contact only).
 * Then sum_we / n estimates the nominal probability of E without bias, with
 * standard error sqrt((sumsq_we / n - p^2) / (n - 1)).
 *   out      DEVICE outputs; status and x_ref required
 *   weights  DEVICE array of n likelihood ratios (aeb_sample_params_is)
 *   stats    DEVICE aeb_wstats written (fixed summation order: the same bits
 *            for the same inputs)
 * Asynchronous on `stream`.  AEB_EINVAL: NULL pointers, misaligned stats, NaN
 * x_thr.
 */
aeb_status aeb_reduce_weighted(const aeb_outputs *out, const double *weights, uint64_t n,
                               double x_thr, aeb_wstats *stats, void *stream);


/*
 * aeb_rollout -- integrate every sample until contact, stop or horizon
 * (Sec. IV-D RK4 of Eq. 7-9, termination Sec. V-D) and write per-sample
 * outputs.  One CUDA lane owns one rollout at a time (Sec. V-A); lanes whose
 * rollout ends pick up the next sample of their warp's tile.
 *   model      host
 *   params     device columns, n entries each (caller-owned)
 *   precision  AEB_FP64_PLAIN: every output bit-identical to the plain binary64
 *              definition; AEB_FP32_COMP: see the precision enum
 *   out        device columns (caller-owned; NULL members are skipped)
 *   stream     cudaStream_t
 * Asynchronous.  n == 0 is a no-op.
 * AEB_EINVAL: NULL params column, bad model (non-finite constant, dt <= 0,
 * t_max < 0, t_max/dt beyond 2^31 - 2 steps, unknown mode, reserved != 0,
 * wheelbase <= 0), unknown precision, misaligned column.
 * AEB_ECUDA / AEB_EDEVICE on launch failure.
 */
aeb_status aeb_rollout(const aeb_model *model, const aeb_params *params, uint64_t n,
                       aeb_precision precision, const aeb_outputs *out, void *stream);

/*
 * aeb_reduce -- counts, moments, extremes and fixed-bin histograms of a set of
 * outputs (Sec. VI-B; Sec. VI-C reads P(D_stop > H0) off hist_d at bin edges).
 * Sums are taken in a fixed order that depends only on n, so repeated calls
 * give identical bits.
 *   out        device columns status, x_ref, v_imp, n_steps (n entries)
 *   hist       host
 *   stats      DEVICE pointer to one aeb_stats (caller-owned, 8-byte aligned)
 * Asynchronous.  Uses library scratch on the stream's device.
 * AEB_EINVAL: NULL column, width not a positive power of two, non-finite lo.
 */
aeb_status aeb_reduce(const aeb_outputs *out, uint64_t n, const aeb_hist_spec *hist,
                      aeb_stats *stats, void *stream);

/*
 * aeb_reduce_noalloc -- aeb_reduce without any device allocation, for callers
 * that must not allocate once running (a real-time loop whose rules forbid
 * allocation after start-up, or a process whose device memory is already held
 * in full by another allocator).  The paper has no counterpart; this is a
 * deployment variant of aeb_reduce.
 *   Same arguments, ordering and results as aeb_reduce, for
 *   n <= AEB_REDUCE_NOALLOC_MAX_N samples; larger n is rejected with
 *   AEB_EINVAL and a message naming the limit.
 *   Scratch: a fixed array of per-block partial sums compiled into the library
 *   (26.6 KB on every GPU that loads it, held until the process exits).  All
 *   calls share it, so calls whose GPU work overlaps (for example on two
 *   streams) race and must be serialised by the caller.  Each call overwrites
 *   the partials it reads and clears the histogram of `stats` first.
 *   The first call on a device looks up the array's device address (no
 *   allocation); make that first call before any stream capture.
 * Asynchronous.  Calls no cudaMalloc, cudaFree or allocating routine.
 */
#define AEB_REDUCE_NOALLOC_MAX_N 2097152u
aeb_status aeb_reduce_noalloc(const aeb_outputs *out, uint64_t n, const aeb_hist_spec *hist,
                              aeb_stats *stats, void *stream);

/*
 * aeb_evaluate -- the whole path from host buffers: copy the parameter columns
 * to device buffers owned by the library, roll out, reduce, copy the stats
 * (and the requested per-sample outputs) back, and wait for the stream.
 *   params      HOST columns (pinned memory gives the fastest copies)
 *   host_stats  host aeb_stats written on success
 *   host_out    host columns for per-sample outputs, or NULL / NULL members
 * Above 2^19 samples the upload is cut into chunks of growing length (2^18
 * samples first, then each a factor g longer than the one before), each
 * rolled out as soon as it has arrived, on internal streams ordered after the
 * work already queued on `stream`.  g is 2 on the first call on a stream;
 * each call times its uploads and its first chunk's rollouts and sets g for
 * the next call on that stream (within [1.25, 4]), so that a chunk's upload
 * ends before the previous chunk's rollouts on this machine's copy rate.
 * Results are the same bits as one aeb_rollout + aeb_reduce of all n samples
 * (sample i keeps row i for its perception readings), whatever the chunks.
 * The device buffers, internal streams and events are kept per (device,
 * stream) and grown as needed until the process exits; calls on the same
 * stream from several threads must be serialised by the caller.
 * Synchronous.  AEB_ENOMEM if the device buffers cannot be grown.
 */
aeb_status aeb_evaluate(const aeb_model *model, const aeb_params *params, uint64_t n,
                        aeb_precision precision, const aeb_hist_spec *hist,
                        aeb_stats *host_stats, const aeb_outputs *host_out, void *stream);

/*
 * aeb_evaluate_scenario -- the whole path from the seed (Sec. IV-C sampling,
 * then the rollout and reduction of aeb_evaluate): samples first .. first+n-1
 * of `scenario` are drawn on the host in chunks of 2^20 into pinned staging
 * buffers owned by the library, and each chunk is uploaded and rolled out
 * while the host draws the next one; then the reduction and the copy of the
 * stats back.  Results are the same bits as aeb_sample_params(first, n) into
 * host columns followed by aeb_evaluate of those n samples (sample i keeps row
 * i for its perception readings).
 *   n_threads   host sampling threads (0: all hardware threads)
 *   host_stats  host aeb_stats written on success
 * The device buffers, two staging buffers of 2^20 samples, internal streams
 * and events are kept per (device, stream) as for aeb_evaluate; calls on the
 * same stream from several threads must be serialised by the caller.
 * Synchronous.  AEB_EINVAL for a bad model, scenario, precision or histogram
 * spec (nothing runs); AEB_ENOMEM if the buffers cannot be grown.
 */
aeb_status aeb_evaluate_scenario(const aeb_model *model, const aeb_scenario *scenario,
                                 uint64_t first, uint64_t n, aeb_precision precision,
                                 const aeb_hist_spec *hist, int32_t n_threads,
                                 aeb_stats *host_stats, void *stream);

/*
 * aeb_batch_create -- plan a batched launch over n_jobs jobs (the per-sample
 * method is that of aeb_rollout, Sec. IV-D, V-A..V-D).  Builds
 * the table of (job, tile) work items, allocates the device tables and
 * scratch (owned by the plan), and captures one CUDA graph: reset of the work
 * counter, one persistent rollout launch over all tiles, and the per-job
 * fixed-order reduction into stats[0 .. n_jobs).
 *   jobs       host array (copied)
 *   params     device columns (caller-owned; must outlive the plan)
 *   out        device output columns covering every job's out rows; status,
 *              x_ref, v_imp and n_steps are required
 *   stats      DEVICE array of n_jobs aeb_job_stats (caller-owned)
 * The launch shape is the library's current configuration for `precision`.
 * Synchronous (allocation, table upload, capture).  AEB_EINVAL on bad
 * arguments (n_jobs == 0, NULL columns, a job with n > 2^32 - 1 tiles).
 */
aeb_status aeb_batch_create(const aeb_model *model, const aeb_job *jobs, uint32_t n_jobs,
                            const aeb_params *params, aeb_precision precision,
                            const aeb_outputs *out, aeb_job_stats *stats, aeb_batch **plan);

/* aeb_batch_run -- launch the plan's graph on `stream` (asynchronous).  A plan
 * may be run any number of times; runs of one plan must not overlap. */
aeb_status aeb_batch_run(aeb_batch *plan, void *stream);

/* aeb_batch_destroy -- wait for the plan's work and free it (NULL is a no-op). */
void aeb_batch_destroy(aeb_batch *plan);

/*
 * aeb_rollout_batched -- create, run once on `stream` and destroy a plan
 * (synchronous: returns when the stats are written).
 */
aeb_status aeb_rollout_batched(const aeb_model *model, const aeb_job *jobs, uint32_t n_jobs,
                               const aeb_params *params, aeb_precision precision,
                               const aeb_outputs *out, aeb_job_stats *stats, void *stream);

/* Launch shape in use for `precision` (get / set).  Setting validates the
 * shape (AEB_EINVAL) and applies to later launches and plans. */
aeb_status aeb_get_launch_config(aeb_precision precision, aeb_launch_config *cfg);
aeb_status aeb_set_launch_config(aeb_precision precision, const aeb_launch_config *cfg);

/*
 * aeb_autotune -- time the rollout of the first n samples of `params` under
 * each candidate shape (tile 32/64/128 x blocks per SM 3..8 that fit), keep the
 * fastest for `precision` and return it in *best.  If cache_path is not NULL,
 * a shape recorded there for this device, precision and model mode is used
 * without timing, and a newly timed one is recorded.  Synchronous; writes the
 * outputs of the timed runs into `out`.
 */
aeb_status aeb_autotune(const aeb_model *model, const aeb_params *params, uint64_t n,
                        aeb_precision precision, const aeb_outputs *out, void *stream,
                        const char *cache_path, aeb_launch_config *best);

/*
 * aeb_serve_create -- start a serving engine on cfg->device for `model`
 * (continuous batching of scenario requests, latency against the 530 ms
 * Monte Carlo budget of Sec. VI-F).  A request is a scenario and a
 * sample count; the engine samples it on the host (Sec. IV-C), keeps its
 * parameters and outputs resident in a device arena, cuts it into fixed
 * chunks and runs chunks of all admitted requests together in waves (one
 * persistent launch each; consecutive waves overlap on two streams).  A
 * request's statistics are the fixed-order combination of its chunks' and do
 * not depend on what it shares waves with.
 * Allocates the arena, pinned staging and wave buffers, and starts two host
 * threads.  AEB_EINVAL on a bad configuration, AEB_ENOMEM if the arena cannot
 * be allocated.
 */
aeb_status aeb_serve_create(const aeb_serve_cfg *cfg, const aeb_model *model, aeb_server **out);

/* Queue a request; returns its ticket.  Thread-safe.  AEB_EINVAL for n == 0,
 * n > max_request_samples or an invalid scenario. */
aeb_status aeb_serve_submit(aeb_server *srv, const aeb_scenario *scenario, uint64_t n,
                            uint64_t *ticket);

/*
 * Wait up to timeout_ms (0: do not wait, < 0: no limit) for a request.  On
 * AEB_OK the statistics and latency are written and the ticket is released.
 * AEB_EAGAIN (timeout_ms == 0) or AEB_ETIMEOUT if still running (the ticket
 * stays valid), AEB_ECANCELLED if cancelled, AEB_EINVAL for an unknown ticket.
 * A failed request releases its ticket and returns its error: AEB_ENOMEM (no
 * arena rows could be granted), AEB_ECUDA (a wave holding one of its chunks
 * failed), AEB_ETIMEOUT (the wave watchdog, see wave_timeout_ms; the message
 * says which).  Thread-safe.
 */
aeb_status aeb_serve_poll(aeb_server *srv, uint64_t ticket, int32_t timeout_ms,
                          aeb_job_stats *stats, aeb_latency *lat);

/* Cancel a request not yet admitted (an admitted one runs to the end and its
 * result is discarded).  AEB_EINVAL for an unknown ticket. */
aeb_status aeb_serve_cancel(aeb_server *srv, uint64_t ticket);

/* Engine counters (thread-safe snapshot). */
aeb_status aeb_serve_counters_get(aeb_server *srv, aeb_serve_counters *out);

/*
 * aeb_serve_inject_faults -- make the engine's next admissions or waves fail
 * on the host, to test the failure handling (no GPU fault is made: an
 * injected launch error skips the launch, an injected completion error or
 * hold replaces what the wave's finished event reports).  The paper has no
 * counterpart; it supports the serving loop of Sec. VI-F.  Whatever fails, a
 * failed request's queued chunks are dropped and its arena rows return once
 * none of its chunks is on the GPU (counters.rows_free shows them back);
 * other requests carry on.  Replaces any earlier injection.  Thread-safe.
 * AEB_EINVAL: NULL argument, hold_waves_ms < 0, reserved != 0.
 */
aeb_status aeb_serve_inject_faults(aeb_server *srv, const aeb_serve_faults *faults);

/* Stop the engine after the work in flight, release everything (NULL: no-op). */
void aeb_serve_destroy(aeb_server *srv);

/*
 * aeb_ttc_sweep -- collision probability against the TTC trigger threshold
 * (TTC = H0 / v_rel, Sec. VI-C).  Samples n_per_scenario
 * parameter sets of every scenario once on the host (Sec. IV-C), keeps them
 * resident, and runs every (threshold, scenario) pair as a job of batched
 * launches (thresholds in chunks, all reading the same parameter rows) with
 * model->trigger forced to AEB_TRIGGER_TTC.
 *   per_threshold  host, n_thr entries: pooled counts, p, Wilson 95 % interval
 *   per_job        host, n_thr * n_scen entries (threshold-major) or NULL
 * Synchronous; allocates and frees its device buffers (about
 * 80 B x n_scen x n_per_scenario for parameters plus up to 4.5 GB of outputs).
 */
aeb_status aeb_ttc_sweep(const aeb_model *model, const aeb_scenario *scenarios, uint32_t n_scen,
                         uint64_t n_per_scenario, const double *thresholds, uint32_t n_thr,
                         aeb_precision precision, aeb_sweep_result *per_threshold,
                         aeb_job_stats *per_job, void *stream);

/*
 * aeb_stats_merge / aeb_job_stats_merge -- add the statistics of another
 * disjoint set of samples into `acc` (host memory; the exchange step when the
 * samples of one workload are split across GPUs or calls).  Counts and
 * histograms add exactly; sums add in call order, so merging the parts in a
 * fixed order (e.g. rank order) gives the same bits every time.  aeb_stats
 * parts must share the histogram spec (AEB_EINVAL otherwise).
 */
aeb_status aeb_stats_merge(aeb_stats *acc, const aeb_stats *part);
aeb_status aeb_job_stats_merge(aeb_job_stats *acc, const aeb_job_stats *part);

/*
 * aeb_stats_summary / aeb_job_stats_summary -- the summary of a reduction
 * (host memory; see aeb_summary): counts, the mean, standard deviation and
 * range of the stopping distance over stopped samples and of the impact
 * speed over contact samples (Sec. VI-B, Table I), and the collision
 * probability n_contact / n_valid with its 95 % Wilson interval.
 * Host only, allocates nothing.  AEB_EINVAL: NULL argument, or counts that do
 * not add up to n.
 */
aeb_status aeb_stats_summary(const aeb_stats *stats, aeb_summary *out);
aeb_status aeb_job_stats_summary(const aeb_job_stats *stats, aeb_summary *out);

/*
 * aeb_hist_quantile -- the bin of a fixed histogram of `stats` (host memory)
 * that holds its q-quantile, i.e. the order statistic x_(k), k = ceil(q N)
 * clamped to [1, N], of the N samples the histogram counts (which =
 * AEB_HIST_D: x_ref of the stopped samples; AEB_HIST_V: v_imp of the contact
 * samples).  The safe headway at risk level p is the (1 - p) quantile of the
 * stopping distance (Sec. VI-C: 5, 1 and 0.1 % risk); *hi is then the
 * conservative value.  On return x_(k) lies in [*lo, *hi), a bin of width w;
 * the first bin starts at -inf and the last ends at +inf, because values
 * beyond the histogram's range are counted in its end bins.
 * Host only.  AEB_EINVAL: NULL argument, q outside [0, 1], unknown `which`,
 * an empty histogram, or a histogram whose bins do not add up to its count.
 */
aeb_status aeb_hist_quantile(const aeb_stats *stats, int32_t which, double q, double *lo,
                             double *hi);

/*
 * aeb_hist_exceedance -- P(X >= x) read off a fixed histogram of `stats` at
 * an inner bin edge x = lo + j w, 1 <= j <= AEB_NBINS - 1: the samples of the
 * histogram in bins j and above, over the valid samples (n - n_invalid), with
 * the 95 % Wilson interval.  With X = the stopping distance and x = H0 this is
 * Eq. 19's P(D_stop > H0) (Sec. VI-C; no sample lies exactly on an edge unless
 * the inputs put it there): exact, because every bin at or above j holds only
 * values >= x.  With a lead vehicle, contact and horizon samples count as
 * trials but not as events (their stopping distance is not observed); their
 * share is p_contact of aeb_stats_summary.
 * Host only.  AEB_EINVAL: NULL argument, unknown `which`, x not such an edge,
 * a histogram whose bins do not add up to its count.
 */
aeb_status aeb_hist_exceedance(const aeb_stats *stats, int32_t which, double x, aeb_prob *out);

/*
 * aeb_is_estimate -- the importance-sampling estimate of an event's
 * probability under the nominal scenario from the weighted sums of
 * aeb_reduce_weighted (host memory; rare-event estimation, Sec. VIII): p =
 * sum_we / n, its standard error sqrt(var / n) with the unbiased sample
 * variance var = (sumsq_we - (n p) p) / (n - 1), and the 95 % normal interval
 * p -+ 1.959963984540054 se.  Host only.  AEB_EINVAL: NULL argument, counts
 * that are inconsistent (n_event > n_valid > n).
 */
aeb_status aeb_is_estimate(const aeb_wstats *ws, aeb_is_result *out);

/* Wilson score interval of k successes in n trials at normal quantile z
 * (z = 1.959963984540054 for 95 %).  n == 0 gives [0, 1]. */
aeb_status aeb_wilson(uint64_t k, uint64_t n, double z, double *lo, double *hi);

/*
 * aeb_pipe_peaks -- measured throughput of the arithmetic pipes the rollout
 * kernels are bound by (no counterpart in the paper; the roofline denominators
 * of Sec. V-E's compute-bound kernels): binary32 FMA and binary64 FMA in
 * TFLOP/s (an FMA counts two), binary64 add in Tops/s, from many independent
 * dependency chains per thread.  Synchronous; ~10 ms of GPU time.
 */
aeb_status aeb_pipe_peaks(double *fp32_fma_tflops, double *fp64_fma_tflops, double *fp64_add_tops,
                          void *stream);

#ifdef __cplusplus
}
#endif

#endif /* AEB_H */
