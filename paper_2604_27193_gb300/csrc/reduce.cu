// reduce.cu -- counts, moments, extremes and fixed-bin histograms of a set of
// rollout outputs (Sec. VI-B statistics; Sec. VI-C reads P(D_stop > H0) and the
// safe headways off the stopping-distance histogram).
//
// Two launches on the caller's stream:
//   1. G blocks; block b owns samples [b*chunk, (b+1)*chunk).  Each thread
//      walks its strided share in index order, the warp combines lanes with a
//      fixed xor butterfly, warp 0 adds the warps in warp order, and the block
//      writes one partial.  Histogram bins are counted with shared-memory
//      atomics and flushed with 64-bit global atomics (integer adds commute,
//      so they are exact and order-free).
//   2. one block adds the G partials in the same fixed pattern.
// G and chunk depend only on n, so the floating-point sums are the same bits
// on every call.  The work is a single pass over 21 bytes per sample
// (status, x_ref, v_imp, n_steps); its time is set by the binary64 sums and
// squares (1/64 rate on GB300), so the bin index and the extremes are taken
// from the bits with integer instructions.
#include <cfloat>
#include <cmath>

#include "aeb_internal.h"

namespace aeb {
namespace {

constexpr int kRedThreads = 256;
constexpr int kRedWarps = kRedThreads / 32;

// floor((x - lo) / w) clamped to [0, NBINS - 1] for the power-of-two width
// w = 2^-k.  (x - lo) is one binary64 subtraction, as in the definition; the
// exact scaling by 2^k and the floor are done on its bits with integer
// instructions, which keeps the binary64 pipe (1/64 rate on GB300) for the
// sums.  y = m 2^ex with the 53-bit significand m, so floor(y 2^k) is m shifted
// right by -(ex + k); a normal y with ex + k >= -40 is already >= 2^12.
__device__ __forceinline__ int bin_index(double x, double lo, int k)
{
    const long long b = __double_as_longlong(x - lo);
    if (b <= 0) return 0;  // +0, or negative (sign bit set)
    const int e = (int)((b >> 52) & 0x7ff);
    unsigned long long m = (unsigned long long)b & 0xfffffffffffffull;
    int ex = -1074;        // subnormal: y = m 2^-1074
    if (e != 0) {
        m |= 1ull << 52;
        ex = e - 1075;
    }
    const int sh = ex + k;
    if (sh >= -40) return AEB_NBINS - 1;
    const int r = -sh;
    const unsigned long long q = (r >= 64) ? 0ull : (m >> r);
    return q > (unsigned long long)(AEB_NBINS - 1) ? AEB_NBINS - 1 : (int)q;
}

// Total-order key of a double (an involution): the bits for a non-negative
// value, the magnitude bits flipped for a negative one, so that keys compare as
// signed integers in the order of the values (-0 just below +0).  The thread
// loop keeps its extremes as keys, on the integer pipe.
__device__ __forceinline__ long long order_key(long long b)
{
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}

__device__ __forceinline__ void init_partial(RedPartial &a)
{
    a.n_stop = a.n_contact = a.n_horizon = a.n_invalid = a.steps = 0;
    a.sum_d = a.sumsq_d = a.sum_v = a.sumsq_v = 0.0;
    a.min_d = a.min_v = __longlong_as_double(0x7ff0000000000000ll);   // +inf
    a.max_d = a.max_v = __longlong_as_double(0xfff0000000000000ll);   // -inf
}

__device__ __forceinline__ void add_partial(RedPartial &a, const RedPartial &b)
{
    a.n_stop += b.n_stop;
    a.n_contact += b.n_contact;
    a.n_horizon += b.n_horizon;
    a.n_invalid += b.n_invalid;
    a.steps += b.steps;
    a.sum_d += b.sum_d;
    a.sumsq_d += b.sumsq_d;
    a.sum_v += b.sum_v;
    a.sumsq_v += b.sumsq_v;
    a.min_d = fmin(a.min_d, b.min_d);
    a.max_d = fmax(a.max_d, b.max_d);
    a.min_v = fmin(a.min_v, b.min_v);
    a.max_v = fmax(a.max_v, b.max_v);
}

__device__ __forceinline__ RedPartial shfl_xor_partial(const RedPartial &a, int m)
{
    RedPartial b;
    b.n_stop = __shfl_xor_sync(0xffffffffu, a.n_stop, m);
    b.n_contact = __shfl_xor_sync(0xffffffffu, a.n_contact, m);
    b.n_horizon = __shfl_xor_sync(0xffffffffu, a.n_horizon, m);
    b.n_invalid = __shfl_xor_sync(0xffffffffu, a.n_invalid, m);
    b.steps = __shfl_xor_sync(0xffffffffu, a.steps, m);
    b.sum_d = __shfl_xor_sync(0xffffffffu, a.sum_d, m);
    b.sumsq_d = __shfl_xor_sync(0xffffffffu, a.sumsq_d, m);
    b.sum_v = __shfl_xor_sync(0xffffffffu, a.sum_v, m);
    b.sumsq_v = __shfl_xor_sync(0xffffffffu, a.sumsq_v, m);
    b.min_d = __shfl_xor_sync(0xffffffffu, a.min_d, m);
    b.max_d = __shfl_xor_sync(0xffffffffu, a.max_d, m);
    b.min_v = __shfl_xor_sync(0xffffffffu, a.min_v, m);
    b.max_v = __shfl_xor_sync(0xffffffffu, a.max_v, m);
    return b;
}

// Combine a block's per-thread partials in a fixed pattern; result in thread 0.
__device__ __forceinline__ RedPartial block_combine(RedPartial acc, RedPartial *sh)
{
    // butterfly: every lane ends with the same value, combined in a fixed order
    for (int m = 16; m > 0; m >>= 1) {
        RedPartial o = shfl_xor_partial(acc, m);
        // order the two operands by lane so both lanes of a pair add a + b
        const bool low = ((threadIdx.x & 31) & m) == 0;
        RedPartial first = low ? acc : o, second = low ? o : acc;
        add_partial(first, second);
        acc = first;
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) sh[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        RedPartial t = sh[0];
        for (int j = 1; j < kRedWarps; ++j) add_partial(t, sh[j]);
        acc = t;
    }
    return acc;
}

// HIST: accumulate the two histograms.  With a block table, block b reduces
// rows [out_offset + first, + count) of job table[b].job (a segment of one
// job), otherwise rows [b chunk, (b+1) chunk) of [0, n).
template <bool HIST>
__global__ void __launch_bounds__(kRedThreads)
k_reduce_partial(const uint8_t *__restrict__ st, const double *__restrict__ xr,
                 const double *__restrict__ vi, const int32_t *__restrict__ ns, uint64_t n,
                 uint64_t chunk, const TileDesc *__restrict__ table, const JobDev *__restrict__ jobs,
                 double lo_d, int k_d, double lo_v, int k_v,
                 RedPartial *__restrict__ part, unsigned long long *__restrict__ hist_d,
                 unsigned long long *__restrict__ hist_v)
{
    __shared__ unsigned int sh_d[HIST ? AEB_NBINS : 1];
    __shared__ unsigned int sh_v[HIST ? AEB_NBINS : 1];
    __shared__ RedPartial sh_p[kRedWarps];
    if (HIST) {
        for (int j = threadIdx.x; j < AEB_NBINS; j += kRedThreads) {
            sh_d[j] = 0u;
            sh_v[j] = 0u;
        }
        __syncthreads();
    }

    uint64_t lo, hi;
    if (table) {
        const TileDesc d = table[blockIdx.x];
        lo = jobs[d.job].out_offset + d.first;
        hi = lo + d.count;
    } else {
        lo = (uint64_t)blockIdx.x * chunk;
        hi = (lo + chunk < n) ? lo + chunk : n;
    }
    RedPartial acc;
    init_partial(acc);
    long long kmin_d = order_key(0x7ff0000000000000ll), kmax_d = order_key(0xfff0000000000000ll);
    long long kmin_v = kmin_d, kmax_v = kmax_d;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += kRedThreads) {
        const uint8_t s = st[i];
        acc.steps += (unsigned long long)(long long)ns[i];
        if (s == AEB_STOP) {
            const double d = xr[i];
            const long long kd = order_key(__double_as_longlong(d));
            acc.n_stop++;
            acc.sum_d += d;
            acc.sumsq_d += d * d;
            kmin_d = kd < kmin_d ? kd : kmin_d;
            kmax_d = kd > kmax_d ? kd : kmax_d;
            if (HIST) atomicAdd(&sh_d[bin_index(d, lo_d, k_d)], 1u);
        } else if (s == AEB_CONTACT) {
            const double v = vi[i];
            const long long kv = order_key(__double_as_longlong(v));
            acc.n_contact++;
            acc.sum_v += v;
            acc.sumsq_v += v * v;
            kmin_v = kv < kmin_v ? kv : kmin_v;
            kmax_v = kv > kmax_v ? kv : kmax_v;
            if (HIST) atomicAdd(&sh_v[bin_index(v, lo_v, k_v)], 1u);
        } else if (s == AEB_HORIZON) {
            acc.n_horizon++;
        } else {
            acc.n_invalid++;
        }
    }
    acc.min_d = __longlong_as_double(order_key(kmin_d));
    acc.max_d = __longlong_as_double(order_key(kmax_d));
    acc.min_v = __longlong_as_double(order_key(kmin_v));
    acc.max_v = __longlong_as_double(order_key(kmax_v));
    acc = block_combine(acc, sh_p);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
    if (HIST) {
        __syncthreads();
        for (int j = threadIdx.x; j < AEB_NBINS; j += kRedThreads) {
            if (sh_d[j]) atomicAdd(&hist_d[j], (unsigned long long)sh_d[j]);
            if (sh_v[j]) atomicAdd(&hist_v[j], (unsigned long long)sh_v[j]);
        }
    }
}

// Block j adds the partials [first[j], first[j+1]) of job j in index order.
__global__ void __launch_bounds__(kRedThreads)
k_reduce_jobs_final(const RedPartial *__restrict__ part, const uint32_t *__restrict__ first,
                    const JobDev *__restrict__ jobs, aeb_job_stats *__restrict__ out)
{
    __shared__ RedPartial sh_p[kRedWarps];
    const uint32_t b0 = first[blockIdx.x], b1 = first[blockIdx.x + 1];
    RedPartial acc;
    init_partial(acc);
    for (uint32_t j = b0 + threadIdx.x; j < b1; j += kRedThreads) add_partial(acc, part[j]);
    acc = block_combine(acc, sh_p);
    if (threadIdx.x == 0) {
        aeb_job_stats &o = out[blockIdx.x];
        o.n = jobs[blockIdx.x].n;
        o.n_stop = acc.n_stop;
        o.n_contact = acc.n_contact;
        o.n_horizon = acc.n_horizon;
        o.n_invalid = acc.n_invalid;
        o.steps = acc.steps;
        o.sum_d = acc.sum_d;
        o.sumsq_d = acc.sumsq_d;
        o.min_d = acc.min_d;
        o.max_d = acc.max_d;
        o.sum_v = acc.sum_v;
        o.sumsq_v = acc.sumsq_v;
        o.min_v = acc.min_v;
        o.max_v = acc.max_v;
    }
}

__global__ void __launch_bounds__(kRedThreads)
k_reduce_final(const RedPartial *__restrict__ part, int g, uint64_t n, aeb_hist_spec h,
               aeb_stats *__restrict__ out)
{
    __shared__ RedPartial sh_p[kRedWarps];
    RedPartial acc;
    init_partial(acc);
    for (int j = threadIdx.x; j < g; j += kRedThreads) add_partial(acc, part[j]);
    acc = block_combine(acc, sh_p);
    if (threadIdx.x == 0) {
        out->n = n;
        out->n_stop = acc.n_stop;
        out->n_contact = acc.n_contact;
        out->n_horizon = acc.n_horizon;
        out->n_invalid = acc.n_invalid;
        out->steps = acc.steps;
        out->sum_d = acc.sum_d;
        out->sumsq_d = acc.sumsq_d;
        out->min_d = acc.min_d;
        out->max_d = acc.max_d;
        out->sum_v = acc.sum_v;
        out->sumsq_v = acc.sumsq_v;
        out->min_v = acc.min_v;
        out->max_v = acc.max_v;
        out->lo_d = h.lo_d;
        out->w_d = h.w_d;
        out->lo_v = h.lo_v;
        out->w_v = h.w_v;
    }
}

}  // namespace

int reduce_blocks_for(uint64_t n)
{
    uint64_t g = (n + 8191) / 8192;
    if (g < 1) g = 1;
    if (g > 1024) g = 1024;
    return (int)g;
}

cudaError_t launch_reduce(const uint8_t *status, const double *x_ref, const double *v_imp,
                          const int32_t *n_steps, uint64_t n, const aeb_hist_spec &h,
                          RedPartial *partials, aeb_stats *stats, cudaStream_t s)
{
    const int g = reduce_blocks_for(n);
    const uint64_t chunk = (n + (uint64_t)g - 1) / (uint64_t)g;
    cudaError_t e = cudaMemsetAsync(stats->hist_d, 0, 2 * sizeof(uint64_t) * AEB_NBINS, s);
    if (e != cudaSuccess) return e;
    k_reduce_partial<true><<<g, kRedThreads, 0, s>>>(
        status, x_ref, v_imp, n_steps, n, chunk, nullptr, nullptr, h.lo_d, -std::ilogb(h.w_d),
        h.lo_v, -std::ilogb(h.w_v), partials, reinterpret_cast<unsigned long long *>(stats->hist_d),
        reinterpret_cast<unsigned long long *>(stats->hist_v));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, kRedThreads, 0, s>>>(partials, g, n, h, stats);
    return cudaGetLastError();
}

cudaError_t launch_reduce_jobs(const uint8_t *status, const double *x_ref, const double *v_imp,
                               const int32_t *n_steps, const TileDesc *blocks, uint32_t n_blocks,
                               const uint32_t *first, const JobDev *jobs, uint32_t n_jobs,
                               RedPartial *partials, aeb_job_stats *stats, cudaStream_t s)
{
    if (n_blocks > 0) {
        k_reduce_partial<false><<<n_blocks, kRedThreads, 0, s>>>(
            status, x_ref, v_imp, n_steps, 0, 0, blocks, jobs, 0.0, 0, 0.0, 0, partials,
            nullptr, nullptr);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_reduce_jobs_final<<<n_jobs, kRedThreads, 0, s>>>(partials, first, jobs, stats);
    return cudaGetLastError();
}

}  // namespace aeb
