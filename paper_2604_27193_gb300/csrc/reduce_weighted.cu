// reduce_weighted.cu -- weighted event sums of a set of rollout outputs for
// importance sampling (extension: rare-event estimation of low collision
// probabilities).  Each sample carries the likelihood ratio w of its parameter
// set (nominal over proposal density); the event E of a valid sample is a
// contact, or a final position x_ref beyond x_thr (Sec. VI-C: D_stop > H0).
// The sums Σ w, Σ w², Σ w 1[E], Σ w² 1[E] give the unbiased estimate
// Σ w 1[E] / n of the nominal probability of E and its standard error.
//
// Two launches on the caller's stream, in a fixed order so that the sums are
// the same bits for the same inputs:
//   1. G blocks; block b owns samples [b*chunk, (b+1)*chunk); each thread
//      walks its strided share in index order, the block adds the threads with
//      a fixed shared-memory tree and writes one partial;
//   2. one block adds the G partials with the same tree.
// One pass over 17 bytes per sample (status, x_ref, weight): bound by HBM
// bandwidth.
#include "aeb_internal.h"

namespace aeb {
namespace {

constexpr int kWThreads = 256;

struct WPart {
    unsigned long long n_valid, n_event;
    double sum_w, sumsq_w, sum_we, sumsq_we;
};

__device__ __forceinline__ void wadd(WPart &a, const WPart &b)
{
    a.n_valid += b.n_valid;
    a.n_event += b.n_event;
    a.sum_w += b.sum_w;
    a.sumsq_w += b.sumsq_w;
    a.sum_we += b.sum_we;
    a.sumsq_we += b.sumsq_we;
}

// Fixed-order tree over the block's threads (kWThreads a power of two).
__device__ __forceinline__ void block_tree(WPart &mine, WPart *sh)
{
    const int t = threadIdx.x;
    sh[t] = mine;
    __syncthreads();
    for (int stride = kWThreads / 2; stride > 0; stride >>= 1) {
        if (t < stride) wadd(sh[t], sh[t + stride]);
        __syncthreads();
    }
    mine = sh[0];
}

__global__ void __launch_bounds__(kWThreads)
k_reduce_weighted_partial(const uint8_t *status, const double *x_ref, const double *w,
                          uint64_t n, uint64_t chunk, double x_thr, WPart *parts)
{
    __shared__ WPart sh[kWThreads];
    WPart a{0ull, 0ull, 0.0, 0.0, 0.0, 0.0};
    const uint64_t lo = (uint64_t)blockIdx.x * chunk;
    const uint64_t hi = (lo + chunk < n) ? lo + chunk : n;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += kWThreads) {
        const uint8_t s = status[i];
        if (s == AEB_INVALID) continue;
        const double wi = w[i];
        a.n_valid += 1;
        a.sum_w += wi;
        a.sumsq_w += wi * wi;
        if (s == AEB_CONTACT || x_ref[i] > x_thr) {
            a.n_event += 1;
            a.sum_we += wi;
            a.sumsq_we += wi * wi;
        }
    }
    block_tree(a, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = a;
}

__global__ void __launch_bounds__(kWThreads)
k_reduce_weighted_final(const WPart *parts, int g, uint64_t n, aeb_wstats *out)
{
    __shared__ WPart sh[kWThreads];
    WPart a{0ull, 0ull, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < g; b += kWThreads) wadd(a, parts[b]);
    block_tree(a, sh);
    if (threadIdx.x == 0) {
        out->n = n;
        out->n_valid = a.n_valid;
        out->n_event = a.n_event;
        out->sum_w = a.sum_w;
        out->sumsq_w = a.sumsq_w;
        out->sum_we = a.sum_we;
        out->sumsq_we = a.sumsq_we;
    }
}

}  // namespace

size_t weighted_partial_bytes() { return sizeof(WPart) * kWMaxBlocks; }

cudaError_t launch_reduce_weighted(const uint8_t *status, const double *x_ref, const double *w,
                                   uint64_t n, double x_thr, void *partials, aeb_wstats *stats,
                                   cudaStream_t s)
{
    // G and chunk depend only on n: at most kWMaxBlocks blocks of >= 8192 samples
    uint64_t g = (n + 8191) / 8192;
    if (g > (uint64_t)kWMaxBlocks) g = kWMaxBlocks;
    if (g < 1) g = 1;
    const uint64_t chunk = (n + g - 1) / g;
    auto *parts = static_cast<WPart *>(partials);
    k_reduce_weighted_partial<<<(unsigned)g, kWThreads, 0, s>>>(status, x_ref, w, n,
                                                                chunk > 0 ? chunk : 1, x_thr, parts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_weighted_final<<<1, kWThreads, 0, s>>>(parts, (int)g, n, stats);
    return cudaGetLastError();
}

}  // namespace aeb
