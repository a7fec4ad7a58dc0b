// peaks.cu -- throughput of the plain arithmetic pipes the rollout kernels are
// bound by (binary32 FMA, binary64 FMA, binary64 add), measured with many
// independent dependency chains per thread so that latency is hidden and only
// issue/pipe throughput limits.  Used as the roofline denominators of the
// rollout kernels.
#include "aeb_internal.h"
#include "host_util.h"

namespace aeb {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chain(T a, T b, T *sink)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)12345.678) sink[0] = s;  // keeps the chains live; never true in practice
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_add_chain(T b, T *sink)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = x[c] + b;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)12345.678) sink[0] = s;
}

template <class K>
cudaError_t time_kernel(K launch, cudaStream_t s, float *ms)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return e;
    launch();  // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3; ++r) launch();
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    *ms /= 3.0f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

}  // namespace
}  // namespace aeb

extern "C" aeb_status aeb_pipe_peaks(double *fp32_fma_tflops, double *fp64_fma_tflops,
                                     double *fp64_add_tops, void *stream)
{
    using namespace aeb;
    clear_error();
    if (!fp32_fma_tflops || !fp64_fma_tflops || !fp64_add_tops)
        return fail(AEB_EINVAL, "aeb_pipe_peaks: NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "aeb_pipe_peaks: device query");
    void *sink = nullptr;
    e = cudaMalloc(&sink, 64);
    if (e != cudaSuccess) return cuda_fail(e, "aeb_pipe_peaks: cudaMalloc");
    const unsigned blocks32 = (unsigned)sms * 8, blocks64 = (unsigned)sms * 4;
    const double ops32 = (double)blocks32 * kThreads * kChains * kIters;
    const double ops64 = (double)blocks64 * kThreads * kChains * kIters;
    float ms = 0.0f;
    e = time_kernel([&] { k_fma_chain<float><<<blocks32, kThreads, 0, s>>>(1.0000001f, 1e-7f, (float *)sink); },
                    s, &ms);
    if (e == cudaSuccess) *fp32_fma_tflops = 2.0 * ops32 / (ms * 1e-3) / 1e12;
    if (e == cudaSuccess)
        e = time_kernel([&] { k_fma_chain<double><<<blocks64, kThreads, 0, s>>>(1.0000000001, 1e-12, (double *)sink); },
                        s, &ms);
    if (e == cudaSuccess) *fp64_fma_tflops = 2.0 * ops64 / (ms * 1e-3) / 1e12;
    if (e == cudaSuccess)
        e = time_kernel([&] { k_add_chain<double><<<blocks64, kThreads, 0, s>>>(1e-12, (double *)sink); },
                        s, &ms);
    if (e == cudaSuccess) *fp64_add_tops = ops64 / (ms * 1e-3) / 1e12;
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e, "aeb_pipe_peaks: kernels");
    return AEB_OK;
}
