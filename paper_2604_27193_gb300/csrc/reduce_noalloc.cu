// reduce_noalloc.cu -- aeb_reduce for callers that must not allocate device
// memory while they run.
//
// aeb_reduce keeps its per-block partial sums in library scratch that it
// allocates with cudaMalloc on the first call per (device, stream).  Some
// callers cannot allow that: a real-time control loop whose rules forbid any
// allocation after start-up, or a process whose device memory is already
// handed out in full to another allocator, so that a late cudaMalloc may fail.
// aeb_reduce_noalloc runs the same two kernels with the partials placed in a
// fixed array compiled into this library instead; it allocates nothing.
//
// The array lives in every GPU that loads the library, for the life of the
// process, and all calls share it: calls whose work overlaps on the GPU (for
// example on two streams at once) race on it and must be serialised by the
// caller.  Every call overwrites the partials it uses before reading them, and
// the histogram bins it accumulates into are in the caller's aeb_stats, which
// the call clears first, so nothing from an earlier call leaks into a result.
#include <mutex>
#include <string>

#include "aeb_internal.h"
#include "host_util.h"

namespace aeb {
namespace {

// aeb_reduce splits n samples over ceil(n / 8192) blocks (at most 1024); the
// static array holds 256 partials (26.6 KB), so n is limited to 256 * 8192.
constexpr int kNoAllocPartials = 256;
static_assert((uint64_t)kNoAllocPartials * 8192 == AEB_REDUCE_NOALLOC_MAX_N,
              "limit in aeb.h must match the static scratch");

static __device__ __align__(256) RedPartial g_noalloc_partials[kNoAllocPartials];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
RedPartial *g_partials_addr[kMaxDevices];  // device address per device ordinal

}  // namespace
}  // namespace aeb

extern "C" aeb_status aeb_reduce_noalloc(const aeb_outputs *out, uint64_t n,
                                         const aeb_hist_spec *hist, aeb_stats *stats,
                                         void *stream)
{
    using namespace aeb;
    clear_error();
    if (!out || !stats) return fail(AEB_EINVAL, "aeb_reduce_noalloc: NULL argument");
    if (n > AEB_REDUCE_NOALLOC_MAX_N)
        return fail(AEB_EINVAL, "aeb_reduce_noalloc: n = " + std::to_string(n) +
                                    " exceeds the limit of its fixed scratch (" +
                                    std::to_string(AEB_REDUCE_NOALLOC_MAX_N) +
                                    " samples); use aeb_reduce for larger sets");
    if (n > 0 && (!out->status || !out->x_ref || !out->v_imp || !out->n_steps))
        return fail(AEB_EINVAL, "aeb_reduce_noalloc: status, x_ref, v_imp and n_steps are required");
    if (reinterpret_cast<uintptr_t>(stats) % 8 != 0)
        return fail(AEB_EINVAL, "aeb_reduce_noalloc: stats is not 8-byte aligned");
    aeb_status st = check_hist(hist);  // the same rule as aeb_reduce
    if (st != AEB_OK) return st;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return fail(AEB_EDEVICE, std::string("aeb_reduce_noalloc: cudaGetDevice: ") +
                                     cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(AEB_EDEVICE, "aeb_reduce_noalloc: device ordinal beyond 63");
    RedPartial *partials = nullptr;
    {
        // Host code cannot use the array's name as a device address: look the
        // address up once per device, with that device current.
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_partials_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess)
                return fail(AEB_ECUDA, std::string("aeb_reduce_noalloc: cudaGetSymbolAddress: ") +
                                           cudaGetErrorString(e));
            g_partials_addr[dev] = static_cast<RedPartial *>(p);
        }
        partials = g_partials_addr[dev];
    }
    e = launch_reduce(out->status, out->x_ref, out->v_imp, out->n_steps, n, *hist, partials,
                      stats, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return fail(AEB_ECUDA, std::string("aeb_reduce_noalloc: launch: ") + cudaGetErrorString(e));
    return AEB_OK;
}
