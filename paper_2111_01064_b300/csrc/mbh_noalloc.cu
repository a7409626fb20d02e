// direct_loglike_stored_noalloc: the stored-template direct likelihood for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point where they
// evaluate a likelihood: code that runs under another framework's memory manager with a fixed
// device budget, host callbacks that must not block on the driver's allocator, or services that
// pre-reserve all device memory at start-up.  This variant of direct_loglike_stored takes its
// per-(template, chunk) partial sums from a fixed file-scope device buffer instead of
// cudaMallocAsync.  The buffer (kNoAllocScratchBytes) exists on every device that loads the
// library, for the lifetime of the process.
#include <cuda_runtime.h>

#include <mutex>

#include "mbh_internal.cuh"

using namespace mbh;

namespace {
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;   // 8 MiB: W x chunks x 16 B partial sums
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device
}  // namespace

extern "C" mbh_status direct_loglike_stored_noalloc(const mbh_data* data, const void* h_dev, int64_t W,
                                                    mbh_precision precision, double* out_dev,
                                                    void* stream)
{
    if (!data) return fail(MBH_EINVAL, "data is NULL");
    if (W < 0) return fail(MBH_EINVAL, "W < 0");
    if (W == 0) return MBH_OK;
    if (precision != MBH_FP64 && precision != MBH_MIXED)
        return fail(MBH_EINVAL, "unknown precision %d", (int)precision);
    int64_t chunk;
    int nchunks;
    if (mbh_status s = stored_plan(data, W, chunk, nchunks)) return s;
    const size_t need = sizeof(double2) * (size_t)W * (size_t)nchunks;
    if (need > kNoAllocScratchBytes)
        return fail(MBH_EINVAL,
                    "direct_loglike_stored_noalloc: W=%lld needs %zu bytes of scratch "
                    "(%d chunks x 16 B per template) but its static buffer holds %zu bytes; "
                    "use direct_loglike_stored or split the batch",
                    (long long)W, need, nchunks, kNoAllocScratchBytes);
    if (!h_dev || !out_dev) return fail(MBH_EINVAL, "NULL buffer");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "direct_loglike_stored_noalloc");
    if (dev != data->device) return fail(MBH_EINVAL, "data lives on device %d, current device is %d", data->device, dev);
    if (dev < 0 || dev >= kMaxDevices) return fail(MBH_EINVAL, "device index %d beyond %d", dev, kMaxDevices);
    void* scratch = nullptr;
    {
        // first call on this device: look up the device address of the static buffer with
        // this device current (the host-side name is not a device address)
        std::lock_guard<std::mutex> lk(g_noalloc_mutex);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
            g_noalloc_addr[dev] = p;
        }
        scratch = g_noalloc_addr[dev];
    }
    // every partial-sum slot the finalize pass reads is written by the reduction first, so
    // nothing in the buffer has to start at zero
    cudaStream_t st = (cudaStream_t)stream;
    if (mbh_status s = launch_stored(data, h_dev, W, precision, (double2*)scratch, chunk, nchunks, st))
        return s;
    return launch_direct_finalize((const double2*)scratch, nchunks, W, data->dd, out_dev, st);
}
