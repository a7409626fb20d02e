// Device-side status word of libmbhlike and its host side: mbh_sync_status, and the debug
// build's test hook mbh_debug_ref_limit (declarations: include/mbhlike.h).
//
// Every launch of the heterodyne kernels carries the address of the current device's status
// word.  In builds with MBH_DEBUG_CHECKS the kernels check the index of every edge record they
// read against the source's logical edge range; a failed check records (kernel, source, index,
// range) with an atomic compare-and-swap on the code (the first failure wins) and skips the
// access.  Nothing traps, and a check never changes which memory is read.
#include <cuda_runtime.h>

#include <mutex>

#include "mbh_internal.cuh"

using namespace mbh;

namespace {
__device__ DevStatus g_dev_status;   // zero-initialised when the module loads on a device

constexpr int kMaxDevices = 64;
std::mutex g_status_mutex;
DevStatus* g_status_addr[kMaxDevices] = {};

const char* kernel_name(unsigned k)
{
    switch (k) {
    case kKernHetX: return "het_x_kernel (MBH_MIXED heterodyne)";
    case kKernHetF32: return "het_mixed_kernel (MBH_MIXED_F32 heterodyne)";
    case kKernHetF64: return "het_f64_kernel (MBH_FP64 heterodyne)";
    default: return "unknown kernel";
    }
}
}  // namespace

namespace mbh {
int sm_count()
{
    static int cache[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 148;
    if (cache[dev] <= 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 148;
        cache[dev] = n;
    }
    return cache[dev];
}

// The symbol's host-side name is not a device address: the address is looked up once per
// device, with that device current (mbh_data_create and het_prepare_reference call this
// first, outside any stream capture).
DevStatus* dev_status()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_status_mutex);
    if (!g_status_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dev_status) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_status_addr[dev] = static_cast<DevStatus*>(p);
    }
    return g_status_addr[dev];
}
}  // namespace mbh

extern "C" int32_t mbh_debug_checks(void)
{
#ifdef MBH_DEBUG_CHECKS
    return 1;
#else
    return 0;
#endif
}

extern "C" mbh_status mbh_sync_status(void* stream, mbh_device_status* info)
{
    if (info) *info = mbh_device_status{0, 0, 0, 0, 0, 0};
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mbh_sync_status");
    DevStatus* d = dev_status();
    if (!d) return fail(MBH_ECUDA, "mbh_sync_status: no device status word on this device");
    DevStatus h{};
    e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "mbh_sync_status read");
    if (h.code == 0u) return MBH_OK;
    e = cudaMemset(d, 0, sizeof(DevStatus));
    if (e != cudaSuccess) return cuda_fail(e, "mbh_sync_status clear");
    if (info) *info = mbh_device_status{(int32_t)h.code, (int32_t)h.kernel, h.source, 0, h.index, h.limit};
    return fail(MBH_EDEVICE, "%s: index %lld outside its range [0, %lld) (source %d); the access was skipped",
                kernel_name(h.kernel), h.index, h.limit, h.source);
}

extern "C" mbh_status mbh_debug_ref_limit(mbh_ref* ref, int32_t e_check)
{
#ifdef MBH_DEBUG_CHECKS
    if (!ref) return fail(MBH_EINVAL, "ref is NULL");
    if (e_check < -1 || e_check > ref->E) return fail(MBH_EINVAL, "e_check %d outside [-1, E = %d]", e_check, ref->E);
    ref->E_check = e_check;
    return MBH_OK;
#else
    (void)ref;
    (void)e_check;
    return fail(MBH_EINVAL, "mbh_debug_ref_limit: this library was built without MBH_DEBUG_CHECKS");
#endif
}
