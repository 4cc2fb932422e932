// smerf_noalloc.cu -- sampling for callers that cannot allocate device memory.
//
// smerf_sample needs scratch space for the anchor states and takes it from the
// stream-ordered allocator on every call.  Some callers cannot let a library allocate:
// real-time or embedded hosts whose device memory is carved out once at start-up, or
// frameworks that own every byte of device memory through their own pool and forbid
// third-party cudaMalloc calls.  For them,
// smerf_sample_noalloc runs the same anchor and segment kernels with the scratch placed
// in the fixed array below, which lives in this library's device image: every GPU that
// loads the library holds these bytes until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "smerf_internal.cuh"

namespace {

// The fixed scratch.  Host code must not use this name as a pointer: on the host it
// denotes a stand-in object, not the device address.  The device address comes from
// cudaGetSymbolAddress (scratch_address below).
constexpr size_t kNoAllocBytes = (size_t)16 << 20;  // 16 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_address[kMaxDevices] = {};

// Device address of g_noalloc_scratch on device `dev`, which must be current.  Outside stream
// capture it is looked up on every call (cheap, and it follows a context that was reset and
// reloaded the device image); while `st` is capturing, the address found by the last lookup on
// this device is reused, since a capture should make no such runtime queries.
int scratch_address(int dev, cudaStream_t st, void** out)
{
    if (dev < 0 || dev >= kMaxDevices) return SMERF_EINVAL;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return SMERF_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return SMERF_ECUDA;
        g_address[dev] = p;
    } else if (!g_address[dev]) {
        return SMERF_EUNSUPPORTED;  // no lookup outside capture yet on this device
    }
    *out = g_address[dev];
    return SMERF_OK;
}

}  // namespace

extern "C" int smerf_sample_noalloc(const smerf_plan* plan, uint64_t seed, int n_samples, void* out,
                                    void* stream)
{
    if (!plan || n_samples < 0 || n_samples > 65535) return SMERF_EINVAL;
    if (n_samples == 0) return SMERF_OK;
    if (!out || ((uintptr_t)out & 15u)) return SMERF_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SMERF_ECUDA;
    if (dev != plan->dev) return SMERF_EINVAL;
    if (smerf_scratch_bytes(plan, n_samples) > kNoAllocBytes) return SMERF_ESCRATCH;
    void* scratch = nullptr;
    const int rc = scratch_address(dev, (cudaStream_t)stream, &scratch);
    if (rc != SMERF_OK) return rc;
    // Every anchor state the segment kernel reads is first written by the anchor kernel of
    // the same call, so the array needs no clearing between calls.
    return smerf_launch_sample(plan, seed, n_samples, out, scratch, (cudaStream_t)stream);
}
