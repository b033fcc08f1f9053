// b3d_noalloc.cu - log-sum-exp + categorical resampling without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need to resample: code
// running while a CUDA graph is being captured (cudaMalloc is not a capturable operation),
// a host thread holding a custom allocator's lock or working under a hard memory cap owned
// by another framework, or an embedding that forbids the library from touching the
// allocator at all. For them, b3d_lse_resample_noalloc runs the same kernel as
// b3d_lse_resample, but its scratch (the per-block partial sums and the completion
// counter) lives in the fixed-size array below, part of the library's module image:
// every GPU that loads the library holds it until the process exits, and nothing is
// allocated or freed per call.
//
// Because every call shares this one array, calls that overlap on the GPU (on different
// streams, or from different threads without ordering) race on it; serialise them.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "b3d.h"
#include "b3d_internal.h"

namespace {

constexpr int kNoallocBlocks = 1024;  // partial sums held: the resampling kernel's block limit

// scratch[0 .. kNoallocBlocks-1]: (block max, block sum of exp) pairs;
// scratch[kNoallocBlocks]: .x = completion counter bits, .y = device error flag bits.
static __device__ __align__(256) float2 g_lse_scratch[kNoallocBlocks + 1];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float2 *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_lse_scratch on the current device, looked up once per device. In host
// code the name g_lse_scratch is only a host-side stand-in, never a device address.
b3d_status scratch_for_current_device(float2 **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return B3D_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_lse_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return B3D_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<float2 *>(p);
    }
    *out = g_scratch_addr[dev];
    return B3D_OK;
}

}  // namespace

extern "C" b3d_status b3d_lse_resample_noalloc(int64_t n, const float *loglik_dev, int32_t m, uint64_t seed,
                                               int32_t stage, float *logz_dev, int32_t *idx_dev, float *logq_dev,
                                               b3d_stream stream) {
    if (n < 1 || n > B3D_NOALLOC_MAX_SCORES) return B3D_EINVAL;
    if (m < 0 || !loglik_dev || !logz_dev || (m > 0 && (!idx_dev || !logq_dev))) return B3D_EINVAL;
    if (b3d::lse_blocks(n) > kNoallocBlocks) return B3D_EINVAL;
    float2 *scratch = nullptr;
    b3d_status st = scratch_for_current_device(&scratch);
    if (st != B3D_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    float2 *tail = scratch + kNoallocBlocks;
    // the completion counter must start at zero; the error word is cleared with it
    cudaError_t e = cudaMemsetAsync(tail, 0, sizeof(float2), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return B3D_ECUDA;
    }
    unsigned *counter = reinterpret_cast<unsigned *>(tail);
    int *err = reinterpret_cast<int *>(tail) + 1;
    b3d::launch_lse_resample(loglik_dev, n, m, seed, stage, scratch, counter, logz_dev, idx_dev, logq_dev, err, s);
    e = cudaGetLastError();
    return e == cudaSuccess ? B3D_OK : B3D_ECUDA;
}
