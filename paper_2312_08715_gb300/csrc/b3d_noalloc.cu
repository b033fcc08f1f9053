// b3d_noalloc.cu - log-sum-exp + categorical resampling without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need to resample: a host
// thread holding a custom allocator's lock or working under a hard memory cap owned by
// another framework, a loop that cannot afford the implicit synchronisation an allocation
// may bring, or an embedding that forbids the library from touching the allocator at all.
// For them, b3d_lse_resample_noalloc runs the same kernel as b3d_lse_resample, but its
// scratch (the per-block partial sums and the completion counter) lives in the fixed-size
// array below, part of the library's module image: every GPU that loads the library holds
// it until the process exits, and nothing is allocated or freed per call.
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
struct Cached {
    unsigned long long ctx_id = 0;  // the context the address belongs to (0: none yet)
    float2 *addr = nullptr;
};
Cached g_scratch_addr[kMaxDevices];

// The CUDA driver's identifier of the calling thread's current context: unique for the life of
// the process, so a context created after a device reset never matches an old one. 0 when
// there is no current context or the CUDA driver cannot say. Called with g_mu held.
unsigned long long current_context_id() {
    using GetCurrent = int (*)(void **);                       // cuCtxGetCurrent(CUcontext *)
    using GetId = int (*)(void *, unsigned long long *);       // cuCtxGetId(CUcontext, unsigned long long *)
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    }
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
    return 0;
}

// Device address of g_lse_scratch in the current device's context. In host code the name
// g_lse_scratch is only a host-side stand-in, never a device address. The address is looked
// up once per device and context: a context created after a device reset (where the module,
// and with it the array, may load elsewhere) gets a fresh lookup.
b3d_status scratch_for_current_device(float2 **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return B3D_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    Cached &c = g_scratch_addr[dev];
    const unsigned long long id = current_context_id();
    if (!c.addr || id == 0 || id != c.ctx_id) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_lse_scratch);  // creates the context if needed
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return B3D_ECUDA;
        }
        c.addr = static_cast<float2 *>(p);
        c.ctx_id = current_context_id();
    }
    *out = c.addr;
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
    // The kernel raises this word when every score is -inf; that case also shows in the
    // outputs (idx -1, logq -inf, logz -inf), which is how this entry point reports it. The
    // word stays in the shared scratch and the next call clears it.
    int *err = reinterpret_cast<int *>(tail) + 1;
    b3d::launch_lse_resample(loglik_dev, n, m, seed, stage, scratch, counter, logz_dev, idx_dev, logq_dev, err, s);
    e = cudaGetLastError();
    return e == cudaSuccess ? B3D_OK : B3D_ECUDA;
}
