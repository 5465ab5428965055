// Allocation-free entry point: the FP64 Gram G = B B^T with its per-CTA
// partial sums kept in a fixed, file-scope device array instead of memory
// the caller or the library allocates.
//
// Some callers cannot let a library allocate device memory: a host framework
// that owns every byte of device memory through its own pool and forbids
// plugins from calling cudaMalloc / cudaFree, or a latency-critical loop in
// which the implicit device synchronisation of cudaFree (and possibly
// cudaMalloc) is not acceptable.  dsanls_gram_noalloc serves them: the
// caller passes B and G, and the only scratch is kScratch below, which every
// GPU that loads this library holds until the process exits.
#include <mutex>

#include "../../include/dsanls.h"
#include "common.cuh"
#include "kernels.cuh"

namespace dsanls {

namespace {

// 2 MiB of FP64 partial Gram matrices: room for floor(262144 / k^2) CTAs
// (16 at k = 128, 26 at k = 100, 64 at k = 64, 256 at k = 32; the kernel
// never launches more than 304).  The cost of the fixed size: at k = 128 the
// partial Gram runs on 16 of the 152 SMs and at k = 100 on 26, against up to
// 304 CTAs with a handle's workspace, so for large d it is correspondingly
// slower; from k <= 29 on it gets the full grid.
constexpr int64_t kScratchDoubles = 262144;
static __device__ __align__(256) double kScratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of kScratch for the current device, resolved once per
// device with that device current.  In host code kScratch is only a host-side
// stand-in; the kernel must be given this address.  The set-up calls
// (cudaGetSymbolAddress, cudaFuncSetAttribute) must not run while `stream`
// is being captured into a graph: such a first call is refused with EINVAL
// before anything reaches the stream.
double *scratch_for_current_device(cudaStream_t stream) {
    int dev = 0;
    DSANLS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) throw ArgError{"device ordinal out of range"};
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        DSANLS_CUDA(cudaStreamIsCapturing(stream, &cs));
        if (cs != cudaStreamCaptureStatusNone)
            throw ArgError{"the first call on a device sets up the scratch address and must come before any "
                           "stream capture"};
        void *p = nullptr;
        DSANLS_CUDA(cudaGetSymbolAddress(&p, kScratch));
        prime_kernel_attributes();
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    return g_scratch_ptr[dev];
}

}  // namespace

}  // namespace dsanls

extern "C" int dsanls_gram_noalloc(const float *B, int32_t k, int64_t d, double *G, void *stream) {
    using namespace dsanls;
    if (!B || !G) {
        record_handleless_error("dsanls_gram_noalloc: B and G must be device pointers");
        return DSANLS_EINVAL;
    }
    if (k < 1 || k > 128) {
        record_handleless_error("dsanls_gram_noalloc: k must be in [1, 128] (the fixed scratch and the kernel "
                                "hold at most 128 x 128 pairs)");
        return DSANLS_EINVAL;
    }
    if (d < 1 || d > (1ll << 31) - 1) {
        record_handleless_error("dsanls_gram_noalloc: d must be in [1, 2^31 - 1]");
        return DSANLS_EINVAL;
    }
    try {
        double *scratch = scratch_for_current_device((cudaStream_t)stream);
        // every partial the reduction reads is written by this call, so
        // nothing in the scratch needs clearing first
        launch_gram(B, k, d, G, scratch, kScratchDoubles, (cudaStream_t)stream);
    } catch (const CudaError &e) {
        record_handleless_error(std::string("dsanls_gram_noalloc: CUDA error: ") + cudaGetErrorString(e.err));
        cudaGetLastError();
        return DSANLS_ECUDA;
    } catch (const ArgError &e) {
        record_handleless_error("dsanls_gram_noalloc: " + e.what);
        return DSANLS_EINVAL;
    }
    return DSANLS_OK;
}
