// mm_rbffd_weights_ir_noalloc: the FP32 + FP64-refinement weights call
// without any device allocation, for callers that cannot allocate device
// memory at call time.
//
// The mixed-precision solve hands the stencils it cannot finish in FP32 to
// the FP64 solve through a queue (a counter and a list of row indices).  The
// regular entry point takes that queue from the context workspace, which may
// call cudaMalloc/cudaFree.  Here the queue lives in a fixed array in device
// memory that is part of this library image: every GPU that loads the library
// holds it (4 MiB + 4 bytes) until the process exits.
#include <mutex>

#include "mm_internal.cuh"

namespace {

constexpr int64_t kNoAllocMaxRows = int64_t(1) << 20;   // rows per call

// [0] = queue length, [1 .. kNoAllocMaxRows] = queued row indices.  Every call
// shares it; it keeps the last call's contents.
static __device__ __align__(256) int g_fb_queue[1 + kNoAllocMaxRows];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
int *g_queue_addr[kMaxDevices];   // nullptr until a lookup on that device succeeded

// Device address of g_fb_queue on `device` (which must be current).  In host
// code the name g_fb_queue is only a host-side stand-in, so the address is
// looked up per device and cached.  Only a successful lookup is cached: a
// failed one (e.g. attempted inside a stream capture) is retried by the next
// call.  The cached address belongs to the device's primary context; after a
// cudaDeviceReset it is stale, so a process that resets a device must not
// call this entry point on it again.
int queue_address(int device, int **out) {
    if (device < 0 || device >= kMaxDevices) return MM_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_queue_addr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_fb_queue) != cudaSuccess || !p) {
            cudaGetLastError();
            return MM_ECUDA;
        }
        g_queue_addr[device] = (int *)p;
    }
    *out = g_queue_addr[device];
    return MM_OK;
}

}  // namespace

extern "C" int mm_rbffd_weights_ir_noalloc(mm_ctx *ctx, unsigned ops, int k, int m, int dim,
                                           int64_t N, const double *d_pts,
                                           const double *d_normals,
                                           const mm_csr_pattern *stencils, int64_t row_begin,
                                           int64_t row_end, int n_max, double *const *d_vals,
                                           int32_t *d_status) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    WeightsJob job{};
    int rc = weights_job_from_args(ctx, ops, k, m, dim, N, d_pts, d_normals, stencils, row_begin,
                                   row_end, n_max, d_vals, d_status, &job);
    if (rc != MM_OK) return rc;
    if (row_end - row_begin > kNoAllocMaxRows)
        return mm_fail(ctx, MM_EUNSUPPORTED,
                       "mm_rbffd_weights_ir_noalloc handles at most %lld rows per call (got %lld); "
                       "split the row range or use mm_rbffd_weights",
                       (long long)kNoAllocMaxRows, (long long)(row_end - row_begin));
    DeviceGuard g(ctx);
    int *queue = nullptr;
    if (queue_address(ctx->device, &queue) != MM_OK)
        return mm_fail(ctx, MM_ECUDA, "cudaGetSymbolAddress of the fallback queue failed on device %d",
                       ctx->device);
    // the launch clears queue[0] on the stream before the solve kernel runs
    return weights_launch_scratch(ctx, job, MM_FP32_IR, queue, queue + 1);
}
