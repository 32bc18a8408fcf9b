// Internal declarations shared by the libmm translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <map>
#include <string>

#include "mm.h"

struct mm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int num_sms = 0;
    size_t smem_optin = 0;          // largest dynamic shared memory per block
    size_t smem_per_sm = 0;         // shared memory per SM
    size_t smem_reserved = 0;       // shared memory the system reserves per block
    // growable device workspace (bump-allocated per call)
    char *ws = nullptr;
    size_t ws_bytes = 0;
    // a second growable buffer for calls that hold data across another
    // call's use of the workspace (the candidates of the balanced stencils)
    char *ws2 = nullptr;
    size_t ws2_bytes = 0;
    // options
    double ir_tol = 1e-9;
    int ir_max_steps = 4;
    double kappa_max = 0.1;
    int wide64 = 0;     // refinement residuals and projection in native FP64
    int mlp_layered = 0;   // MLP inference layer by layer (mma.sync) instead of fused (tcgen05)
    int gj_shared = 0;     // FP32 inverse in shared memory for every system size
    // tuned launch shapes of the batched weights kernel, by batch signature
    std::map<std::string, mm_launch_config> tiles;
};

// Records a message and returns `code`.
int mm_fail(mm_ctx *ctx, int code, const char *fmt, ...);

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) only when `bytes` exceeds
// what was set before for this kernel on this device (so launches inside a
// stream capture make no attribute call once warmed up).
cudaError_t mm_set_smem(const mm_ctx *ctx, const void *kernel, size_t bytes);

// Warps per block (1 .. max_wpb) that keep the most warps of `kernel`
// resident on an SM when each warp needs `bytes_per_warp` of dynamic shared
// memory (the kernel's shared-memory attribute is raised as needed).
int mm_warps_per_block(const mm_ctx *ctx, const void *kernel, size_t bytes_per_warp, int max_wpb);

// Ensures the workspace holds at least `bytes`; returns its base or nullptr.
char *mm_workspace(mm_ctx *ctx, size_t bytes);
// The same for the second buffer.
char *mm_workspace2(mm_ctx *ctx, size_t bytes);

// Bump allocator over the workspace, 256-byte aligned slices.
struct WsCarve {
    size_t off = 0;
    template <class T>
    size_t take(size_t count) {
        size_t o = off;
        off += (count * sizeof(T) + 255) & ~size_t(255);
        return o;
    }
};

#define MM_CUDA_CHECK(ctx, expr)                                                        \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return mm_fail((ctx), MM_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));   \
    } while (0)

#define MM_LAUNCH_CHECK(ctx)                                                            \
    do {                                                                                \
        cudaError_t e_ = cudaGetLastError();                                            \
        if (e_ != cudaSuccess)                                                          \
            return mm_fail((ctx), MM_ECUDA, "kernel launch: %s", cudaGetErrorString(e_)); \
    } while (0)

// ---------------------------------------------------------------- launchers
int knn_launch(mm_ctx *ctx, int dim, int64_t N, const double *d_pts, int nranges,
               const mm_knn_range *ranges, int method, int32_t *d_status);

struct WeightsJob {
    unsigned ops;
    int k, m, dim;
    int64_t N;
    const double *pts, *normals;
    const int64_t *row_ptr;
    const int32_t *col;
    int64_t row_begin, row_end;
    int n_max;
    double *vals[11];  // per operator bit (nullptr if not requested)
    int32_t *status;
};

// Fused MLP inference on the tensor cores (mlp_tc.cu): x [B x n_in] FP32 ->
// y [B x n_out] FP32 (denormalised); img is the weight image built by
// mlp_tc_image from the padded FP32 parameters (oW: offsets of W1..W4).
struct MlpTcArgs {
    const float *x;
    int n_in;
    int64_t B;
    const __nv_bfloat16 *img;
    const float *b1, *b2, *b3, *b4, *ymean, *ystd;
    int n_out;
    float *y;
    int *err;   // set to 1 if a wait timed out (those rows' outputs are NaN)
};
constexpr int64_t kMlpTcImageElems = 16384 * 9 + 8192;   // W1 + W2 + W3 + W4 as BF16
int mlp_tc_image(mm_ctx *ctx, const float *p, const int64_t oW[4], __nv_bfloat16 *img);
int mlp_tc_forward(mm_ctx *ctx, const MlpTcArgs &args);

// Tensor-core GEMM of the MLP training (gemm_tc.cu): C[M x N] = A[M x K] *
// B[N x K]^T, BF16 K-major operands (rows 16-byte aligned: leading dimensions
// multiples of 8), FP32 accumulation, N <= 256, kslice (K per blockIdx.z) a
// multiple of 64.
enum { kTcPartial = 0, kTcBias = 1, kTcBiasGelu = 2, kTcDGelu = 3 };
struct TcGemmArgs {
    int M, N, K, kslice;
    const __nv_bfloat16 *A;
    int64_t lda;
    const __nv_bfloat16 *B;
    int64_t ldb;
    int epi;
    float *c;              // kTcPartial: slice z at c + z*M*ldc; kTcBias: output
    int64_t ldc;
    const float *bias;     // [N]
    float *z;              // pre-activation: written by kTcBiasGelu, read by kTcDGelu
    int64_t ldz;
    __nv_bfloat16 *h;      // BF16 row-major output (activation or dZ)
    int64_t ldh;
    __nv_bfloat16 *ht;     // optional BF16 transposed output [N x ldht]
    int64_t ldht;
    int *err;              // set to 1 if a wait timed out
};
int tc_gemm(mm_ctx *ctx, const TcGemmArgs &a);

int weights_launch(mm_ctx *ctx, const WeightsJob &job, int precision);
// FP32 + refinement kernel of one class (2D / 3D); handed-over rows go to fb_list
int mixed_launch_2d(mm_ctx *ctx, const WeightsJob &job, int *fb_count, int *fb_list);
int mixed_launch_3d(mm_ctx *ctx, const WeightsJob &job, int *fb_count, int *fb_list);
// GWLS weights (wls.cu) of a validated job (k unused)
int wls_launch(mm_ctx *ctx, const WeightsJob &job, double sigma, int scale);
int mixed_init_device_2d(mm_ctx *ctx);
int mixed_init_device_3d(mm_ctx *ctx);
int weights_launch_scratch(mm_ctx *ctx, const WeightsJob &job, int precision, int *fb_count,
                           int *fb_list);
int spmv_launch(mm_ctx *ctx, const mm_csr_pattern *p, const double *vals, const double *u,
                double alpha, double beta, double *y);
int diffuse_launch(mm_ctx *ctx, const mm_csr_pattern *p, const double *vals, const uint8_t *fixed,
                   const double *g, int neumann, double dt, int steps, double *u, double *work);
int combine_launch(mm_ctx *ctx, const mm_csr_pattern *p, int64_t row_begin, int64_t row_end, int nterms,
                   const double *const *terms, const double *const *coefs, double *out);
int peaks_measure(mm_ctx *ctx, int which, double *flops_per_s);

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(const mm_ctx *ctx) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (ctx && prev != ctx->device) cudaSetDevice(ctx->device);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int weights_job_from_args(mm_ctx *ctx, unsigned ops, int k, int m, int dim, int64_t N,
                          const double *d_pts, const double *d_normals,
                          const mm_csr_pattern *stencils, int64_t row_begin, int64_t row_end,
                          int n_max, double *const *d_vals, int32_t *d_status, WeightsJob *job,
                          bool wls = false);

// Number of monomials of total degree <= m in dim variables: C(m+dim, dim).
inline int mm_num_monomials(int dim, int m) {
    long long c = 1;
    for (int i = 1; i <= dim; ++i) c = c * (m + i) / i;
    return (int)c;
}
