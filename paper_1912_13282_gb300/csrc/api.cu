// The C ABI (mm.h): argument validation on the host, context and workspace
// management, dispatch to the kernels.  No exception leaves this file.
#include <stdarg.h>
#include <math.h>
#include <stdio.h>

#include <map>
#include <mutex>
#include <tuple>
#include <new>

#include "mm_internal.cuh"

int rbffd_init_device(mm_ctx *ctx);
int batched_init_device(mm_ctx *ctx);
int mlp_init_device(mm_ctx *ctx);
int wls_init_device(mm_ctx *ctx);

int mm_fail(mm_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

int mm_warps_per_block(const mm_ctx *ctx, const void *kernel, size_t bytes_per_warp, int max_wpb) {
    // the occupancy calculator's answer (allocation granularity, registers)
    // per candidate, cached per kernel and size.  Larger blocks measured
    // faster at equal occupancy (one-warp blocks were 15% slower on 25-node
    // stencils at one more warp per SM), so a smaller block is taken only for
    // at least two more resident warps.
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, size_t, int>, int> cache;
    const auto key = std::make_tuple(ctx->device, kernel, bytes_per_warp, max_wpb);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int warps[9] = {0};
    int top = 0;
    for (int w = 1; w <= max_wpb && w <= 8; ++w) {
        const size_t blk = bytes_per_warp * (size_t)w;
        if (blk > ctx->smem_optin) break;
        if (mm_set_smem(ctx, kernel, blk) != cudaSuccess) break;
        int blocks = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, 32 * w, blk) != cudaSuccess) {
            cudaGetLastError();
            break;
        }
        warps[w] = blocks * w;
        top = w;
    }
    int best = top > 0 ? top : 1;
    for (int w = top - 1; w >= 1; --w)
        if (warps[w] >= warps[best] + 2) best = w;
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = best;
    return best;
}

char *mm_workspace(mm_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return ctx->ws;
    size_t want = bytes + bytes / 4 + (1 << 20);
    if (ctx->ws) {
        cudaStreamSynchronize(ctx->stream);   // queued kernels may still use it
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return nullptr;
    }
    ctx->ws_bytes = want;
    return ctx->ws;
}

char *mm_workspace2(mm_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->ws2_bytes) return ctx->ws2;
    size_t want = bytes + bytes / 4 + (1 << 20);
    if (ctx->ws2) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->ws2);
        ctx->ws2 = nullptr;
        ctx->ws2_bytes = 0;
    }
    if (cudaMalloc(&ctx->ws2, want) != cudaSuccess) {
        cudaGetLastError();
        ctx->ws2 = nullptr;
        return nullptr;
    }
    ctx->ws2_bytes = want;
    return ctx->ws2;
}

cudaError_t mm_set_smem(const mm_ctx *ctx, const void *kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> done;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair(ctx->device, kernel);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done[key] = bytes;
    return e;
}

namespace {

bool bad_dim(int dim) { return dim != 2 && dim != 3; }

}  // namespace

int weights_job_from_args(mm_ctx *ctx, unsigned ops, int k, int m, int dim, int64_t N,
                          const double *d_pts, const double *d_normals,
                          const mm_csr_pattern *stencils, int64_t row_begin, int64_t row_end,
                          int n_max, double *const *d_vals, int32_t *d_status, WeightsJob *job,
                          bool wls) {
    if (bad_dim(dim)) return mm_fail(ctx, MM_EBADARG, "dim must be 2 or 3");
    if (ops == 0 || ops >= 2048u) return mm_fail(ctx, MM_EBADARG, "ops must be a nonzero MM_* bitmask");
    if ((ops & (MM_DZ | MM_DXZ | MM_DYZ | MM_DZZ)) && dim != 3)
        return mm_fail(ctx, MM_EBADARG, "z derivatives need dim 3");
    if ((ops & (MM_DXX | MM_DXY | MM_DYY | MM_DXZ | MM_DYZ | MM_DZZ)) && m < 2)
        return mm_fail(ctx, MM_EBADARG, "second derivatives need monomials of degree >= 2");
    if ((ops & MM_DN) && !d_normals) return mm_fail(ctx, MM_EBADARG, "MM_DN needs d_normals");
    if (!wls && k != 3 && k != 5 && k != 7) return mm_fail(ctx, MM_EBADARG, "k must be 3, 5 or 7");
    if (m < 0 || m > 6) return mm_fail(ctx, MM_EBADARG, "m must be in [0, 6]");
    if (N < 1 || N >= (int64_t(1) << 31) || !d_pts) return mm_fail(ctx, MM_EBADARG, "bad points");
    if (!stencils || !stencils->d_row_ptr || !stencils->d_col)
        return mm_fail(ctx, MM_EBADARG, "bad stencil pattern");
    if (row_begin < 0 || row_end < row_begin || row_end > stencils->nrows || stencils->nrows > N)
        return mm_fail(ctx, MM_EBADARG, "row range out of [0, nrows]");
    if (n_max < 1) return mm_fail(ctx, MM_EBADARG, "n_max < 1");
    if (!d_vals) return mm_fail(ctx, MM_EBADARG, "d_vals is NULL");
    WeightsJob &J = *job;
    J = WeightsJob{};
    J.ops = ops;
    J.k = k;
    J.m = m;
    J.dim = dim;
    J.N = N;
    J.pts = d_pts;
    J.normals = d_normals;
    J.row_ptr = stencils->d_row_ptr;
    J.col = stencils->d_col;
    J.row_begin = row_begin;
    J.row_end = row_end;
    J.n_max = n_max;
    J.status = d_status;
    int r = 0;
    for (int b = 0; b < 11; ++b) {
        J.vals[b] = nullptr;
        if (ops & (1u << b)) {
            if (!d_vals[r]) return mm_fail(ctx, MM_EBADARG, "d_vals[%d] is NULL", r);
            J.vals[b] = d_vals[r++];
        }
    }
    if (wls) {
        if (n_max > 64) return mm_fail(ctx, MM_EUNSUPPORTED, "n_max = %d > 64", n_max);
    } else if (n_max + mm_num_monomials(dim, m) > 96) {
        return mm_fail(ctx, MM_EUNSUPPORTED, "n_max + l = %d > 96", n_max + mm_num_monomials(dim, m));
    }
    return MM_OK;
}

extern "C" {

int mm_ctx_create(mm_ctx **out, int device, void *cuda_stream) {
    if (!out) return MM_EBADARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return MM_ECUDA;
    }
    mm_ctx *ctx = new (std::nothrow) mm_ctx();
    if (!ctx) return MM_ENOMEM;
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    DeviceGuard g(ctx);
    int sms = 0, optin = 0, per_sm = 0, reserved = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device) != cudaSuccess) {
        delete ctx;
        return MM_ECUDA;
    }
    ctx->num_sms = sms;
    ctx->smem_per_sm = (size_t)per_sm;
    ctx->smem_reserved = (size_t)reserved;
    ctx->smem_optin = (size_t)optin;
    if (rbffd_init_device(ctx) != MM_OK || batched_init_device(ctx) != MM_OK ||
        mlp_init_device(ctx) != MM_OK || mixed_init_device_2d(ctx) != MM_OK ||
        mixed_init_device_3d(ctx) != MM_OK || wls_init_device(ctx) != MM_OK) {
        delete ctx;
        return MM_ECUDA;
    }
    *out = ctx;
    return MM_OK;
}

void mm_ctx_destroy(mm_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->ws2) cudaFree(ctx->ws2);
    delete ctx;
}

int mm_ctx_set_stream(mm_ctx *ctx, void *cuda_stream) {
    if (!ctx) return MM_EBADARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return MM_OK;
}

int mm_ctx_set_option(mm_ctx *ctx, int key, double value) {
    if (!ctx) return MM_EBADARG;
    switch (key) {
        case MM_OPT_IR_TOL:
            if (!(value > 0 && value < 1)) return mm_fail(ctx, MM_EBADARG, "IR tolerance must be in (0,1)");
            ctx->ir_tol = value;
            return MM_OK;
        case MM_OPT_IR_MAX_STEPS:
            if (!(value >= 0 && value <= 32)) return mm_fail(ctx, MM_EBADARG, "IR steps must be in [0,32]");
            ctx->ir_max_steps = (int)value;
            return MM_OK;
        case MM_OPT_KAPPA_MAX:
            if (!(value > 0)) return mm_fail(ctx, MM_EBADARG, "kappa threshold must be > 0");
            ctx->kappa_max = value;
            return MM_OK;
        case MM_OPT_WIDE:
            if (value != MM_WIDE_FF && value != MM_WIDE_FP64)
                return mm_fail(ctx, MM_EBADARG, "wide arithmetic must be MM_WIDE_FF or MM_WIDE_FP64");
            ctx->wide64 = value == MM_WIDE_FP64;
            return MM_OK;
        case MM_OPT_MLP_INFER:
            if (value != MM_MLP_FUSED && value != MM_MLP_LAYERED)
                return mm_fail(ctx, MM_EBADARG, "MLP inference must be MM_MLP_FUSED or MM_MLP_LAYERED");
            ctx->mlp_layered = value == MM_MLP_LAYERED;
            return MM_OK;
        case MM_OPT_GJ:
            if (value != MM_GJ_AUTO && value != MM_GJ_SHARED)
                return mm_fail(ctx, MM_EBADARG, "Gauss-Jordan storage must be MM_GJ_AUTO or MM_GJ_SHARED");
            ctx->gj_shared = value == MM_GJ_SHARED;
            return MM_OK;
    }
    return mm_fail(ctx, MM_EBADARG, "unknown option %d", key);
}

const char *mm_last_error(const mm_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t mm_ctx_workspace_bytes(const mm_ctx *ctx) {
    return ctx ? (int64_t)(ctx->ws_bytes + ctx->ws2_bytes) : -1;
}

int mm_knn_stencils(mm_ctx *ctx, int dim, int64_t N, const double *d_pts, int nranges,
                    const mm_knn_range *ranges, int method, int32_t *d_status) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (bad_dim(dim)) return mm_fail(ctx, MM_EBADARG, "dim must be 2 or 3");
    if (N < 1 || N >= (int64_t(1) << 31)) return mm_fail(ctx, MM_EBADARG, "N out of range");
    if (!d_pts) return mm_fail(ctx, MM_EBADARG, "d_pts is NULL");
    if (nranges < 0 || (nranges > 0 && !ranges)) return mm_fail(ctx, MM_EBADARG, "bad ranges");
    if (method < MM_KNN_AUTO || method > MM_KNN_GRID) return mm_fail(ctx, MM_EBADARG, "bad method");
    for (int r = 0; r < nranges; ++r) {
        const mm_knn_range &R = ranges[r];
        if (R.q_begin < 0 || R.q_end < R.q_begin || R.q_end > N)
            return mm_fail(ctx, MM_EBADARG, "range %d out of [0, N)", r);
        if (R.n < 1) return mm_fail(ctx, MM_EBADARG, "range %d: n < 1", r);
        if (R.n > 64) return mm_fail(ctx, MM_EUNSUPPORTED, "range %d: n = %d > 64", r, R.n);
        if (R.n > N) return mm_fail(ctx, MM_EBADARG, "range %d: n > N", r);
        if (R.q_end > R.q_begin && !R.d_idx) return mm_fail(ctx, MM_EBADARG, "range %d: d_idx NULL", r);
    }
    DeviceGuard g(ctx);
    return knn_launch(ctx, dim, N, d_pts, nranges, ranges, method, d_status);
}

int mm_rbffd_weights(mm_ctx *ctx, unsigned ops, int k, int m, int dim, int64_t N,
                     const double *d_pts, const double *d_normals, const mm_csr_pattern *stencils,
                     int64_t row_begin, int64_t row_end, int n_max, int precision,
                     double *const *d_vals, int32_t *d_status) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (precision != MM_FP64 && precision != MM_FP32_IR)
        return mm_fail(ctx, MM_EBADARG, "unknown precision %d", precision);
    WeightsJob job{};
    int rc = weights_job_from_args(ctx, ops, k, m, dim, N, d_pts, d_normals, stencils, row_begin,
                                   row_end, n_max, d_vals, d_status, &job);
    if (rc != MM_OK) return rc;
    DeviceGuard g(ctx);
    return weights_launch(ctx, job, precision);
}

int mm_wls_weights(mm_ctx *ctx, unsigned ops, int m, double sigma, int scale, int dim, int64_t N,
                   const double *d_pts, const double *d_normals, const mm_csr_pattern *stencils,
                   int64_t row_begin, int64_t row_end, int n_max, double *const *d_vals,
                   int32_t *d_status) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (!(sigma > 0.0) || !isfinite(sigma)) return mm_fail(ctx, MM_EBADARG, "sigma must be finite and > 0");
    if (scale != MM_SCALE_FARTHEST && scale != MM_SCALE_NEAREST)
        return mm_fail(ctx, MM_EBADARG, "scale must be MM_SCALE_FARTHEST or MM_SCALE_NEAREST");
    WeightsJob job{};
    int rc = weights_job_from_args(ctx, ops, 3, m, dim, N, d_pts, d_normals, stencils, row_begin,
                                   row_end, n_max, d_vals, d_status, &job, true);
    if (rc != MM_OK) return rc;
    DeviceGuard g(ctx);
    return wls_launch(ctx, job, sigma, scale);
}

int mm_apply_operator(mm_ctx *ctx, const mm_csr_pattern *stencils, const double *d_vals,
                      const double *d_u, double alpha, double beta, double *d_y) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (!stencils || !stencils->d_row_ptr || !stencils->d_col || stencils->nrows < 0)
        return mm_fail(ctx, MM_EBADARG, "bad stencil pattern");
    if (stencils->nrows > 0 && (!d_vals || !d_u || !d_y))
        return mm_fail(ctx, MM_EBADARG, "NULL vector or values");
    if (d_u == d_y && stencils->nrows > 0) return mm_fail(ctx, MM_EBADARG, "d_y aliases d_u");
    DeviceGuard g(ctx);
    return spmv_launch(ctx, stencils, d_vals, d_u, alpha, beta, d_y);
}

int mm_diffuse(mm_ctx *ctx, const mm_csr_pattern *stencils, const double *d_vals,
               const uint8_t *d_fixed, double dt, int steps, double *d_u, double *d_work) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (!stencils || !stencils->d_row_ptr || !stencils->d_col || stencils->nrows < 0)
        return mm_fail(ctx, MM_EBADARG, "bad stencil pattern");
    if (steps < 0) return mm_fail(ctx, MM_EBADARG, "steps < 0");
    if (stencils->nrows > 0 && (!d_vals || !d_fixed || !d_u || !d_work))
        return mm_fail(ctx, MM_EBADARG, "NULL argument");
    if (d_u == d_work && stencils->nrows > 0) return mm_fail(ctx, MM_EBADARG, "d_work aliases d_u");
    DeviceGuard g(ctx);
    return diffuse_launch(ctx, stencils, d_vals, d_fixed, nullptr, 0, dt, steps, d_u, d_work);
}

int mm_diffuse_bc(mm_ctx *ctx, const mm_csr_pattern *stencils, const double *d_vals,
                  const uint8_t *d_kind, const double *d_g, double dt, int steps, double *d_u,
                  double *d_work) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (!stencils || !stencils->d_row_ptr || !stencils->d_col || stencils->nrows < 0)
        return mm_fail(ctx, MM_EBADARG, "bad stencil pattern");
    if (steps < 0) return mm_fail(ctx, MM_EBADARG, "steps < 0");
    if (stencils->nrows > 0 && (!d_vals || !d_kind || !d_u || !d_work))
        return mm_fail(ctx, MM_EBADARG, "NULL argument");
    if (d_u == d_work && stencils->nrows > 0) return mm_fail(ctx, MM_EBADARG, "d_work aliases d_u");
    if (d_g && (d_g == d_u || d_g == d_work)) return mm_fail(ctx, MM_EBADARG, "d_g aliases d_u or d_work");
    DeviceGuard g(ctx);
    return diffuse_launch(ctx, stencils, d_vals, d_kind, d_g, 1, dt, steps, d_u, d_work);
}

int mm_combine_operators(mm_ctx *ctx, const mm_csr_pattern *stencils, int64_t row_begin, int64_t row_end,
                         int nterms, const double *const *d_terms, const double *const *d_coef,
                         double *d_out) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (!stencils || !stencils->d_row_ptr || stencils->nrows < 0)
        return mm_fail(ctx, MM_EBADARG, "bad stencil pattern");
    if (row_begin < 0 || row_end < row_begin || row_end > stencils->nrows)
        return mm_fail(ctx, MM_EBADARG, "row range out of [0, nrows]");
    if (nterms < 1 || nterms > 10) return mm_fail(ctx, MM_EBADARG, "nterms must be in [1, 10]");
    if (!d_terms || !d_out) return mm_fail(ctx, MM_EBADARG, "NULL argument");
    for (int t = 0; t < nterms; ++t)
        if (!d_terms[t]) return mm_fail(ctx, MM_EBADARG, "d_terms[%d] is NULL", t);
    DeviceGuard g(ctx);
    return combine_launch(ctx, stencils, row_begin, row_end, nterms, d_terms, d_coef, d_out);
}

int mm_measure_fma_peak(mm_ctx *ctx, int which, double *flops_per_s) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if ((which != 0 && which != 1) || !flops_per_s) return mm_fail(ctx, MM_EBADARG, "bad arguments");
    DeviceGuard g(ctx);
    return peaks_measure(ctx, which, flops_per_s);
}

}  // extern "C"
