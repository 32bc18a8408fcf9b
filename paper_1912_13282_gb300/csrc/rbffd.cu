// RBF-FD stencil weights on the GPU, one launch per stencil class: one warp
// per stencil (row), FP64 solver or FP32 + refinement solver (mixed2d.cu,
// mixed3d.cu) with a queue of stragglers handed to the FP64 solver (see
// rbffd_dev.cuh for the math).
#include "rbffd_dev.cuh"

namespace {

template <int DIM>
__global__ void __launch_bounds__(128) k_weights_fp64(WParams P) {
    extern __shared__ double smem[];
    const int wib = threadIdx.x >> 5;
    double *base = smem + (size_t)wib * fp64_warp_doubles(P.M_max, P.pitch64, P.n_max, DIM);
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t count = P.list ? (int64_t)*P.list_count : P.row_end - P.row_begin;
    for (int64_t t = gw; t < count; t += nw) {
        const int64_t row = P.list ? (int64_t)P.list[t] : P.row_begin + t;
        fp64_row<DIM>(P, row, base, P.list != nullptr);
    }
}

}  // namespace

// Uploads the monomial table to the current device.
int rbffd_init_device(mm_ctx *ctx) {
    MonoTable t;
    mono_table_host(t);
    MM_CUDA_CHECK(ctx, cudaMemcpyToSymbol(c_mono, &t, sizeof(t)));
    return MM_OK;
}

// fb_count/fb_list: caller-provided queue for rows the FP32 path hands to the
// FP64 solve ([1] and [rows] ints); nullptr takes them from the context
// workspace.
int weights_launch_scratch(mm_ctx *ctx, const WeightsJob &job, int precision, int *fb_count,
                           int *fb_list) {
    if (__builtin_popcount(job.ops) > 5) {
        // more than 5 operators: launches of at most 5 right-hand-side columns
        // each, in bit order (the factorization is repeated per launch; a
        // row's status is the last launch's)
        unsigned rest = job.ops;
        while (rest) {
            unsigned part = 0;
            for (int b = 0, c = 0; b < 11 && c < 5; ++b)
                if (rest & (1u << b)) { part |= 1u << b; ++c; }
            WeightsJob sub = job;
            sub.ops = part;
            const int rc = weights_launch_scratch(ctx, sub, precision, fb_count, fb_list);
            if (rc != MM_OK) return rc;
            rest &= ~part;
        }
        return MM_OK;
    }
    const int dim = job.dim;
    WParams P = wparams_from_job(ctx, job);
    if (P.M_max > kMaxM) return mm_fail(ctx, MM_EUNSUPPORTED, "n_max + l = %d > %d", P.M_max, kMaxM);
    const int64_t rows = job.row_end - job.row_begin;
    if (rows <= 0) return MM_OK;
    cudaStream_t st = ctx->stream;
    const size_t w64 = fp64_warp_doubles(P.M_max, P.pitch64, P.n_max, dim) * sizeof(double);
    auto warps_for = [&](size_t per_warp) {
        int w = (int)std::min<size_t>(4, (96 * 1024) / per_warp);
        return max(w, 1);
    };
    auto launch_fp64 = [&](const int *list, const int *list_count, int64_t max_rows) -> int {
        WParams Q = P;
        Q.list = list;
        Q.list_count = list_count;
        int wpb = warps_for(w64);
        size_t sm = w64 * wpb;
        if (sm > ctx->smem_optin) return mm_fail(ctx, MM_EUNSUPPORTED, "stencil too large for shared memory");
        int blocks = (int)std::min<int64_t>((max_rows + wpb - 1) / wpb, (int64_t)ctx->num_sms * 32);
        blocks = max(blocks, 1);
        if (dim == 2) {
            MM_CUDA_CHECK(ctx, mm_set_smem(ctx, (const void *)k_weights_fp64<2>, sm));
            k_weights_fp64<2><<<blocks, wpb * 32, sm, st>>>(Q);
        } else {
            MM_CUDA_CHECK(ctx, mm_set_smem(ctx, (const void *)k_weights_fp64<3>, sm));
            k_weights_fp64<3><<<blocks, wpb * 32, sm, st>>>(Q);
        }
        MM_LAUNCH_CHECK(ctx);
        return MM_OK;
    };
    if (precision == MM_FP64) return launch_fp64(nullptr, nullptr, rows);

    // mixed: FP32 inverse + FP64-residual refinement, queue stragglers for FP64
    if (fb_count && fb_list) {
        P.fb_count = fb_count;
        P.fb_list = fb_list;
    } else {
        WsCarve wc;
        size_t o_cnt = wc.take<int>(1);
        size_t o_list = wc.take<int>((size_t)rows);
        char *ws = mm_workspace(ctx, wc.off);
        if (!ws) return mm_fail(ctx, MM_ENOMEM, "weights workspace of %zu bytes", wc.off);
        P.fb_count = (int *)(ws + o_cnt);
        P.fb_list = (int *)(ws + o_list);
    }
    MM_CUDA_CHECK(ctx, cudaMemsetAsync(P.fb_count, 0, sizeof(int), st));
    {
        const int rc = dim == 2 ? mixed_launch_2d(ctx, job, P.fb_count, P.fb_list)
                                : mixed_launch_3d(ctx, job, P.fb_count, P.fb_list);
        if (rc != MM_OK) return rc;
    }
    return launch_fp64(P.fb_list, P.fb_count, rows);
}

int weights_launch(mm_ctx *ctx, const WeightsJob &job, int precision) {
    return weights_launch_scratch(ctx, job, precision, nullptr, nullptr);
}
