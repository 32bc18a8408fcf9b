// The FP32 + refinement weights kernel of one stencil class (one warp per
// stencil), instantiated for one dimension per translation unit (mixed2d.cu,
// mixed3d.cu) so the instantiations compile in parallel.  Rows the solver
// hands over go to fb_list (the caller launches the FP64 solver on them).
#include "rbffd_dev.cuh"

namespace {

// The register-resident inverse (W > 0) is held to 168 registers, which
// keeps three blocks of four warps per SM (the shared-memory limit).
template <int DIM, int RPL, int R, int W>
__global__ void __launch_bounds__(128, W > 0 ? 3 : 1) k_weights_mixed(WParams P) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const MixedLayout Ly = mixed_layout(P.n_max, P.l, R, DIM);
    char *base = (char *)smem + (size_t)wib * Ly.bytes;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = P.row_begin + gw; row < P.row_end; row += nw) {
        if (mixed_row<DIM, RPL, R, W>(P, row, base) && lane == 0) {
            const int slot = atomicAdd(P.fb_count, 1);
            P.fb_list[slot] = (int)row;
        }
        __syncwarp();
    }
}


template <int DIM, int RPL, int R, int W>
int launch_mixed_t(mm_ctx *ctx, const WParams &P, int64_t rows) {
    const MixedLayout Ly = mixed_layout(P.n_max, P.l, R, DIM);
    auto kern = k_weights_mixed<DIM, RPL, R, W>;
    const int wpb = mm_warps_per_block(ctx, (const void *)kern, Ly.bytes, 4);
    const size_t sm = Ly.bytes * wpb;
    if (sm > ctx->smem_optin) return mm_fail(ctx, MM_EUNSUPPORTED, "stencil too large for shared memory");
    MM_CUDA_CHECK(ctx, mm_set_smem(ctx, (const void *)kern, sm));
    const int blocks = (int)std::min<int64_t>((rows + wpb - 1) / wpb, (int64_t)ctx->num_sms * 32);
    kern<<<blocks, wpb * 32, sm, ctx->stream>>>(P);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

template <int DIM, int RPL, int W = 0>
int launch_mixed_r(mm_ctx *ctx, const WParams &P, int64_t rows) {
    switch (P.R) {
        case 1: return launch_mixed_t<DIM, RPL, 1, W>(ctx, P, rows);
        case 2: return launch_mixed_t<DIM, RPL, 2, W>(ctx, P, rows);
        case 3: return launch_mixed_t<DIM, RPL, 3, W>(ctx, P, rows);
        case 4: return launch_mixed_t<DIM, RPL, 4, W>(ctx, P, rows);
        default: return launch_mixed_t<DIM, RPL, 5, W>(ctx, P, rows);
    }
}

// Systems of 33..48 unknowns (two rows per lane) invert with the rows in
// registers (40 or 48 columns); other sizes, or MM_GJ_SHARED, use the
// shared-memory form.
template <int DIM>
int launch_mixed(mm_ctx *ctx, const WParams &P, int64_t rows) {
    const int rpl = (P.M_max + 31) / 32;
    const int w4 = 4 * ((P.M_max + 3) / 4);
    if (rpl <= 1) return launch_mixed_r<DIM, 1>(ctx, P, rows);
    if (rpl == 2) {
        if (!ctx->gj_shared && w4 == 40) return launch_mixed_r<DIM, 2, 40>(ctx, P, rows);
        if (!ctx->gj_shared && w4 == 48) return launch_mixed_r<DIM, 2, 48>(ctx, P, rows);
        return launch_mixed_r<DIM, 2>(ctx, P, rows);
    }
    return launch_mixed_r<DIM, 3>(ctx, P, rows);
}

// Uploads this translation unit's monomial table to the current device.
int mixed_init(mm_ctx *ctx) {
    MonoTable t;
    mono_table_host(t);
    MM_CUDA_CHECK(ctx, cudaMemcpyToSymbol(c_mono, &t, sizeof(t)));
    return MM_OK;
}

template <int DIM>
int mixed_launch(mm_ctx *ctx, const WeightsJob &job, int *fb_count, int *fb_list) {
    WParams P = wparams_from_job(ctx, job);
    P.fb_count = fb_count;
    P.fb_list = fb_list;
    return launch_mixed<DIM>(ctx, P, job.row_end - job.row_begin);
}

}  // namespace
