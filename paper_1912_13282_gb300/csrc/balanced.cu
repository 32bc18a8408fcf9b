// Balanced stencils (Section 3.1 names FindBalancedSupport, stencils
// "balanced around the central node"; the paper gives no rule, this is the
// library's reading): the K nearest nodes of a query c (the kNN ranking, c
// first) are the candidates; every other candidate j lies in the orthant
// o(j) = sum_a 2^a [x_j,a - x_c,a < 0]; each orthant may contribute its
// first quota = (n - 1) / 2^dim candidates in ranking order, and the slots
// left over go to the nearest candidates not yet taken.  The row is c and
// the taken candidates in ranking order.
//
// One warp per row: the K <= 64 candidates sit two per lane in ranking
// order; a candidate's rank inside its orthant, and its rank among the
// candidates not taken by the quota, are ballot prefix counts, so the
// selection takes no loop over the candidates.
#include <algorithm>
#include <new>

#include "mm_internal.cuh"

namespace {

template <int DIM>
__global__ void __launch_bounds__(256) k_balanced(const double *__restrict__ pts, const int32_t *__restrict__ cand,
                                                  int64_t rows, int K, int n, int32_t *__restrict__ out,
                                                  int64_t q_begin, int32_t *status) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int quota = (n - 1) >> DIM;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < rows; r += nw) {
        const int32_t *cr = cand + r * K;
        const int c = cr[0];
        int id[2], orth[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int t = lane + 32 * s;
            id[s] = (t >= 1 && t < K) ? cr[t] : -1;
            orth[s] = -1;
            if (id[s] >= 0) {
                int o = 0;
#pragma unroll
                for (int a = 0; a < DIM; ++a)
                    if (pts[(int64_t)id[s] * DIM + a] - pts[(int64_t)c * DIM + a] < 0.0) o |= 1 << a;
                orth[s] = o;
            }
        }
        // quota pass: rank inside the orthant, in ranking order
        bool take[2] = {false, false};
#pragma unroll
        for (int o = 0; o < (1 << DIM); ++o) {
            const unsigned m0 = __ballot_sync(0xffffffffu, orth[0] == o);
            const unsigned m1 = __ballot_sync(0xffffffffu, orth[1] == o);
            if (orth[0] == o) take[0] = __popc(m0 & lt) < quota;
            if (orth[1] == o) take[1] = __popc(m0) + __popc(m1 & lt) < quota;
        }
        const unsigned t0 = __ballot_sync(0xffffffffu, take[0]), t1 = __ballot_sync(0xffffffffu, take[1]);
        const int need = n - 1 - (__popc(t0) + __popc(t1));
        // fill pass: the nearest candidates not taken yet
        const bool rest0 = id[0] >= 0 && !take[0], rest1 = id[1] >= 0 && !take[1];
        const unsigned f0 = __ballot_sync(0xffffffffu, rest0), f1 = __ballot_sync(0xffffffffu, rest1);
        if (rest0 && __popc(f0 & lt) < need) take[0] = true;
        if (rest1 && __popc(f0) + __popc(f1 & lt) < need) take[1] = true;
        const unsigned s0 = __ballot_sync(0xffffffffu, take[0]), s1 = __ballot_sync(0xffffffffu, take[1]);
        const int got = __popc(s0) + __popc(s1);
        int32_t *orow = out + r * n;
        if (take[0]) orow[1 + __popc(s0 & lt)] = id[0];
        if (take[1]) orow[1 + __popc(s0) + __popc(s1 & lt)] = id[1];
        for (int w = 1 + got + lane; w < n; w += 32) orow[w] = -1;
        if (lane == 0) {
            orow[0] = c;
            if (status && got < n - 1) status[q_begin + r] = MM_ST_BADARG;
        }
    }
}

}  // namespace

extern "C" int mm_balanced_stencils(mm_ctx *ctx, int dim, int64_t N, const double *d_pts, int nranges,
                                    const mm_knn_range *ranges, int K, int method, int32_t *d_status) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (dim != 2 && dim != 3) return mm_fail(ctx, MM_EBADARG, "dim must be 2 or 3");
    if (N < 1 || N >= (int64_t(1) << 31) || !d_pts) return mm_fail(ctx, MM_EBADARG, "bad points");
    if (nranges < 0 || (nranges > 0 && !ranges)) return mm_fail(ctx, MM_EBADARG, "bad ranges");
    if (K < 1 || K > 64) return mm_fail(ctx, MM_EUNSUPPORTED, "K = %d outside [1, 64]", K);
    if (K > N) return mm_fail(ctx, MM_EBADARG, "K > N");
    int64_t total = 0;
    for (int r = 0; r < nranges; ++r) {
        const mm_knn_range &R = ranges[r];
        if (R.q_begin < 0 || R.q_end < R.q_begin || R.q_end > N)
            return mm_fail(ctx, MM_EBADARG, "range %d out of [0, N)", r);
        if (R.n < 1 || R.n > K) return mm_fail(ctx, MM_EBADARG, "range %d: n must be in [1, K]", r);
        if (R.q_end > R.q_begin && !R.d_idx) return mm_fail(ctx, MM_EBADARG, "range %d: d_idx NULL", r);
        total += R.q_end - R.q_begin;
    }
    if (total == 0) return MM_OK;
    DeviceGuard g(ctx);
    int32_t *cand = (int32_t *)mm_workspace2(ctx, (size_t)total * K * sizeof(int32_t));
    if (!cand) return mm_fail(ctx, MM_ENOMEM, "candidate buffer of %lld x %d", (long long)total, K);
    // candidates: the K nearest nodes of every query, ranges one after another
    mm_knn_range *cr = new (std::nothrow) mm_knn_range[nranges];
    if (!cr) return mm_fail(ctx, MM_ENOMEM, "range table");
    int64_t off = 0;
    for (int r = 0; r < nranges; ++r) {
        cr[r] = ranges[r];
        cr[r].n = K;
        cr[r].d_idx = cand + off * K;
        off += ranges[r].q_end - ranges[r].q_begin;
    }
    int rc = knn_launch(ctx, dim, N, d_pts, nranges, cr, method, d_status);
    delete[] cr;
    if (rc != MM_OK) return rc;
    off = 0;
    for (int r = 0; r < nranges && rc == MM_OK; ++r) {
        const mm_knn_range &R = ranges[r];
        const int64_t rows = R.q_end - R.q_begin;
        if (rows > 0) {
            const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, (int64_t)ctx->num_sms * 16));
            if (dim == 2)
                k_balanced<2><<<blocks, 256, 0, ctx->stream>>>(d_pts, cand + off * K, rows, K, R.n, R.d_idx,
                                                               R.q_begin, d_status);
            else
                k_balanced<3><<<blocks, 256, 0, ctx->stream>>>(d_pts, cand + off * K, rows, K, R.n, R.d_idx,
                                                               R.q_begin, d_status);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) rc = mm_fail(ctx, MM_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
        }
        off += rows;
    }
    return rc;
}
