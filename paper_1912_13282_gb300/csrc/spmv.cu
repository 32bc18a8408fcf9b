// Operator application (Section 2.3.1 of the paper, explicit evaluation
// w^T u_I(i)): CSR SpMV y = alpha L u + beta y, and explicit Euler steps
// u <- u + dt L u on free rows (eq. exp-start .. exp-end, Dirichlet rows held).
//
// A group of G lanes (G a power of two, chosen from the mean row length)
// handles a row: the lanes read consecutive value/column entries of the row
// (coalesced), gather u, and reduce with shuffles inside the group.  The
// kernel is bound by HBM traffic: 12 bytes per nonzero (value + column), the
// row pointer, the y write, and the u gather (mostly cache hits when stencil
// neighbours have nearby indices).
#include <algorithm>

#include "mm_internal.cuh"

namespace {

// A group of G lanes takes RB consecutive rows per iteration, their loads
// interleaved, so several independent chains of dependent loads (row pointer,
// value/column, gathered u) are in flight per group.  Narrow groups (4 lanes
// for stencil rows of 10-48 nonzeros: one 32-byte sector of values per load)
// measured best on the 1e6-node disk operator: 3.2 TB/s against 1.4 TB/s
// with 16 lanes per row.
constexpr int RB = 2;

template <int G>
__device__ __forceinline__ void rows_dot(int64_t base, int64_t nrows, int sub, const int64_t *__restrict__ rp,
                                         const int32_t *__restrict__ col, const double *__restrict__ val,
                                         const double *__restrict__ u, double (&acc)[RB]) {
    int64_t b[RB], e[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const bool in = base + r < nrows;
        b[r] = in ? __ldg(rp + base + r) : 0;
        e[r] = in ? __ldg(rp + base + r + 1) : 0;
        acc[r] = 0.0;
    }
    int64_t p[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) p[r] = b[r] + sub;
    bool more = true;
    while (more) {
        more = false;
#pragma unroll
        for (int r = 0; r < RB; ++r)
            if (p[r] < e[r]) {
                acc[r] = fma(__ldg(val + p[r]), __ldg(u + __ldg(col + p[r])), acc[r]);
                p[r] += G;
                more |= p[r] < e[r];
            }
    }
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int o = G / 2; o; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o, G);
}

template <int G>
__global__ void __launch_bounds__(256) k_spmv(int64_t nrows, const int64_t *__restrict__ rp,
                                              const int32_t *__restrict__ col,
                                              const double *__restrict__ val,
                                              const double *__restrict__ u, double alpha,
                                              double beta, double *__restrict__ y) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int sub = threadIdx.x & (G - 1);
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
    for (int64_t base = (tid / G) * RB; base < nrows; base += ngroups * RB) {
        double acc[RB];
        rows_dot<G>(base, nrows, sub, rp, col, val, u, acc);
#pragma unroll
        for (int r = 0; r < RB; ++r)
            if (r % G == sub && base + r < nrows) {
                const int64_t row = base + r;
                y[row] = beta == 0.0 ? alpha * acc[r] : fma(alpha, acc[r], beta * y[row]);
            }
    }
}

template <int G>
__global__ void __launch_bounds__(256) k_diffuse_step(int64_t nrows, const int64_t *__restrict__ rp,
                                                      const int32_t *__restrict__ col,
                                                      const double *__restrict__ val,
                                                      const uint8_t *__restrict__ fixed,
                                                      const double *__restrict__ u, double dt,
                                                      double *__restrict__ unew) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int sub = threadIdx.x & (G - 1);
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
    for (int64_t base = (tid / G) * RB; base < nrows; base += ngroups * RB) {
        double acc[RB];
        rows_dot<G>(base, nrows, sub, rp, col, val, u, acc);
#pragma unroll
        for (int r = 0; r < RB; ++r)
            if (r % G == sub && base + r < nrows) {
                const int64_t row = base + r;
                unew[row] = fixed[row] ? u[row] : fma(dt, acc[r], u[row]);
            }
    }
}

int group_for(const mm_csr_pattern *p) {
    double avg = p->nrows > 0 ? (double)p->nnz / (double)p->nrows : 1.0;
    return avg >= 48 ? 8 : 4;
}

// one wave at full occupancy (8 blocks of 256 threads per SM), fewer for small matrices
int grid_for(mm_ctx *ctx, int64_t nrows, int G) {
    int64_t need = ((nrows + RB - 1) / RB * G + 255) / 256;
    int64_t cap = (int64_t)ctx->num_sms * 8;
    return (int)std::max<int64_t>(1, std::min(need, cap));
}

}  // namespace

int spmv_launch(mm_ctx *ctx, const mm_csr_pattern *p, const double *vals, const double *u,
                double alpha, double beta, double *y) {
    if (p->nrows == 0) return MM_OK;
    const int G = group_for(p);
    const int blocks = grid_for(ctx, p->nrows, G);
    cudaStream_t st = ctx->stream;
    switch (G) {
        case 8: k_spmv<8><<<blocks, 256, 0, st>>>(p->nrows, p->d_row_ptr, p->d_col, vals, u, alpha, beta, y); break;
        default: k_spmv<4><<<blocks, 256, 0, st>>>(p->nrows, p->d_row_ptr, p->d_col, vals, u, alpha, beta, y); break;
    }
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

int diffuse_launch(mm_ctx *ctx, const mm_csr_pattern *p, const double *vals, const uint8_t *fixed,
                   double dt, int steps, double *u, double *work) {
    if (p->nrows == 0 || steps <= 0) return MM_OK;
    const int G = group_for(p);
    const int blocks = grid_for(ctx, p->nrows, G);
    cudaStream_t st = ctx->stream;
    double *src = u, *dst = work;
    for (int t = 0; t < steps; ++t) {
        switch (G) {
            case 8: k_diffuse_step<8><<<blocks, 256, 0, st>>>(p->nrows, p->d_row_ptr, p->d_col, vals, fixed, src, dt, dst); break;
            default: k_diffuse_step<4><<<blocks, 256, 0, st>>>(p->nrows, p->d_row_ptr, p->d_col, vals, fixed, src, dt, dst); break;
        }
        MM_LAUNCH_CHECK(ctx);
        double *t2 = src; src = dst; dst = t2;
    }
    if (src != u)
        MM_CUDA_CHECK(ctx, cudaMemcpyAsync(u, src, sizeof(double) * (size_t)p->nrows,
                                           cudaMemcpyDeviceToDevice, st));
    return MM_OK;
}
