// Operator application (Section 2.3.1 of the paper, explicit evaluation
// w^T u_I(i)): CSR SpMV y = alpha L u + beta y, explicit Euler steps
// u <- u + dt L u on internal rows (eq. exp-start .. exp-end: Dirichlet rows
// held, Neumann rows solved from their own d/dn row), and the general
// second-order operator as a per-node combination of derivative weights
// (eq. gen-op, one warp per 32 rows streaming their entries flat).
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

// kind[i]: 0 internal (u + dt L u), 2 with `neumann` set: the row holds the
// node's d/dn weights, centre first, and u_i <- (g_i - sum_{j>=2} w_ij u_j) /
// w_i1 (eq. exp-end; g may be NULL for 0); any other value keeps u_i.  All
// from the previous step's field.
template <int G>
__global__ void __launch_bounds__(256) k_diffuse_step(int64_t nrows, const int64_t *__restrict__ rp,
                                                      const int32_t *__restrict__ col,
                                                      const double *__restrict__ val,
                                                      const uint8_t *__restrict__ kind,
                                                      const double *__restrict__ g, int neumann,
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
                const int k = kind[row];
                double v = u[row];
                if (k == 0) {
                    v = fma(dt, acc[r], v);
                } else if (k == 2 && neumann) {
                    const double w1 = __ldg(val + __ldg(rp + row));   // centre weight
                    const double rest = fma(-w1, v, acc[r]);          // sum over the other nodes
                    v = ((g ? g[row] : 0.0) - rest) / w1;
                }
                unew[row] = v;
            }
    }
}

// General second-order operator (eq. gen-op): out[e] = sum_t a_t(i) term_t[e]
// for the entries e of row i, a_t(i) = coef_t[i] (1 if coef_t is NULL).  G
// lanes per row read consecutive entries; bound by HBM traffic ((T + 1) x 8
// bytes per nonzero).
constexpr int kMaxTerms = 10;
struct CombineArgs {
    int nterms;
    const double *term[kMaxTerms];
    const double *coef[kMaxTerms];
};

// One warp per 32 consecutive rows: the rows' pointers in one coalesced load,
// then the rows' entries as one flat range, 32 consecutive entries per step
// (every load coalesced and independent of the others); a lane finds the
// row of its entry among the 32 pointers by a shuffle binary search and
// reads that row's coefficients (cached).  Bound by HBM traffic: (T + 1) x 8
// bytes per entry plus the coefficients.
__global__ void __launch_bounds__(256) k_combine(int64_t row_begin, int64_t row_end, const int64_t *__restrict__ rp,
                                                 const __grid_constant__ CombineArgs A, double *out) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = row_begin + (((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) << 5); r0 < row_end;
         r0 += nw * 32) {
        const int nr = (int)(row_end - r0 < 32 ? row_end - r0 : 32);
        // lane l holds the start of row r0 + l (lanes past the block: the end)
        const int64_t start = __ldg(rp + r0 + min(lane, nr));
        const int64_t e_all = __ldg(rp + r0 + nr);
        const int64_t b_all = __shfl_sync(0xffffffffu, start, 0);
        for (int64_t e = b_all + lane; e - lane < e_all; e += 32) {
            // the largest row index q in [0, nr) with start(q) <= e
            int q = 0;
#pragma unroll
            for (int step = 16; step; step >>= 1) {
                const int cand = q + step;
                const int64_t sc = __shfl_sync(0xffffffffu, start, cand < 32 ? cand : 31);
                if (cand < nr && sc <= e) q = cand;
            }
            if (e < e_all) {
                const int64_t row = r0 + q;
                double s = 0.0;
#pragma unroll
                for (int t = 0; t < kMaxTerms; ++t)
                    if (t < A.nterms) s = fma(A.coef[t] ? __ldg(A.coef[t] + row) : 1.0, __ldg(A.term[t] + e), s);
                out[e] = s;
            }
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

int combine_launch(mm_ctx *ctx, const mm_csr_pattern *p, int64_t row_begin, int64_t row_end, int nterms,
                   const double *const *terms, const double *const *coefs, double *out) {
    if (row_end <= row_begin) return MM_OK;
    CombineArgs A{};
    A.nterms = nterms;
    for (int t = 0; t < nterms; ++t) {
        A.term[t] = terms[t];
        A.coef[t] = coefs ? coefs[t] : nullptr;
    }
    const int64_t rows = row_end - row_begin;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 255) / 256, (int64_t)ctx->num_sms * 8));
    k_combine<<<blocks, 256, 0, ctx->stream>>>(row_begin, row_end, p->d_row_ptr, A, out);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

int diffuse_launch(mm_ctx *ctx, const mm_csr_pattern *p, const double *vals, const uint8_t *fixed,
                   const double *g, int neumann, double dt, int steps, double *u, double *work) {
    if (p->nrows == 0 || steps <= 0) return MM_OK;
    const int G = group_for(p);
    const int blocks = grid_for(ctx, p->nrows, G);
    cudaStream_t st = ctx->stream;
    double *src = u, *dst = work;
    for (int t = 0; t < steps; ++t) {
        switch (G) {
            case 8: k_diffuse_step<8><<<blocks, 256, 0, st>>>(p->nrows, p->d_row_ptr, p->d_col, vals, fixed, g, neumann, src, dt, dst); break;
            default: k_diffuse_step<4><<<blocks, 256, 0, st>>>(p->nrows, p->d_row_ptr, p->d_col, vals, fixed, g, neumann, src, dt, dst); break;
        }
        MM_LAUNCH_CHECK(ctx);
        double *t2 = src; src = dst; dst = t2;
    }
    if (src != u)
        MM_CUDA_CHECK(ctx, cudaMemcpyAsync(u, src, sizeof(double) * (size_t)p->nrows,
                                           cudaMemcpyDeviceToDevice, st));
    return MM_OK;
}
