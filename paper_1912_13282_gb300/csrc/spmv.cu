// Operator application (Section 2.3.1 of the paper, explicit evaluation
// w^T u_I(i)): CSR SpMV y = alpha L u + beta y, explicit Euler steps
// u <- u + dt L u on internal rows (eq. exp-start .. exp-end: Dirichlet rows
// held, Neumann rows solved from their own d/dn row), and the general
// second-order operator as a per-node combination of derivative weights
// (eq. gen-op, one warp per 32 rows streaming their entries flat).
//
// A group of G lanes (G a power of two, chosen from the mean row length)
// handles a row: the lanes read interleaved value/column entries of the row
// (all of a lane's entries of a batch at once), gather u, and reduce with
// shuffles inside the group.  The traffic is 12 bytes per nonzero (value +
// column), the row pointer, the y write and the u gather (mostly cache hits
// when stencil neighbours have nearby indices); on GB300 the FP64 pipe (one
// multiply-add per nonzero) bounds it about as much as HBM does.
#include <algorithm>

#include "mm_internal.cuh"

namespace {

// A group of G lanes takes RB consecutive rows per iteration; lane `sub`
// handles the row's entries sub, sub + G, sub + 2G, ... (cnt of them) in
// batches: it issues all value and column loads of a batch, then all gathers
// of u, then the multiply-adds in entry order, so a row costs three dependent
// memory round trips (row pointer, value/column, u).  Batches of 8, then one
// of 4, 2 and 1 as the lane's remaining count allows, so no multiply-add is
// issued for an entry that does not exist: GB300's FP64 pipe (~1/64 of the
// FP32 rate) is the bound of this kernel, one FP64 warp instruction per
// entry batch step plus log2(G) for the group's shuffle reduction, so two
// lanes per row (one reduction step, rows of 25-30 entries split 13/12 or
// 15/15) issue few FP64 instructions per row while a load instruction still
// reads 16-byte runs of a row.  Measured on the 1e6-node disk operator (3
// applications): 4 lanes per row 0.299 ms, 2 lanes 0.248 ms, one lane per
// row (uncoalesced row reads) 0.399 ms.
constexpr int RB = 1;

template <int NB, int G>
__device__ __forceinline__ void dot_batch(int64_t p, const int32_t *__restrict__ col, const double *__restrict__ val,
                                          const double *__restrict__ u, double &acc) {
    int c[NB];
    double v[NB], x[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        c[k] = __ldg(col + p + (int64_t)G * k);
        v[k] = __ldg(val + p + (int64_t)G * k);
    }
#pragma unroll
    for (int k = 0; k < NB; ++k) x[k] = __ldg(u + c[k]);
#pragma unroll
    for (int k = 0; k < NB; ++k) acc = fma(v[k], x[k], acc);
}

template <int G>
__device__ __forceinline__ void rows_dot(int64_t base, int64_t nrows, int sub, const int64_t *__restrict__ rp,
                                         const int32_t *__restrict__ col, const double *__restrict__ val,
                                         const double *__restrict__ u, double (&acc)[RB]) {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        acc[r] = 0.0;
        if (base + r >= nrows) continue;
        const int64_t b = __ldg(rp + base + r), e = __ldg(rp + base + r + 1);
        int64_t p = b + sub;
        int64_t cnt = e > p ? (e - p + G - 1) / G : 0;
        for (; cnt >= 8; cnt -= 8, p += 8 * G) dot_batch<8, G>(p, col, val, u, acc[r]);
        if (cnt >= 4) { dot_batch<4, G>(p, col, val, u, acc[r]); cnt -= 4; p += 4 * G; }
        if (cnt >= 2) { dot_batch<2, G>(p, col, val, u, acc[r]); cnt -= 2; p += 2 * G; }
        if (cnt >= 1) dot_batch<1, G>(p, col, val, u, acc[r]);
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
                y[row] = beta == 0.0 ? (alpha == 1.0 ? acc[r] : alpha * acc[r]) : fma(alpha, acc[r], beta * y[row]);
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
    return avg >= 96 ? 4 : 2;
}

// one wave at the kernel's occupancy (blocks of 256 threads), fewer for small matrices
int grid_for(mm_ctx *ctx, int64_t nrows, int G, const void *kernel) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t need = ((nrows + RB - 1) / RB * G + 255) / 256;
    int64_t cap = (int64_t)ctx->num_sms * per_sm;
    return (int)std::max<int64_t>(1, std::min(need, cap));
}

}  // namespace

int spmv_launch(mm_ctx *ctx, const mm_csr_pattern *p, const double *vals, const double *u,
                double alpha, double beta, double *y) {
    if (p->nrows == 0) return MM_OK;
    const int G = group_for(p);
    const int blocks = grid_for(ctx, p->nrows, G, G == 4 ? (const void *)k_spmv<4> : (const void *)k_spmv<2>);
    cudaStream_t st = ctx->stream;
    switch (G) {
        case 4: k_spmv<4><<<blocks, 256, 0, st>>>(p->nrows, p->d_row_ptr, p->d_col, vals, u, alpha, beta, y); break;
        default: k_spmv<2><<<blocks, 256, 0, st>>>(p->nrows, p->d_row_ptr, p->d_col, vals, u, alpha, beta, y); break;
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
    const int blocks = grid_for(ctx, p->nrows, G,
                                G == 4 ? (const void *)k_diffuse_step<4> : (const void *)k_diffuse_step<2>);
    cudaStream_t st = ctx->stream;
    double *src = u, *dst = work;
    for (int t = 0; t < steps; ++t) {
        switch (G) {
            case 4: k_diffuse_step<4><<<blocks, 256, 0, st>>>(p->nrows, p->d_row_ptr, p->d_col, vals, fixed, g, neumann, src, dt, dst); break;
            default: k_diffuse_step<2><<<blocks, 256, 0, st>>>(p->nrows, p->d_row_ptr, p->d_col, vals, fixed, g, neumann, src, dt, dst); break;
        }
        MM_LAUNCH_CHECK(ctx);
        double *t2 = src; src = dst; dst = t2;
    }
    if (src != u)
        MM_CUDA_CHECK(ctx, cudaMemcpyAsync(u, src, sizeof(double) * (size_t)p->nrows,
                                           cudaMemcpyDeviceToDevice, st));
    return MM_OK;
}
