// Generalized weighted least squares (GWLS) stencil weights, Section 2.2.1:
// with the monomials b of total degree <= m in xi = (x - x_c)/s, the weight
// matrix W = diag(omega(xi_i)), omega(x) = exp(-|x|^2 / sigma^2), and
// B_ij = b_j(xi_i), the weights of an operator L are w = W y where y is the
// minimum-norm solution of (W B)^T y = (L b)(0).  FP64 throughout: Householder
// QR of W B, R^T z = (L b)(0) by forward substitution, y = Q [z; 0], stored
// weights w / s^q.  Small systems run one stencil per thread (k_wls_thread),
// larger ones one stencil per warp with the rows on the lanes (k_wls).
#include "rbffd_dev.cuh"

namespace {

struct WlsParams {
    int dim, m, l, R, n_max, pitch;
    double inv_sigma2;          // 1 / sigma^2
    int scale;                  // MM_SCALE_FARTHEST or MM_SCALE_NEAREST
    int64_t N;
    const double *pts, *normals;
    const int64_t *row_ptr;
    const int32_t *col;
    int64_t row_begin, row_end;
    int opcode[5];
    double *vals[5];
    int32_t *status;
};

// Per-warp shared memory (doubles): W B [n_max x pitch] (the Householder
// vectors below the diagonal and R above it after the factorization), then
// omega [n_max], diag(R) [l], v^T v [l], z [l x R].
__host__ __device__ inline size_t wls_warp_doubles(int n_max, int pitch, int l, int R) {
    return (size_t)n_max * pitch + n_max + 2 * (size_t)l + (size_t)l * R;
}

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

template <int DIM, int RPL>
__device__ void wls_row(const WlsParams &P, int64_t row, double *base) {
    const int lane = threadIdx.x & 31, l = P.l, R = P.R, pitch = P.pitch, di = DIM - 2;
    double *WB = base;
    double *om = WB + (size_t)P.n_max * pitch;
    double *rdiag = om + P.n_max;
    double *vtv = rdiag + l;
    double *Z = vtv + l;
    const int64_t rb = P.row_ptr[row];
    const int64_t n64 = P.row_ptr[row + 1] - rb;
    int st = MM_ST_OK;
    const int n = (n64 >= 1 && n64 <= P.n_max) ? (int)n64 : 0;
    if (n == 0) st = MM_ST_BADARG;
    // offsets from the centre (FP64, registers) and the scale
    double d[RPL][DIM];
    double c[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) c[a] = P.pts[row * DIM + a];
    double dmax = 0.0, dmin = INFINITY;
    bool bad = false;
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        const int i = lane + 32 * q;
#pragma unroll
        for (int a = 0; a < DIM; ++a) d[q][a] = 0.0;
        if (i < n) {
            const int g = P.col[rb + i];
            if (g < 0 || g >= P.N || (i == 0 && g != row)) {
                bad = true;
            } else {
                double r2 = 0.0;
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    d[q][a] = P.pts[(int64_t)g * DIM + a] - c[a];
                    r2 = fma(d[q][a], d[q][a], r2);
                }
                const double r = sqrt(r2);
                dmax = fmax(dmax, r);
                if (i > 0) dmin = fmin(dmin, r);
            }
        }
    }
    bad = __any_sync(kFull, bad);
    dmax = warp_max(dmax);
    dmin = warp_min(dmin);
    const double s = P.scale == MM_SCALE_NEAREST ? dmin : dmax;
    if (bad || !(s > 0.0) || !(s < INFINITY)) st = MM_ST_BADARG;
    if (st == MM_ST_OK && n < l) st = MM_ST_SINGULAR;
    if (st != MM_ST_OK) {
        for (int cI = 0; cI < P.R; ++cI)
            for (int j = lane; j < n; j += 32) P.vals[cI][rb + j] = 0.0;
        if (P.status && lane == 0) P.status[row] = st;
        return;
    }
    const double inv_s = 1.0 / s;
    // W B, row by row on the lanes: b_0 = 1, b_j = b_parent(j) * xi_var(j)
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        const int i = lane + 32 * q;
        if (i < n) {
            double xi[DIM], r2 = 0.0;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                xi[a] = d[q][a] * inv_s;
                r2 = fma(xi[a], xi[a], r2);
            }
            const double w = exp(-r2 * P.inv_sigma2);
            om[i] = w;
            double *Wi = WB + (size_t)i * pitch;
            Wi[0] = 1.0;
            for (int b = 1; b < l; ++b) Wi[b] = Wi[c_mono.parent[di][b]] * xi[c_mono.var[di][b]];
            for (int b = 0; b < l; ++b) Wi[b] *= w;
        }
    }
    __syncwarp();
    // Householder QR: column k gets v (rows k..n-1, v_k on the diagonal),
    // R's off-diagonal part stays in rows < k, diag(R) and v^T v aside
    double rmax = 0.0;
    bool singular = false;
    for (int k = 0; k < l; ++k) {
        double a[RPL], tail = 0.0;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int i = lane + 32 * q;
            a[q] = (i >= k && i < n) ? WB[(size_t)i * pitch + k] : 0.0;
            if (i > k) tail = fma(a[q], a[q], tail);
        }
        tail = warp_sum(tail);
        const double akk = WB[(size_t)k * pitch + k];
        const double nrm = sqrt(fma(akk, akk, tail));
        const double alpha = akk >= 0.0 ? -nrm : nrm;
        const double vk = akk - alpha;
        const double vv = fma(vk, vk, tail);
        rmax = fmax(rmax, nrm);
        if (!(nrm > (double)max(n, l) * DBL_EPSILON * rmax)) singular = true;
        __syncwarp();
        if (lane == 0) {
            WB[(size_t)k * pitch + k] = vk;
            rdiag[k] = alpha;
            vtv[k] = vv;
        }
        double v[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int i = lane + 32 * q;
            v[q] = i == k ? vk : (i > k ? a[q] : 0.0);
        }
        const double f = vv > 0.0 ? 2.0 / vv : 0.0;
        for (int j = k + 1; j < l; ++j) {
            double dot = 0.0;
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const int i = lane + 32 * q;
                if (i >= k && i < n) dot = fma(v[q], WB[(size_t)i * pitch + j], dot);
            }
            dot = warp_sum(dot) * f;
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const int i = lane + 32 * q;
                if (i >= k && i < n) WB[(size_t)i * pitch + j] = fma(-dot, v[q], WB[(size_t)i * pitch + j]);
            }
        }
        __syncwarp();
    }
    if (singular) {
        for (int cI = 0; cI < P.R; ++cI)
            for (int j = lane; j < n; j += 32) P.vals[cI][rb + j] = 0.0;
        if (P.status && lane == 0) P.status[row] = MM_ST_SINGULAR;
        __syncwarp();
        return;
    }
    // R^T z = (L b)(0): one lane per operator, forward substitution
    if (lane < R) {
        const int op = P.opcode[lane];
        for (int k = 0; k < l; ++k) {
            double rhs;
            if (op == 0) rhs = (double)c_mono.lap[di][k];
            else if (op >= 5) rhs = (double)d2_of_monomial(di, k, op);
            else {
                const int a = c_mono.lin[di][k];
                rhs = a < 0 ? 0.0 : (op == 4 ? P.normals[row * DIM + a] : (a == op - 1 ? 1.0 : 0.0));
            }
            for (int i = 0; i < k; ++i) rhs = fma(-WB[(size_t)i * pitch + k], Z[i * R + lane], rhs);
            Z[k * R + lane] = rhs / rdiag[k];
        }
    }
    __syncwarp();
    // y = H_0 ... H_{l-1} [z; 0], all operators at once
    double y[RPL][5];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        const int i = lane + 32 * q;
#pragma unroll
        for (int cI = 0; cI < 5; ++cI) y[q][cI] = (i < l && cI < R) ? Z[i * R + cI] : 0.0;
    }
    for (int k = l - 1; k >= 0; --k) {
        double v[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int i = lane + 32 * q;
            v[q] = (i >= k && i < n) ? WB[(size_t)i * pitch + k] : 0.0;
        }
        const double f = vtv[k] > 0.0 ? 2.0 / vtv[k] : 0.0;
#pragma unroll
        for (int cI = 0; cI < 5; ++cI) {
            if (cI >= R) break;
            double dot = 0.0;
#pragma unroll
            for (int q = 0; q < RPL; ++q) dot = fma(v[q], y[q][cI], dot);
            dot = warp_sum(dot) * f;
#pragma unroll
            for (int q = 0; q < RPL; ++q) y[q][cI] = fma(-dot, v[q], y[q][cI]);
        }
    }
    // w = W y / s^q
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        const int i = lane + 32 * q;
        if (i < n)
#pragma unroll
            for (int cI = 0; cI < 5; ++cI) {
                if (cI >= R) break;
                const double sc = op_order(P.opcode[cI]) == 2 ? inv_s * inv_s : inv_s;
                P.vals[cI][rb + i] = om[i] * y[q][cI] * sc;
            }
    }
    if (P.status && lane == 0) P.status[row] = MM_ST_OK;
    __syncwarp();
}

// The same computation with one thread per stencil, for small systems: every
// lane does useful FP64 work (the warp form leaves lanes idle when n < 32 and
// spends FP64 adds on its reductions).  Per-thread arrays live in shared
// memory interleaved across the warp (element e of lane L at e * 32 + L), so
// the lanes' accesses fall in distinct banks.
__host__ __device__ inline int wls_thread_doubles(int n_max, int l, int dim) {
    return n_max * (l + dim + 2) + 3 * l;
}

template <int DIM>
__device__ void wls_row_thread(const WlsParams &P, int64_t row, double *base) {
    const int l = P.l, nm = P.n_max, di = DIM - 2;
    const int oD = nm * l, oOM = oD + nm * DIM, oRD = oOM + nm, oVV = oRD + l, oZ = oVV + l, oY = oZ + l;
    auto at = [&](int e) -> double & { return base[(size_t)e << 5]; };
    const int64_t rb = P.row_ptr[row];
    const int64_t n64 = P.row_ptr[row + 1] - rb;
    const int n = (n64 >= 1 && n64 <= nm) ? (int)n64 : 0;
    int st = n == 0 ? MM_ST_BADARG : MM_ST_OK;
    double c[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) c[a] = P.pts[row * DIM + a];
    double dmax = 0.0, dmin = INFINITY;
    for (int i = 0; i < n; ++i) {
        const int g = P.col[rb + i];
        if (g < 0 || g >= P.N || (i == 0 && g != row)) {
            st = MM_ST_BADARG;
            break;
        }
        double r2 = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const double d = P.pts[(int64_t)g * DIM + a] - c[a];
            at(oD + i * DIM + a) = d;
            r2 = fma(d, d, r2);
        }
        const double r = sqrt(r2);
        dmax = fmax(dmax, r);
        if (i > 0) dmin = fmin(dmin, r);
    }
    const double s = P.scale == MM_SCALE_NEAREST ? dmin : dmax;
    if (st == MM_ST_OK && (!(s > 0.0) || !(s < INFINITY))) st = MM_ST_BADARG;
    if (st == MM_ST_OK && n < l) st = MM_ST_SINGULAR;
    if (st == MM_ST_OK) {
        const double inv_s = 1.0 / s;
        for (int i = 0; i < n; ++i) {
            double xi[DIM], r2 = 0.0;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                xi[a] = at(oD + i * DIM + a) * inv_s;
                r2 = fma(xi[a], xi[a], r2);
            }
            const double w = exp(-r2 * P.inv_sigma2);
            at(oOM + i) = w;
            at(i * l) = 1.0;
            for (int b = 1; b < l; ++b) at(i * l + b) = at(i * l + c_mono.parent[di][b]) * xi[c_mono.var[di][b]];
            for (int b = 0; b < l; ++b) at(i * l + b) *= w;
        }
        // Householder QR (v below and on the diagonal, R above; diag(R), 2 / v^T v aside)
        double rmax = 0.0;
        for (int k = 0; k < l && st == MM_ST_OK; ++k) {
            const double akk = at(k * l + k);
            double tail = 0.0;
            for (int i = k + 1; i < n; ++i) tail = fma(at(i * l + k), at(i * l + k), tail);
            const double nrm = sqrt(fma(akk, akk, tail));
            const double alpha = akk >= 0.0 ? -nrm : nrm;
            const double vk = akk - alpha;
            const double vv = fma(vk, vk, tail);
            rmax = fmax(rmax, nrm);
            if (!(nrm > (double)max(n, l) * DBL_EPSILON * rmax)) st = MM_ST_SINGULAR;
            const double f = vv > 0.0 ? 2.0 / vv : 0.0;
            at(k * l + k) = vk;
            at(oRD + k) = alpha;
            at(oVV + k) = f;
            for (int j = k + 1; j < l; ++j) {
                double dot = 0.0;
                for (int i = k; i < n; ++i) dot = fma(at(i * l + k), at(i * l + j), dot);
                dot *= f;
                for (int i = k; i < n; ++i) at(i * l + j) = fma(-dot, at(i * l + k), at(i * l + j));
            }
        }
    }
    if (st != MM_ST_OK) {
        for (int cI = 0; cI < P.R; ++cI)
            for (int j = 0; j < n; ++j) P.vals[cI][rb + j] = 0.0;
        if (P.status) P.status[row] = st;
        return;
    }
    const double inv_s = 1.0 / s;
    for (int cI = 0; cI < P.R; ++cI) {
        const int op = P.opcode[cI];
        // R^T z = (L b)(0)
        for (int k = 0; k < l; ++k) {
            double rhs;
            if (op == 0) rhs = (double)c_mono.lap[di][k];
            else if (op >= 5) rhs = (double)d2_of_monomial(di, k, op);
            else {
                const int a = c_mono.lin[di][k];
                rhs = a < 0 ? 0.0 : (op == 4 ? P.normals[row * DIM + a] : (a == op - 1 ? 1.0 : 0.0));
            }
            for (int i = 0; i < k; ++i) rhs = fma(-at(i * l + k), at(oZ + i), rhs);
            at(oZ + k) = rhs / at(oRD + k);
        }
        // y = H_0 ... H_{l-1} [z; 0]
        for (int i = 0; i < n; ++i) at(oY + i) = i < l ? at(oZ + i) : 0.0;
        for (int k = l - 1; k >= 0; --k) {
            double dot = 0.0;
            for (int i = k; i < n; ++i) dot = fma(at(i * l + k), at(oY + i), dot);
            dot *= at(oVV + k);
            for (int i = k; i < n; ++i) at(oY + i) = fma(-dot, at(i * l + k), at(oY + i));
        }
        const double sc = op_order(op) == 2 ? inv_s * inv_s : inv_s;
        for (int i = 0; i < n; ++i) P.vals[cI][rb + i] = at(oOM + i) * at(oY + i) * sc;
    }
    if (P.status) P.status[row] = MM_ST_OK;
}

template <int DIM>
__global__ void __launch_bounds__(128) k_wls_thread(const __grid_constant__ WlsParams P) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double *base = smem + (size_t)wib * 32 * wls_thread_doubles(P.n_max, P.l, DIM) + lane;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t row = P.row_begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < P.row_end;
         row += stride)
        wls_row_thread<DIM>(P, row, base);
}

template <int DIM, int RPL>
__global__ void __launch_bounds__(128) k_wls(const __grid_constant__ WlsParams P) {
    extern __shared__ double smem[];
    const int wib = threadIdx.x >> 5;
    double *base = smem + (size_t)wib * wls_warp_doubles(P.n_max, P.pitch, P.l, P.R);
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = P.row_begin + gw; row < P.row_end; row += nw) wls_row<DIM, RPL>(P, row, base);
}

template <int DIM>
int wls_launch_thread(mm_ctx *ctx, const WlsParams &P) {
    const size_t bytes = (size_t)32 * wls_thread_doubles(P.n_max, P.l, DIM) * sizeof(double);
    auto kern = k_wls_thread<DIM>;
    const int wpb = mm_warps_per_block(ctx, (const void *)kern, bytes, 4);
    const size_t sm = bytes * wpb;
    MM_CUDA_CHECK(ctx, mm_set_smem(ctx, (const void *)kern, sm));
    const int64_t rows = P.row_end - P.row_begin;
    const int64_t per_block = (int64_t)wpb * 32;
    const int blocks = (int)std::min<int64_t>((rows + per_block - 1) / per_block, (int64_t)ctx->num_sms * 32);
    kern<<<max(blocks, 1), wpb * 32, sm, ctx->stream>>>(P);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

template <int DIM, int RPL>
int wls_launch_t(mm_ctx *ctx, const WlsParams &P) {
    const size_t bytes = wls_warp_doubles(P.n_max, P.pitch, P.l, P.R) * sizeof(double);
    auto kern = k_wls<DIM, RPL>;
    if (bytes > ctx->smem_optin) return mm_fail(ctx, MM_EUNSUPPORTED, "stencil too large for shared memory");
    const int wpb = mm_warps_per_block(ctx, (const void *)kern, bytes, 4);
    const size_t sm = bytes * wpb;
    MM_CUDA_CHECK(ctx, mm_set_smem(ctx, (const void *)kern, sm));
    const int64_t rows = P.row_end - P.row_begin;
    const int blocks = (int)std::min<int64_t>((rows + wpb - 1) / wpb, (int64_t)ctx->num_sms * 32);
    kern<<<max(blocks, 1), wpb * 32, sm, ctx->stream>>>(P);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

}  // namespace

// Uploads this translation unit's monomial table to the current device.
int wls_init_device(mm_ctx *ctx) {
    MonoTable t;
    mono_table_host(t);
    MM_CUDA_CHECK(ctx, cudaMemcpyToSymbol(c_mono, &t, sizeof(t)));
    return MM_OK;
}

// Systems whose per-thread arrays take at most this many doubles (the
// paper's example, 9 nodes and 6 monomials, takes 120) run one stencil per
// thread; larger ones one stencil per warp.
constexpr int kWlsThreadMax = 160;

// job: a validated weights job (k unused); more than 5 operators run as
// launches of at most 5 columns.
int wls_launch(mm_ctx *ctx, const WeightsJob &job, double sigma, int scale) {
    if (job.row_end <= job.row_begin) return MM_OK;
    unsigned rest = job.ops;
    while (rest) {
        WlsParams P{};
        P.dim = job.dim;
        P.m = job.m;
        P.l = mm_num_monomials(job.dim, job.m);
        P.n_max = job.n_max;
        P.pitch = P.l | 1;
        P.inv_sigma2 = 1.0 / (sigma * sigma);
        P.scale = scale;
        P.N = job.N;
        P.pts = job.pts;
        P.normals = job.normals;
        P.row_ptr = job.row_ptr;
        P.col = job.col;
        P.row_begin = job.row_begin;
        P.row_end = job.row_end;
        P.status = job.status;
        int R = 0;
        for (int b = 0; b < 11 && R < 5; ++b)
            if (rest & (1u << b)) {
                P.opcode[R] = b;
                P.vals[R] = job.vals[b];
                ++R;
                rest &= ~(1u << b);
            }
        P.R = R;
        const int rpl = (job.n_max + 31) / 32;
        int rc;
        if (wls_thread_doubles(P.n_max, P.l, P.dim) <= kWlsThreadMax)
            rc = job.dim == 2 ? wls_launch_thread<2>(ctx, P) : wls_launch_thread<3>(ctx, P);
        else if (job.dim == 2)
            rc = rpl == 1 ? wls_launch_t<2, 1>(ctx, P) : wls_launch_t<2, 2>(ctx, P);
        else
            rc = rpl == 1 ? wls_launch_t<3, 1>(ctx, P) : wls_launch_t<3, 2>(ctx, P);
        if (rc != MM_OK) return rc;
    }
    return MM_OK;
}
