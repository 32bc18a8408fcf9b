// RBF-FD stencil weights on the GPU: one warp per stencil.
//
// For every node (row) the warp assembles the scaled augmented system of
// Section 2.2.2 (eq. rbf-system-aug) of the paper,
//     [A Q; Q^T 0] [w; lambda] = [l_phi; l_q],
//     xi_j = (x_j - x_c)/s, s = max_j ||x_j - x_c||,
//     A_ij = ||xi_i - xi_j||^k,  Q_ib = q_b(xi_i) (monomials of degree <= m),
// with one right-hand side per requested operator, solves it and stores
// w / s^q (q = 2 for the Laplacian, 1 for first derivatives) into the CSR
// value array of each operator, coalesced across the stencil.
//
// Two solvers:
//  * k_weights_fp64: partial-pivot LU of the augmented matrix [K | B] in
//    shared memory (FP64), back substitution, unscaled store.
//  * k_weights_mixed: the same LU in FP32, a 1-norm condition estimate from
//    the FP32 factors (Hager's method as refined by Higham), then iterative
//    refinement whose residuals b - K x are formed in FP64 from an FP64 copy
//    of K.  Stencils whose estimate says FP32 cannot converge, or whose
//    refinement does not converge, are queued for the FP64 kernel.
#include <float.h>
#include <math.h>

#include <algorithm>

#include "mm_internal.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxMono = 84;   // C(6 + 3, 3): monomials of degree <= 6 in 3D
constexpr int kMaxM = 96;      // largest augmented system handled

// Monomials of degree <= 6 in graded order (degree ascending; inside a degree
// the exponent of x descending, then y).  Each non-constant monomial is its
// parent times one variable: q_b = q_parent[b] * xi_var[b].  A table for
// degree <= m is the first C(m + d, d) entries.
struct MonoTable {
    signed char parent[2][kMaxMono];
    signed char var[2][kMaxMono];
    signed char lap[2][kMaxMono];   // Laplacian of q_b at 0 (0 or 2)
    signed char lin[2][kMaxMono];   // a if q_b = xi_a, else -1
};
__constant__ MonoTable c_mono;

struct WParams {
    int dim, k, m, l, R;
    int n_max, M_max;
    int pitch64, pitch32;      // shared-memory row pitches (elements)
    int64_t N;
    const double *pts, *normals;
    const int64_t *row_ptr;
    const int32_t *col;
    int64_t row_begin, row_end;
    double *vals[5];           // per right-hand-side column
    int opcode[5];             // operator bit index per column (0 LAP, 1..3 d/dx_a, 4 d/dn)
    int32_t *status;
    // mixed-path controls
    int *fb_list;              // rows queued for the FP64 solve
    int *fb_count;
    double ir_tol;
    int ir_max_steps;
    double kappa_max;
    // indirect mode (FP64 fallback): rows come from list[0..*count)
    const int *list;
    const int *list_count;
};

__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ float warp_maxf(float v) {
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Warp argmax of (value, row): larger value wins, the smaller row on ties.
__device__ __forceinline__ void warp_argmax(double &v, int &r) {
    for (int o = 16; o; o >>= 1) {
        double ov = __shfl_xor_sync(kFull, v, o);
        int orow = __shfl_xor_sync(kFull, r, o);
        if (ov > v || (ov == v && orow < r)) { v = ov; r = orow; }
    }
}

// r^k for odd k from r^2: (r^2)^((k-1)/2) * r.
__device__ __forceinline__ double phs(double r2, int k) {
    double r = sqrt(r2);
    double p = r;
    for (int i = 1; i < k; i += 2) p *= r2;
    return p;
}

// Per-row prologue: validates the stencil, loads and scales offsets into
// xi [n x DIM] (shared), returns n and s (0 if the row is bad).
template <int DIM>
__device__ bool load_stencil(const WParams &P, int64_t row, int &n, int64_t &rb, double *xi,
                             double &s) {
    const int lane = threadIdx.x & 31;
    rb = P.row_ptr[row];
    int64_t n64 = P.row_ptr[row + 1] - rb;
    bool bad = n64 < 1 || n64 > P.n_max;
    n = bad ? 0 : (int)n64;
    double c[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) c[a] = P.pts[row * DIM + a];
    double r2max = 0.0;
    for (int j = lane; j < n; j += 32) {
        int g = P.col[rb + j];
        if (g < 0 || g >= P.N || (j == 0 && g != row)) { bad = true; continue; }
        double r2 = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            double d = P.pts[(int64_t)g * DIM + a] - c[a];
            xi[j * DIM + a] = d;
            r2 = fma(d, d, r2);
        }
        r2max = fmax(r2max, r2);
    }
    bad = __any_sync(kFull, bad);
    r2max = warp_max(r2max);
    if (bad || !(r2max > 0.0)) { s = 0.0; return false; }
    s = sqrt(r2max);
    double inv = 1.0 / s;
    __syncwarp();
    for (int j = lane; j < n * DIM; j += 32) xi[j] *= inv;
    __syncwarp();
    return true;
}

// Zero the weights of a rejected row and record its status.
__device__ void reject_row(const WParams &P, int64_t row, int64_t rb, int n, int st) {
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < P.R; ++c)
        for (int j = lane; j < n; j += 32) P.vals[c][rb + j] = 0.0;
    if (P.status && lane == 0) P.status[row] = st;
}

// Assemble [K | B] (FP64) into shared memory, row pitch `pitch`.  Returns the
// warp-uniform max |K| over the A and Q blocks.
template <int DIM>
__device__ double assemble_fp64(const WParams &P, int64_t row, int n, const double *xi, double *K,
                                int pitch) {
    const int lane = threadIdx.x & 31;
    const int l = P.l, M = n + l, k = P.k;
    const int di = DIM - 2;
    double amax = 0.0;
    // A: unordered pairs (r, (r + d) mod n), d = 1 .. n/2, each once
    for (int d = 1; d <= n / 2; ++d) {
        int cnt = (2 * d == n) ? n / 2 : n;
        for (int r = lane; r < cnt; r += 32) {
            int c = r + d;
            if (c >= n) c -= n;
            double r2 = 0.0;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                double t = xi[r * DIM + a] - xi[c * DIM + a];
                r2 = fma(t, t, r2);
            }
            double v = phs(r2, k);
            K[r * pitch + c] = v;
            K[c * pitch + r] = v;
            amax = fmax(amax, v);
        }
    }
    for (int r = lane; r < n; r += 32) K[r * pitch + r] = 0.0;
    // Q and Q^T: q_0 = 1, q_b = q_parent * xi_var
    for (int r = lane; r < n; r += 32) {
        double *Kr = K + r * pitch + n;
        Kr[0] = 1.0;
        K[n * pitch + r] = 1.0;
        for (int b = 1; b < l; ++b) {
            double v = Kr[c_mono.parent[di][b]] * xi[r * DIM + c_mono.var[di][b]];
            Kr[b] = v;
            K[(n + b) * pitch + r] = v;
            amax = fmax(amax, fabs(v));
        }
    }
    amax = fmax(amax, 1.0);
    for (int e = lane; e < l * l; e += 32) K[(n + e / l) * pitch + n + e % l] = 0.0;
    // right-hand sides in columns M .. M+R-1
    for (int j = lane; j < n; j += 32) {
        double r2 = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) r2 = fma(xi[j * DIM + a], xi[j * DIM + a], r2);
        // r^(k-2) (odd k >= 3): r * (r^2)^((k-3)/2)
        double rk2 = sqrt(r2);
        for (int i = 3; i < k; i += 2) rk2 *= r2;
        for (int cI = 0; cI < P.R; ++cI) {
            int op = P.opcode[cI];
            double v;
            if (op == 0) {
                v = (double)(k * (k + DIM - 2)) * rk2;
            } else {
                double dot;
                if (op == 4) {
                    dot = 0.0;
#pragma unroll
                    for (int a = 0; a < DIM; ++a) dot = fma(P.normals[row * DIM + a], xi[j * DIM + a], dot);
                } else {
                    dot = xi[j * DIM + (op - 1)];
                }
                v = -(double)k * rk2 * dot;
            }
            K[j * pitch + M + cI] = v;
        }
    }
    for (int b = lane; b < l; b += 32) {
        for (int cI = 0; cI < P.R; ++cI) {
            int op = P.opcode[cI];
            double v = 0.0;
            if (op == 0) {
                v = (double)c_mono.lap[di][b];
            } else {
                int a = c_mono.lin[di][b];
                if (a >= 0) {
                    if (op == 4) v = P.normals[row * DIM + a];
                    else v = (a == op - 1) ? 1.0 : 0.0;
                }
            }
            K[(n + b) * pitch + M + cI] = v;
        }
    }
    __syncwarp();
    return warp_max(amax);
}

// Unscaled store of the first n rows of columns M..M+R-1 of X (pitch xp).
template <class T>
__device__ void store_weights(const WParams &P, int64_t rb, int n, double s, const T *X, int xp,
                              int col0) {
    const int lane = threadIdx.x & 31;
    double inv_s = 1.0 / s;
    for (int cI = 0; cI < P.R; ++cI) {
        double sc = P.opcode[cI] == 0 ? inv_s * inv_s : inv_s;
        double *out = P.vals[cI] + rb;
        for (int j = lane; j < n; j += 32) out[j] = (double)X[j * xp + col0 + cI] * sc;
    }
}

// ------------------------------------------------------------ FP64 solver
// Gaussian elimination with row partial pivoting on [K | B] (M rows, M+R
// columns), then back substitution; solution overwrites columns M..M+R-1.
// Returns false if a pivot is not larger than M * u * amax.
__device__ bool lu_solve_fp64(double *K, int pitch, int M, int R, double amax, double *invp,
                              double *mul) {
    const int lane = threadIdx.x & 31;
    const double tiny = (double)M * (DBL_EPSILON * 0.5) * amax;
    const int W_all = M + R;
    for (int kk = 0; kk < M; ++kk) {
        double best = -1.0;
        int prow = M;
        for (int r = kk + lane; r < M; r += 32) {
            double v = fabs(K[r * pitch + kk]);
            if (v > best) { best = v; prow = r; }
        }
        warp_argmax(best, prow);
        if (!(best > tiny)) return false;
        if (prow != kk) {
            for (int c = kk + lane; c < W_all; c += 32) {
                double t = K[kk * pitch + c];
                K[kk * pitch + c] = K[prow * pitch + c];
                K[prow * pitch + c] = t;
            }
            __syncwarp();
        }
        double ip = 1.0 / K[kk * pitch + kk];
        if (lane == 0) invp[kk] = ip;
        for (int r = kk + 1 + lane; r < M; r += 32) mul[r] = K[r * pitch + kk] * ip;
        __syncwarp();
        const int W = W_all - kk - 1, H = M - kk - 1;
        if (H > 0) {
            const int q32 = 32 / W, r32 = 32 % W;
            int r = lane / W, c = lane % W;
            const double *Uk = K + kk * pitch + kk + 1;
            for (; r < H;) {
                double *dst = K + (kk + 1 + r) * pitch + kk + 1 + c;
                *dst = fma(-mul[kk + 1 + r], Uk[c], *dst);
                c += r32;
                r += q32;
                if (c >= W) { c -= W; ++r; }
            }
        }
        __syncwarp();
    }
    // back substitution, R columns at once
    for (int kk = M - 1; kk >= 0; --kk) {
        if (lane < R) K[kk * pitch + M + lane] *= invp[kk];
        __syncwarp();
        for (int e = lane; e < kk * R; e += 32) {
            int r = e / R, c = e - r * R;
            K[r * pitch + M + c] = fma(-K[r * pitch + kk], K[kk * pitch + M + c], K[r * pitch + M + c]);
        }
        __syncwarp();
    }
    return true;
}

// Per-warp shared-memory layout of the FP64 kernel (in doubles).
__host__ __device__ inline size_t fp64_warp_doubles(int M_max, int pitch64, int n_max, int dim) {
    return (size_t)M_max * pitch64 + 2 * (size_t)M_max + (size_t)n_max * dim + 2;
}

template <int DIM>
__global__ void __launch_bounds__(128) k_weights_fp64(WParams P) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double *base = smem + (size_t)wib * fp64_warp_doubles(P.M_max, P.pitch64, P.n_max, DIM);
    double *K = base;
    double *invp = K + (size_t)P.M_max * P.pitch64;
    double *mul = invp + P.M_max;
    double *xi = mul + P.M_max;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t count = P.list ? (int64_t)*P.list_count : P.row_end - P.row_begin;
    for (int64_t t = gw; t < count; t += nw) {
        const int64_t row = P.list ? (int64_t)P.list[t] : P.row_begin + t;
        int n;
        int64_t rb;
        double s;
        if (!load_stencil<DIM>(P, row, n, rb, xi, s)) {
            reject_row(P, row, rb, n, MM_ST_BADARG);
            continue;
        }
        const int M = n + P.l;
        double amax = assemble_fp64<DIM>(P, row, n, xi, K, P.pitch64);
        bool ok = lu_solve_fp64(K, P.pitch64, M, P.R, amax, invp, mul);
        if (!ok) {
            reject_row(P, row, rb, n, MM_ST_SINGULAR);
            __syncwarp();
            continue;
        }
        store_weights(P, rb, n, s, K, P.pitch64, M);
        if (P.status && lane == 0) P.status[row] = P.list ? MM_ST_FALLBACK : MM_ST_OK;
        __syncwarp();
    }
}

// ------------------------------------------------------------ mixed solver
// FP32 LU with row partial pivoting in place (L below the diagonal, unit
// diagonal implied; U on and above), perm[kk] = row swapped with kk,
// invU[kk] = 1/U_kk.  Returns false on a pivot <= M * u32 * amax.
__device__ bool lu_factor_fp32(float *A, int p, int M, float amax, int *perm, float *invU) {
    const int lane = threadIdx.x & 31;
    const float tiny = (float)M * (FLT_EPSILON * 0.5f) * amax;
    for (int kk = 0; kk < M; ++kk) {
        float best = -1.0f;
        int prow = M;
        for (int r = kk + lane; r < M; r += 32) {
            float v = fabsf(A[r * p + kk]);
            if (v > best) { best = v; prow = r; }
        }
        for (int o = 16; o; o >>= 1) {
            float ov = __shfl_xor_sync(kFull, best, o);
            int orow = __shfl_xor_sync(kFull, prow, o);
            if (ov > best || (ov == best && orow < prow)) { best = ov; prow = orow; }
        }
        if (!(best > tiny)) return false;
        if (lane == 0) perm[kk] = prow;
        if (prow != kk) {
            for (int c = lane; c < M; c += 32) {
                float t = A[kk * p + c];
                A[kk * p + c] = A[prow * p + c];
                A[prow * p + c] = t;
            }
            __syncwarp();
        }
        float ip = 1.0f / A[kk * p + kk];
        if (lane == 0) invU[kk] = ip;
        for (int r = kk + 1 + lane; r < M; r += 32) A[r * p + kk] *= ip;
        __syncwarp();
        const int W = M - kk - 1, H = W;
        if (H > 0) {
            const int q32 = 32 / W, r32 = 32 % W;
            int r = lane / W, c = lane % W;
            for (; r < H;) {
                float *dst = A + (kk + 1 + r) * p + kk + 1 + c;
                *dst = fmaf(-A[(kk + 1 + r) * p + kk], A[kk * p + kk + 1 + c], *dst);
                c += r32;
                r += q32;
                if (c >= W) { c -= W; ++r; }
            }
        }
        __syncwarp();
    }
    return true;
}

// Solve K y = b (trans = false) or K^T y = b (trans = true) in place for the
// R columns of y [M x R] (row-major, FP32) with the factors above.
__device__ void lu_solve_fp32(const float *A, int p, int M, const int *perm, const float *invU,
                              float *y, int R, bool trans) {
    const int lane = threadIdx.x & 31;
    if (!trans) {
        if (lane < R)
            for (int kk = 0; kk < M; ++kk) {
                int q = perm[kk];
                if (q != kk) { float t = y[kk * R + lane]; y[kk * R + lane] = y[q * R + lane]; y[q * R + lane] = t; }
            }
        __syncwarp();
        for (int kk = 0; kk < M - 1; ++kk) {             // L (unit lower)
            for (int e = lane; e < (M - kk - 1) * R; e += 32) {
                int r = kk + 1 + e / R, c = e % R;
                y[r * R + c] = fmaf(-A[r * p + kk], y[kk * R + c], y[r * R + c]);
            }
            __syncwarp();
        }
        for (int kk = M - 1; kk >= 0; --kk) {            // U
            if (lane < R) y[kk * R + lane] *= invU[kk];
            __syncwarp();
            for (int e = lane; e < kk * R; e += 32) {
                int r = e / R, c = e % R;
                y[r * R + c] = fmaf(-A[r * p + kk], y[kk * R + c], y[r * R + c]);
            }
            __syncwarp();
        }
    } else {
        for (int kk = 0; kk < M; ++kk) {                 // U^T (lower)
            if (lane < R) y[kk * R + lane] *= invU[kk];
            __syncwarp();
            for (int e = lane; e < (M - kk - 1) * R; e += 32) {
                int r = kk + 1 + e / R, c = e % R;
                y[r * R + c] = fmaf(-A[kk * p + r], y[kk * R + c], y[r * R + c]);
            }
            __syncwarp();
        }
        for (int kk = M - 1; kk > 0; --kk) {             // L^T (unit upper)
            for (int e = lane; e < kk * R; e += 32) {
                int r = e / R, c = e % R;
                y[r * R + c] = fmaf(-A[kk * p + r], y[kk * R + c], y[r * R + c]);
            }
            __syncwarp();
        }
        if (lane < R)
            for (int kk = M - 1; kk >= 0; --kk) {
                int q = perm[kk];
                if (q != kk) { float t = y[kk * R + lane]; y[kk * R + lane] = y[q * R + lane]; y[q * R + lane] = t; }
            }
        __syncwarp();
    }
}

// Estimate of ||K^-1||_1 from the FP32 factors: Hager's method with
// Higham's refinements (at most `iters` power steps, plus the alternating
// test vector).  v is an [M] scratch vector, w another.
__device__ float inv_norm1_est(const float *A, int p, int M, const int *perm, const float *invU,
                               float *v, int iters) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < M; i += 32) v[i] = 1.0f / M;
    __syncwarp();
    float est = 0.0f;
    int jlast = -1;
    for (int it = 0; it < iters; ++it) {
        lu_solve_fp32(A, p, M, perm, invU, v, 1, false);      // v = K^-1 x
        float s1 = 0.0f;
        for (int i = lane; i < M; i += 32) s1 += fabsf(v[i]);
        s1 = warp_sumf(s1);
        if (it > 0 && s1 <= est) break;
        est = s1;
        __syncwarp();
        for (int i = lane; i < M; i += 32) v[i] = v[i] >= 0.0f ? 1.0f : -1.0f;
        __syncwarp();
        lu_solve_fp32(A, p, M, perm, invU, v, 1, true);       // z = K^-T sign(v)
        float zmax = -1.0f, zx = 0.0f;
        int j = M;
        for (int i = lane; i < M; i += 32) {
            float a = fabsf(v[i]);
            if (a > zmax) { zmax = a; j = i; }
            zx += it == 0 ? v[i] / M : (i == jlast ? v[i] : 0.0f);   // z^T x
        }
        zx = warp_sumf(zx);
        for (int o = 16; o; o >>= 1) {
            float oz = __shfl_xor_sync(kFull, zmax, o);
            int oj = __shfl_xor_sync(kFull, j, o);
            if (oz > zmax || (oz == zmax && oj < j)) { zmax = oz; j = oj; }
        }
        if (zmax <= zx || j == jlast) break;   // no ascent direction left
        jlast = j;
        __syncwarp();
        for (int i = lane; i < M; i += 32) v[i] = (i == j) ? 1.0f : 0.0f;
        __syncwarp();
    }
    // alternating-sign vector, catches matrices where the power steps stall
    __syncwarp();
    for (int i = lane; i < M; i += 32)
        v[i] = ((i & 1) ? -1.0f : 1.0f) * (1.0f + (float)i / (float)max(M - 1, 1));
    __syncwarp();
    lu_solve_fp32(A, p, M, perm, invU, v, 1, false);
    float s2 = 0.0f;
    for (int i = lane; i < M; i += 32) s2 += fabsf(v[i]);
    s2 = warp_sumf(s2);
    __syncwarp();
    return fmaxf(est, 2.0f * s2 / (3.0f * M));
}

__host__ __device__ inline size_t mixed_warp_bytes(int M_max, int pitch64, int pitch32, int n_max,
                                                    int dim, int R) {
    size_t d = (size_t)M_max * pitch64 + (size_t)M_max * R + (size_t)n_max * dim;  // K64|b, x64, xi
    size_t f = (size_t)M_max * pitch32 + (size_t)M_max * R + 2 * (size_t)M_max;    // K32, y32, invU, v
    size_t i = (size_t)M_max;                                                       // perm
    // every warp's block starts with FP64 data: keep the stride 16-byte aligned
    return (d * 8 + f * 4 + i * 4 + 16 + 15) & ~size_t(15);
}

template <int DIM>
__global__ void __launch_bounds__(128) k_weights_mixed(WParams P) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int R = P.R;
    char *base = (char *)smem + (size_t)wib * mixed_warp_bytes(P.M_max, P.pitch64, P.pitch32,
                                                               P.n_max, DIM, R);
    double *K64 = (double *)base;                       // [M_max x pitch64], B in cols M..
    double *x64 = K64 + (size_t)P.M_max * P.pitch64;    // [M_max x R]
    double *xi = x64 + (size_t)P.M_max * R;             // [n_max x DIM]
    float *K32 = (float *)(xi + (size_t)P.n_max * DIM); // [M_max x pitch32]
    float *y32 = K32 + (size_t)P.M_max * P.pitch32;     // [M_max x R]
    float *invU = y32 + (size_t)P.M_max * R;
    float *v32 = invU + P.M_max;
    int *perm = (int *)(v32 + P.M_max);
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float u32 = FLT_EPSILON * 0.5f;
    for (int64_t row = P.row_begin + gw; row < P.row_end; row += nw) {
        int n;
        int64_t rb;
        double s;
        if (!load_stencil<DIM>(P, row, n, rb, xi, s)) {
            reject_row(P, row, rb, n, MM_ST_BADARG);
            continue;
        }
        const int M = n + P.l, p64 = P.pitch64, p32 = P.pitch32;
        double amax = assemble_fp64<DIM>(P, row, n, xi, K64, p64);
        // FP32 copy and its 1-norm
        float cmax = 0.0f;
        for (int c = lane; c < M; c += 32) {
            float cs = 0.0f;
            for (int r = 0; r < M; ++r) {
                float v = (float)K64[r * p64 + c];
                K32[r * p32 + c] = v;
                cs += fabsf(v);
            }
            cmax = fmaxf(cmax, cs);
        }
        float norm1 = warp_maxf(cmax);
        __syncwarp();
        bool queue = !lu_factor_fp32(K32, p32, M, (float)amax, perm, invU);
        if (!queue) {
            float kest = norm1 * inv_norm1_est(K32, p32, M, perm, invU, v32, 3);
            queue = !((double)kest * u32 <= P.kappa_max);
        }
        bool conv = false;
        if (!queue) {
            // x = 0, r = b; refine: y = K32^-1 r; x += y; r = b - K64 x (FP64)
            for (int e = lane; e < M * R; e += 32) {
                int r = e / R, c = e - r * R;
                x64[e] = 0.0;
                y32[e] = (float)K64[r * p64 + M + c];
            }
            __syncwarp();
            double dprev = 0.0;
            for (int step = 0; step <= P.ir_max_steps; ++step) {
                lu_solve_fp32(K32, p32, M, perm, invU, y32, R, false);
                double dmax = 0.0, xmax = 0.0;
                for (int e = lane; e < M * R; e += 32) {
                    double d = (double)y32[e];
                    double xn = x64[e] + d;
                    x64[e] = xn;
                    dmax = fmax(dmax, fabs(d));
                    if (e < n * R) xmax = fmax(xmax, fabs(xn));
                }
                dmax = warp_max(dmax);
                xmax = warp_max(xmax);
                if (step > 0) {
                    // observed contraction of the last step bounds the error left
                    double theta = dmax / fmax(dprev, 1e-300);
                    if (theta < 0.5 && theta / (1.0 - theta) * dmax <= P.ir_tol * xmax) {
                        conv = true;
                        break;
                    }
                }
                if (step == P.ir_max_steps) break;
                dprev = dmax;
                __syncwarp();
                // FP64 residual r = b - K64 x (skipping the zero block), rounded to FP32
                for (int e = lane; e < M * R; e += 32) {
                    int i = e / R, c = e - i * R;
                    const double *Ki = K64 + i * p64;
                    double acc = Ki[M + c];
                    int jend = i < n ? M : n;
                    for (int j = 0; j < jend; ++j) acc = fma(-Ki[j], x64[j * R + c], acc);
                    y32[e] = (float)acc;
                }
                __syncwarp();
            }
        }
        if (conv) {
            // Constraint rows: one more FP64 residual on Q^T w = l_q only (A rows
            // taken as satisfied), corrected through the FP32 factors, so the
            // monomials are reproduced to FP64 rounding rather than to the
            // refinement tolerance.
            for (int e = lane; e < M * R; e += 32) {
                int i = e / R, c = e - i * R;
                float rv = 0.0f;
                if (i >= n) {
                    const double *Ki = K64 + i * p64;
                    double acc = Ki[M + c];
                    for (int j = 0; j < n; ++j) acc = fma(-Ki[j], x64[j * R + c], acc);
                    rv = (float)acc;
                }
                y32[e] = rv;
            }
            __syncwarp();
            lu_solve_fp32(K32, p32, M, perm, invU, y32, R, false);
            for (int e = lane; e < M * R; e += 32) x64[e] += (double)y32[e];
            __syncwarp();
        }
        if (!conv) {
            if (lane == 0) {
                int slot = atomicAdd(P.fb_count, 1);
                P.fb_list[slot] = (int)row;
                if (P.status) P.status[row] = MM_ST_NONCONVERGED;
            }
            __syncwarp();
            continue;
        }
        store_weights(P, rb, n, s, x64, R, 0);
        if (P.status && lane == 0) P.status[row] = MM_ST_OK;
        __syncwarp();
    }
}

// ------------------------------------------------------------- host side
void mono_table_host(MonoTable &t) {
    for (int di = 0; di < 2; ++di) {
        const int dim = di + 2;
        int exps[kMaxMono][3];
        int cnt = 0;
        for (int deg = 0; deg <= 6; ++deg) {
            // exponents with sum deg, x descending, then y descending
            for (int ex = deg; ex >= 0; --ex) {
                if (dim == 2) {
                    exps[cnt][0] = ex; exps[cnt][1] = deg - ex; exps[cnt][2] = 0; ++cnt;
                } else {
                    for (int ey = deg - ex; ey >= 0; --ey) {
                        exps[cnt][0] = ex; exps[cnt][1] = ey; exps[cnt][2] = deg - ex - ey; ++cnt;
                    }
                }
            }
        }
        for (int b = 0; b < cnt; ++b) {
            int deg = exps[b][0] + exps[b][1] + exps[b][2];
            t.parent[di][b] = -1;
            t.var[di][b] = 0;
            if (b > 0) {
                int v = 0;
                while (exps[b][v] == 0) ++v;
                int pe[3] = {exps[b][0], exps[b][1], exps[b][2]};
                pe[v] -= 1;
                for (int q = 0; q < b; ++q)
                    if (exps[q][0] == pe[0] && exps[q][1] == pe[1] && exps[q][2] == pe[2]) {
                        t.parent[di][b] = (signed char)q;
                        break;
                    }
                t.var[di][b] = (signed char)v;
            }
            int twos = 0, ones = 0, which = -1;
            for (int a = 0; a < 3; ++a) {
                if (exps[b][a] == 2) ++twos;
                if (exps[b][a] == 1) { ++ones; which = a; }
            }
            t.lap[di][b] = (deg == 2 && twos == 1) ? 2 : 0;
            t.lin[di][b] = (deg == 1 && ones == 1) ? (signed char)which : -1;
        }
        for (int b = cnt; b < kMaxMono; ++b) {
            t.parent[di][b] = t.var[di][b] = t.lap[di][b] = 0;
            t.lin[di][b] = -1;
        }
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
    const int dim = job.dim;
    const int l = mm_num_monomials(dim, job.m);
    WParams P{};
    P.dim = dim;
    P.k = job.k;
    P.m = job.m;
    P.l = l;
    P.n_max = job.n_max;
    P.M_max = job.n_max + l;
    P.N = job.N;
    P.pts = job.pts;
    P.normals = job.normals;
    P.row_ptr = job.row_ptr;
    P.col = job.col;
    P.row_begin = job.row_begin;
    P.row_end = job.row_end;
    P.status = job.status;
    int R = 0;
    for (int b = 0; b < 5; ++b)
        if (job.ops & (1u << b)) {
            P.vals[R] = job.vals[b];
            P.opcode[R] = b;
            ++R;
        }
    P.R = R;
    P.pitch64 = (P.M_max + R) | 1;
    P.pitch32 = P.M_max | 1;
    P.ir_tol = ctx->ir_tol;
    P.ir_max_steps = ctx->ir_max_steps;
    P.kappa_max = ctx->kappa_max;
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
            MM_CUDA_CHECK(ctx, cudaFuncSetAttribute(k_weights_fp64<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_weights_fp64<2><<<blocks, wpb * 32, sm, st>>>(Q);
        } else {
            MM_CUDA_CHECK(ctx, cudaFuncSetAttribute(k_weights_fp64<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_weights_fp64<3><<<blocks, wpb * 32, sm, st>>>(Q);
        }
        MM_LAUNCH_CHECK(ctx);
        return MM_OK;
    };
    if (precision == MM_FP64) return launch_fp64(nullptr, nullptr, rows);

    // mixed: FP32 LU + FP64-residual refinement, queue stragglers for FP64
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
    const size_t wm = mixed_warp_bytes(P.M_max, P.pitch64, P.pitch32, P.n_max, dim, R);
    int wpb = warps_for(wm);
    size_t sm = wm * wpb;
    if (sm > ctx->smem_optin) return mm_fail(ctx, MM_EUNSUPPORTED, "stencil too large for shared memory");
    int blocks = (int)std::min<int64_t>((rows + wpb - 1) / wpb, (int64_t)ctx->num_sms * 32);
    if (dim == 2) {
        MM_CUDA_CHECK(ctx, cudaFuncSetAttribute(k_weights_mixed<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_weights_mixed<2><<<blocks, wpb * 32, sm, st>>>(P);
    } else {
        MM_CUDA_CHECK(ctx, cudaFuncSetAttribute(k_weights_mixed<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_weights_mixed<3><<<blocks, wpb * 32, sm, st>>>(P);
    }
    MM_LAUNCH_CHECK(ctx);
    return launch_fp64(P.fb_list, P.fb_count, rows);
}

int weights_launch(mm_ctx *ctx, const WeightsJob &job, int precision) {
    return weights_launch_scratch(ctx, job, precision, nullptr, nullptr);
}
