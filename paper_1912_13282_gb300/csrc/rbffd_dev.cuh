// Device-side building blocks of the RBF-FD weights kernels (one warp per
// stencil): stencil loading and scaling, assembly of the augmented system of
// Section 2.2.2 (eq. rbf-system-aug), the FP64 partial-pivot LU, the FP32
// implicit-pivot LU and solves, and the per-row FP64 and FP32+refinement
// solvers.  Included by the per-class kernels (rbffd.cu) and the persistent
// batched kernel (batched.cu); each translation unit gets its own copy of the
// constant monomial table and uploads it at context creation.
#pragma once

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
    int pitch64;               // shared-memory row pitch of the FP64 kernel (elements)
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

// Assemble [K | B] (FP64) into shared memory, row pitch `pitch`.  The Q block
// starts at row/column `qoff` >= n; rows and columns n .. qoff-1 are padding
// (identity row and column, zero right-hand side), so a stencil of n nodes can
// sit in a system laid out for qoff nodes.  The right-hand sides occupy
// columns qoff + l .. qoff + l + R - 1.  Returns the warp-uniform max |K|
// over the A and Q blocks.
template <int DIM>
__device__ double assemble_fp64(const WParams &P, int64_t row, int n, const double *xi, double *K,
                                int pitch, int qoff) {
    const int lane = threadIdx.x & 31;
    const int l = P.l, M = qoff + l, k = P.k;
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
    // padding rows/columns n .. qoff-1: identity
    for (int e = lane; e < (qoff - n) * (M + P.R); e += 32) {
        int j = n + e / (M + P.R), c = e % (M + P.R);
        K[j * pitch + c] = (c == j) ? 1.0 : 0.0;
    }
    for (int e = lane; e < (qoff - n) * M; e += 32) {
        int j = n + e / M, r = e % M;
        if (r < n || r >= qoff) K[r * pitch + j] = 0.0;
    }
    // Q and Q^T: q_0 = 1, q_b = q_parent * xi_var
    for (int r = lane; r < n; r += 32) {
        double *Kr = K + r * pitch + qoff;
        Kr[0] = 1.0;
        K[qoff * pitch + r] = 1.0;
        for (int b = 1; b < l; ++b) {
            double v = Kr[c_mono.parent[di][b]] * xi[r * DIM + c_mono.var[di][b]];
            Kr[b] = v;
            K[(qoff + b) * pitch + r] = v;
            amax = fmax(amax, fabs(v));
        }
    }
    amax = fmax(amax, 1.0);
    for (int e = lane; e < l * l; e += 32) K[(qoff + e / l) * pitch + qoff + e % l] = 0.0;
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
            K[(qoff + b) * pitch + M + cI] = v;
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

// One stencil (row) with the FP64 solver; `base` is the warp's shared memory.
// from_fallback: the row was handed over by the mixed-precision solver.
template <int DIM>
__device__ __noinline__ void fp64_row(const WParams &P, int64_t row, double *base, bool from_fallback) {
    const int lane = threadIdx.x & 31;
    double *K = base;
    double *invp = K + (size_t)P.M_max * P.pitch64;
    double *mul = invp + P.M_max;
    double *xi = mul + P.M_max;
    int n;
    int64_t rb;
    double s;
    if (!load_stencil<DIM>(P, row, n, rb, xi, s)) {
        reject_row(P, row, rb, n, MM_ST_BADARG);
        __syncwarp();
        return;
    }
    const int M = n + P.l;
    const double amax = assemble_fp64<DIM>(P, row, n, xi, K, P.pitch64, n);
    if (!lu_solve_fp64(K, P.pitch64, M, P.R, amax, invp, mul)) {
        reject_row(P, row, rb, n, MM_ST_SINGULAR);
        __syncwarp();
        return;
    }
    store_weights(P, rb, n, s, K, P.pitch64, M);
    if (P.status && lane == 0) P.status[row] = from_fallback ? MM_ST_FALLBACK : MM_ST_OK;
    __syncwarp();
}

// ------------------------------------------------------------ mixed solver
// FP32 LU with implicit partial pivoting: rows are never exchanged; the row
// chosen at step kk is marked (step = kk) and copied to a per-warp buffer
// from which the remaining rows are updated.  Lane t owns rows t, t+32, t+64
// (RPL of them).  A32 [M x p32] (row-major, p32 odd) holds L below the pivots
// and U in the pivot rows; A32[perm[kk]][kk] holds 1/U_kk.
constexpr int kBig = 1 << 30;

template <int RPL>
__device__ bool lu32_implicit(float *A, int p32, int M, int *step, int *perm, float *ubuf,
                              float tiny) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    for (int kk = 0; kk < M; ++kk) {
        float best = -1.0f;
        int brow = kBig;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            if (step[q] == kBig) {
                const int r = lane + 32 * q;
                const float v = fabsf(A[r * p32 + kk]);
                if (v > best) { best = v; brow = r; }
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float ob = __shfl_xor_sync(kFull, best, o);
            const int orow = __shfl_xor_sync(kFull, brow, o);
            if (ob > best || (ob == best && orow < brow)) { best = ob; brow = orow; }
        }
        const bool good = best > tiny;
        ok &= good;
        if (brow == kBig) brow = 0;               // only when every row is exhausted (not reached)
        // pivot row from the even column c0 <= kk+1 on, zeros at columns <= kk, so
        // the updates below can run on column pairs
        const int c0 = (kk + 1) & ~1;
        const float *Up = A + brow * p32;
        for (int c = c0 + lane; c < p32; c += 32) ubuf[c] = (c > kk && c < M) ? Up[c] : 0.0f;
        const float piv = Up[kk];
        if (lane == 0) perm[kk] = brow;
        __syncwarp();
        const float ip = good ? 1.0f / piv : 0.0f;
        float l[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int r = lane + 32 * q;
            if (r == brow) { step[q] = kk; A[r * p32 + kk] = ip; }
            l[q] = 0.0f;
            if (step[q] == kBig) {
                l[q] = A[r * p32 + kk] * ip;
                A[r * p32 + kk] = l[q];
            }
        }
        __syncwarp();
        const float2 *u2 = reinterpret_cast<const float2 *>(ubuf);
        for (int c = c0; c < M; c += 2) {
            const float2 u = u2[c >> 1];
#pragma unroll
            for (int q = 0; q < RPL; ++q)
                if (step[q] == kBig) {
                    float2 *dst = reinterpret_cast<float2 *>(A + (lane + 32 * q) * p32 + c);
                    float2 a = *dst;
                    a.x = fmaf(-l[q], u.x, a.x);
                    a.y = fmaf(-l[q], u.y, a.y);
                    *dst = a;
                }
        }
        __syncwarp();
    }
    return ok;
}

// Solve K x = b for R right-hand sides with the factors above.  z holds b
// by row for the lane's own rows (consumed).  The solution x, by column, is
// written to X [M x R] (shared) and returned after a warp barrier.
template <int RPL, int R>
__device__ void lu32_solve(const float *A, int p32, int M, const int *step, const int *perm,
                           float (&z)[RPL][R], float *X) {
    const int lane = threadIdx.x & 31;
    for (int kk = 0; kk < M; ++kk) {
        const int p = perm[kk], owner = p & 31, qp = p >> 5;
        float y[R];
#pragma unroll
        for (int c = 0; c < R; ++c) {
            float v = z[0][c];
#pragma unroll
            for (int q = 1; q < RPL; ++q)
                if (qp == q) v = z[q][c];
            y[c] = __shfl_sync(kFull, v, owner);
        }
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            if (step[q] > kk) {
                const float a = A[(lane + 32 * q) * p32 + kk];
#pragma unroll
                for (int c = 0; c < R; ++c) z[q][c] = fmaf(-a, y[c], z[q][c]);
            }
    }
    for (int kk = M - 1; kk >= 0; --kk) {
        const int p = perm[kk], owner = p & 31, qp = p >> 5;
        const float ip = A[p * p32 + kk];
        float xk[R];
#pragma unroll
        for (int c = 0; c < R; ++c) {
            float v = z[0][c];
#pragma unroll
            for (int q = 1; q < RPL; ++q)
                if (qp == q) v = z[q][c];
            xk[c] = __shfl_sync(kFull, v, owner) * ip;
        }
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            if (step[q] >= 0 && step[q] < kk) {
                const float a = A[(lane + 32 * q) * p32 + kk];
#pragma unroll
                for (int c = 0; c < R; ++c) z[q][c] = fmaf(-a, xk[c], z[q][c]);
            }
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < R; ++c) X[kk * R + c] = xk[c];
    }
    __syncwarp();
}

// Per-warp shared memory of the mixed kernel (byte offsets, 16-aligned).
struct MixedLayout {
    int pA, p32;
    size_t a64, q64, b64, x64, xi, a32, u32, v32, perm, bytes;
};

__host__ __device__ inline MixedLayout mixed_layout(int n_max, int l, int R, int dim) {
    MixedLayout L{};
    const int M = n_max + l;
    L.pA = n_max | 1;
    L.p32 = ((M + 1) & ~1) | 2;        // 2 * odd: float2 rows, few column conflicts
    if (L.p32 < M) L.p32 += 4;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += (bytes + 15) & ~size_t(15);
        return at;
    };
    L.a64 = take((size_t)n_max * L.pA * 8);
    L.q64 = take((size_t)n_max * l * 8);
    L.b64 = take((size_t)M * R * 8);
    L.x64 = take((size_t)M * R * 8);
    L.xi = take((size_t)n_max * dim * 8);
    L.a32 = take((size_t)M * L.p32 * 4);
    L.u32 = take((size_t)L.p32 * 4);
    L.v32 = take((size_t)M * (R + 1) * 4);
    L.perm = take((size_t)M * 4);
    L.bytes = o;
    return L;
}

// Compact FP64 system for the residuals: A64 [n x pA] (diagonal 0), Q64
// [n x l], B64 [M x R] (rows < n: l_phi, rows n + b: l_q).  Returns max |K|.
template <int DIM>
__device__ double assemble_mixed(const WParams &P, int64_t row, int n, const double *xi,
                                 double *A64, int pA, double *Q64, double *B64, int R) {
    const int lane = threadIdx.x & 31;
    const int l = P.l, k = P.k, di = DIM - 2;
    double amax = 0.0;
    for (int d = 1; d <= n / 2; ++d) {
        const int cnt = (2 * d == n) ? n / 2 : n;
        for (int r = lane; r < cnt; r += 32) {
            int c = r + d;
            if (c >= n) c -= n;
            double r2 = 0.0;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const double t = xi[r * DIM + a] - xi[c * DIM + a];
                r2 = fma(t, t, r2);
            }
            const double v = phs(r2, k);
            A64[r * pA + c] = v;
            A64[c * pA + r] = v;
            amax = fmax(amax, v);
        }
    }
    for (int r = lane; r < n; r += 32) {
        A64[r * pA + r] = 0.0;
        double *Qr = Q64 + r * l;
        Qr[0] = 1.0;
        for (int b = 1; b < l; ++b) {
            const double v = Qr[c_mono.parent[di][b]] * xi[r * DIM + c_mono.var[di][b]];
            Qr[b] = v;
            amax = fmax(amax, fabs(v));
        }
        double r2 = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) r2 = fma(xi[r * DIM + a], xi[r * DIM + a], r2);
        double rk2 = sqrt(r2);
        for (int i = 3; i < k; i += 2) rk2 *= r2;
        for (int cI = 0; cI < R; ++cI) {
            const int op = P.opcode[cI];
            double v;
            if (cI >= P.R) {
                v = 0.0;                  // unused solver column
            } else if (op == 0) {
                v = (double)(k * (k + DIM - 2)) * rk2;
            } else {
                double dot;
                if (op == 4) {
                    dot = 0.0;
#pragma unroll
                    for (int a = 0; a < DIM; ++a) dot = fma(P.normals[row * DIM + a], xi[r * DIM + a], dot);
                } else {
                    dot = xi[r * DIM + (op - 1)];
                }
                v = -(double)k * rk2 * dot;
            }
            B64[r * R + cI] = v;
        }
    }
    for (int b = lane; b < l; b += 32) {
        for (int cI = 0; cI < R; ++cI) {
            const int op = P.opcode[cI];
            double v = 0.0;
            if (cI >= P.R) {
                v = 0.0;
            } else if (op == 0) {
                v = (double)c_mono.lap[di][b];
            } else {
                const int a = c_mono.lin[di][b];
                if (a >= 0) v = op == 4 ? P.normals[row * DIM + a] : ((a == op - 1) ? 1.0 : 0.0);
            }
            B64[(n + b) * R + cI] = v;
        }
    }
    __syncwarp();
    return warp_max(fmax(amax, 1.0));
}

// One stencil (row) with the FP32 + FP64-refinement solver; `base` is the
// warp's shared memory.  Returns true if the row must go to the FP64 solver
// (its status is then MM_ST_NONCONVERGED and its weights are not written).
template <int DIM, int RPL, int R>
__device__ __noinline__ bool mixed_row(const WParams &P, int64_t row, char *base) {
    const int lane = threadIdx.x & 31;
    const MixedLayout Ly = mixed_layout(P.n_max, P.l, R, DIM);
    double *A64 = (double *)(base + Ly.a64);
    double *Q64 = (double *)(base + Ly.q64);
    double *B64 = (double *)(base + Ly.b64);
    double *X64 = (double *)(base + Ly.x64);
    double *xi = (double *)(base + Ly.xi);
    float *A32 = (float *)(base + Ly.a32);
    float *U32 = (float *)(base + Ly.u32);
    float *V32 = (float *)(base + Ly.v32);
    int *perm = (int *)(base + Ly.perm);
    const int pA = Ly.pA, p32 = Ly.p32, l = P.l;
    const float u32 = FLT_EPSILON * 0.5f;
    {
        int n;
        int64_t rb;
        double s;
        if (!load_stencil<DIM>(P, row, n, rb, xi, s)) {
            reject_row(P, row, rb, n, MM_ST_BADARG);
            __syncwarp();
            return false;
        }
        const int M = n + l;
        const double amax = assemble_mixed<DIM>(P, row, n, xi, A64, pA, Q64, B64, R);
        // FP32 system: the A block as fl32 of the FP64 one, Q and Q^T from the
        // FP32 offsets (own rows; Q^T entries written by the row's owner)
        int step[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int r = lane + 32 * q;
            step[q] = r < M ? kBig : -1;
            if (r < n) {
                float *Ar = A32 + r * p32;
                for (int c = 0; c < n; ++c) Ar[c] = (float)A64[r * pA + c];
                float x32[DIM];
#pragma unroll
                for (int d = 0; d < DIM; ++d) x32[d] = (float)xi[r * DIM + d];
                float *Qr = Ar + n;
                Qr[0] = 1.0f;
                A32[n * p32 + r] = 1.0f;
                for (int b = 1; b < l; ++b) {
                    const float v = Qr[c_mono.parent[DIM - 2][b]] * x32[c_mono.var[DIM - 2][b]];
                    Qr[b] = v;
                    A32[(n + b) * p32 + r] = v;
                }
            } else if (r < M) {
                for (int c = n; c < M; ++c) A32[r * p32 + c] = 0.0f;
            }
        }
        __syncwarp();
        float n1 = 0.0f;   // ||K||_1 = max row sum (symmetric)
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int r = lane + 32 * q;
            if (r < M) {
                float rs = 0.0f;
                for (int c = 0; c < M; ++c) rs += fabsf(A32[r * p32 + c]);
                n1 = fmaxf(n1, rs);
            }
        }
        n1 = warp_maxf(n1);
        bool queue = !lu32_implicit<RPL>(A32, p32, M, step, perm, U32, (float)M * u32 * (float)amax);
        bool conv = false;
        if (!queue) {
            // Refinement.  The first two solves carry one extra column: a step of
            // Hager's 1-norm estimator of K^-1 (y = K^-1 e/M, then z = K^-T sign(y),
            // est = max(||y||_1, ||z||_inf); K is symmetric), which gates the
            // stencil to the FP64 solve if est * ||K||_1 * u32 is too large.
            constexpr int RC = R + 1;
            float z[RPL][RC];
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const int r = lane + 32 * q;
#pragma unroll
                for (int c = 0; c < R; ++c) z[q][c] = r < M ? (float)B64[r * R + c] : 0.0f;
                z[q][R] = r < M ? 1.0f / M : 0.0f;
            }
            lu32_solve<RPL, RC>(A32, p32, M, step, perm, z, V32);
            float est = 0.0f;
            double dmax = 0.0;
            for (int i = lane; i < M; i += 32) {
                est += fabsf(V32[i * RC + R]);
#pragma unroll
                for (int c = 0; c < R; ++c) {
                    const double d = (double)V32[i * RC + c];
                    X64[i * R + c] = d;
                    dmax = fmax(dmax, fabs(d));
                }
            }
            est = warp_sumf(est);
            double dprev = warp_max(dmax);
            float sg[RPL];
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const int r = lane + 32 * q;
                sg[q] = r < M ? (V32[r * RC + R] >= 0.0f ? 1.0f : -1.0f) : 0.0f;
            }
            __syncwarp();
            for (int it = 1; it <= P.ir_max_steps; ++it) {
                // FP64 residual b - K64 x over the nonzero blocks
                for (int e = lane; e < M * R; e += 32) {
                    const int i = e / R, c = e - i * R;
                    double acc = B64[e];
                    if (i < n) {
                        const double *Ai = A64 + i * pA;
                        const double *Qi = Q64 + i * l;
                        for (int j = 0; j < n; ++j) acc = fma(-Ai[j], X64[j * R + c], acc);
                        for (int b = 0; b < l; ++b) acc = fma(-Qi[b], X64[(n + b) * R + c], acc);
                    } else {
                        const int b = i - n;
                        for (int j = 0; j < n; ++j) acc = fma(-Q64[j * l + b], X64[j * R + c], acc);
                    }
                    V32[e] = (float)acc;
                }
                __syncwarp();
                double dmx = 0.0, xmax = 0.0;
                if (it == 1) {
#pragma unroll
                    for (int q = 0; q < RPL; ++q) {
                        const int r = lane + 32 * q;
#pragma unroll
                        for (int c = 0; c < R; ++c) z[q][c] = r < M ? V32[r * R + c] : 0.0f;
                        z[q][R] = sg[q];
                    }
                    __syncwarp();
                    lu32_solve<RPL, RC>(A32, p32, M, step, perm, z, V32);
                    float zinf = 0.0f;
                    for (int i = lane; i < M; i += 32) {
                        zinf = fmaxf(zinf, fabsf(V32[i * RC + R]));
#pragma unroll
                        for (int c = 0; c < R; ++c) {
                            const double d = (double)V32[i * RC + c];
                            const double xn = X64[i * R + c] + d;
                            X64[i * R + c] = xn;
                            dmx = fmax(dmx, fabs(d));
                            if (i < n) xmax = fmax(xmax, fabs(xn));
                        }
                    }
                    zinf = warp_maxf(zinf);
                    const float kest = n1 * fmaxf(est, zinf);
                    if (!((double)kest * u32 <= P.kappa_max)) { queue = true; break; }
                } else {
                    float zr[RPL][R];
#pragma unroll
                    for (int q = 0; q < RPL; ++q) {
                        const int r = lane + 32 * q;
#pragma unroll
                        for (int c = 0; c < R; ++c) zr[q][c] = r < M ? V32[r * R + c] : 0.0f;
                    }
                    __syncwarp();
                    lu32_solve<RPL, R>(A32, p32, M, step, perm, zr, V32);
                    for (int e = lane; e < M * R; e += 32) {
                        const double d = (double)V32[e];
                        const double xn = X64[e] + d;
                        X64[e] = xn;
                        dmx = fmax(dmx, fabs(d));
                        if (e < n * R) xmax = fmax(xmax, fabs(xn));
                    }
                }
                dmx = warp_max(dmx);
                xmax = warp_max(xmax);
                // the observed contraction of the last step bounds the error left
                const double theta = dmx / fmax(dprev, 1e-300);
                if (theta < 0.5 && theta / (1.0 - theta) * dmx <= P.ir_tol * xmax) {
                    conv = true;
                    break;
                }
                dprev = dmx;
                __syncwarp();
            }
            if (conv) {
                // Constraint rows Q^T w = l_q: one more FP64 residual on those rows
                // only, corrected through the FP32 factors, so the monomials are
                // reproduced to FP64 rounding rather than to the refinement tolerance.
                __syncwarp();
                for (int e = lane; e < l * R; e += 32) {
                    const int b = e / R, c = e - b * R;
                    double acc = B64[(n + b) * R + c];
                    for (int j = 0; j < n; ++j) acc = fma(-Q64[j * l + b], X64[j * R + c], acc);
                    V32[e] = (float)acc;
                }
                __syncwarp();
                float zr[RPL][R];
#pragma unroll
                for (int q = 0; q < RPL; ++q) {
                    const int r = lane + 32 * q;
#pragma unroll
                    for (int c = 0; c < R; ++c) zr[q][c] = (r >= n && r < M) ? V32[(r - n) * R + c] : 0.0f;
                }
                __syncwarp();
                lu32_solve<RPL, R>(A32, p32, M, step, perm, zr, V32);
                for (int e = lane; e < n * R; e += 32) X64[e] += (double)V32[e];
                __syncwarp();
            }
        }
        if (!conv) {
            if (P.status && lane == 0) P.status[row] = MM_ST_NONCONVERGED;
            __syncwarp();
            return true;
        }
        store_weights(P, rb, n, s, X64, R, 0);
        if (P.status && lane == 0) P.status[row] = MM_ST_OK;
        __syncwarp();
    }
    return false;
}


// Host: kernel parameters of one stencil class from a validated job.
inline WParams wparams_from_job(const mm_ctx *ctx, const WeightsJob &job) {
    WParams P{};
    P.dim = job.dim;
    P.k = job.k;
    P.m = job.m;
    P.l = mm_num_monomials(job.dim, job.m);
    P.n_max = job.n_max;
    P.M_max = job.n_max + P.l;
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
    P.ir_tol = ctx->ir_tol;
    P.ir_max_steps = ctx->ir_max_steps;
    P.kappa_max = ctx->kappa_max;
    return P;
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
