// Device-side building blocks of the RBF-FD weights kernels (one warp per
// stencil): stencil loading and scaling, assembly of the augmented system of
// Section 2.2.2 (eq. rbf-system-aug), the FP64 partial-pivot LU, the FP32
// Gauss-Jordan inverse (shared-memory and register forms) and its products,
// the per-row FP64 and FP32+refinement solvers.  Included by the per-class kernels (rbffd.cu) and the persistent
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
    signed char d2[2][kMaxMono];    // for degree-2 q_b = xi_a xi_c (a <= c): 3a + c, else -1
};

__constant__ MonoTable c_mono;

// second-derivative operator code (5..10) -> index pair (a, c), a <= c
__host__ __device__ inline int d2_a(int op) { return op == 5 || op == 6 || op == 8 ? 0 : (op == 7 || op == 9 ? 1 : 2); }
__host__ __device__ inline int d2_c(int op) { return op == 5 ? 0 : (op == 6 || op == 7 ? 1 : 2); }
// d2/dxi_a dxi_c of monomial b at 0: 2 for xi_a^2, 1 for xi_a xi_c (a != c), 0 otherwise
__device__ inline int d2_of_monomial(int di, int b, int op) {
    const int a = d2_a(op), c = d2_c(op);
    return c_mono.d2[di][b] == 3 * a + c ? (a == c ? 2 : 1) : 0;
}
// derivative order of an operator column (the weights unscale by s^-order)
__host__ __device__ inline int op_order(int op) { return op == 0 || op >= 5 ? 2 : 1; }
// d2/dx_a dx_c of ||x - xi_j||^k at the centre, from r^2 = ||xi_j||^2 and
// rk2 = r^(k-2): k r^(k-2) delta_ac + k (k-2) r^(k-4) xi_a xi_c (0 at r = 0)
__device__ inline double phs_d2(int op, int k, double r2, double rk2, const double *x) {
    const int a = d2_a(op), c = d2_c(op);
    double v = a == c ? (double)k * rk2 : 0.0;
    if (r2 > 0.0) v += (double)(k * (k - 2)) * (rk2 / r2) * x[a] * x[c];
    return v;
}

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
    int opcode[5];             // operator bit index per column (0 LAP, 1..3 d/dx_a, 4 d/dn,
                               // 5..10 d2/dx_a dx_b: xx, xy, yy, xz, yz, zz)
    int32_t *status;
    // mixed-path controls
    int *fb_list;              // rows queued for the FP64 solve
    int *fb_count;
    double ir_tol;
    int ir_max_steps;
    double kappa_max;
    int wide64;                // refinement residuals in native FP64 (else double-FP32)
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

// 1/d from an FP32 seed refined by one Halley step.  The seed is the FP32
// reciprocal of d's sign, exponent and leading 23 mantissa bits, moved
// between the formats by integer operations on the bit patterns (relative
// error below 2^-22, no FP64 instruction: GB300's FP64 pipe issues at ~1/64
// of the FP32 rate and charges a conversion like an FMA).  With e = 1 - d y,
// 1/d = y (1 + e + e^2 + ...), so y + y (e + e^2) leaves a relative error of
// ~e^3 < 2^-66 before its final rounding: three FP64 FMAs.  An exponent
// outside +-120 takes the IEEE division.
__device__ __forceinline__ double recip_nr(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int ex = (int)((b >> 52) & 0x7FFull) - 1023;
    if (ex < -120 || ex > 120) return 1.0 / d;
    const unsigned fb = ((unsigned)(b >> 32) & 0x80000000u) | ((unsigned)(ex + 127) << 23) |
                        (unsigned)((b >> 29) & 0x7FFFFFull);
    const unsigned yb = __float_as_uint(__frcp_rn(__uint_as_float(fb)));
    const int ey = (int)((yb >> 23) & 0xFFu) - 127;
    const double y = __longlong_as_double((long long)(((unsigned long long)(yb & 0x80000000u) << 32) |
                                                      ((unsigned long long)(ey + 1023) << 52) |
                                                      ((unsigned long long)(yb & 0x7FFFFFu) << 29)));
    const double e = fma(-d, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// |v| > tiny (tiny >= 0) on the bit patterns: integer compares instead of an
// FP64 one; NaN fails, as `!(fabs(v) > tiny)` would.
__device__ __forceinline__ bool abs_gt(double v, double tiny) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
    return a > (unsigned long long)__double_as_longlong(tiny) && a <= 0x7FF0000000000000ull;
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
    // the largest r^2 kept as the largest bit pattern (r^2 >= 0): integer
    // compares and shuffles instead of FP64 ones
    unsigned long long r2bits = 0ull;
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
        r2bits = max(r2bits, (unsigned long long)__double_as_longlong(r2));
    }
    bad = __any_sync(kFull, bad);
#pragma unroll
    for (int o = 16; o; o >>= 1) r2bits = max(r2bits, __shfl_xor_sync(kFull, r2bits, o));
    const double r2max = __longlong_as_double((long long)r2bits);
    if (bad || !(r2bits > 0ull && r2bits < 0x7FF0000000000000ull)) { s = 0.0; return false; }
    s = sqrt(r2max);
    const double inv = recip_nr(s);
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
    // max |K| kept as the largest bit pattern of the (non-negative) |values|:
    // integer compares instead of FP64 ones
    unsigned long long amax_bits = 0ull;
    // A: the n (n - 1) / 2 unordered pairs (r, (r + d) mod n), d = 1 .. n/2
    // (r < n/2 for d = n/2), numbered t = (d - 1) n + r and dealt to the
    // lanes in turn, so every lane has a pair in all but the last round
    const int npairs = n * (n - 1) / 2;
    int dd = 1 + lane / max(n, 1), rr = lane % max(n, 1);
    for (int t = lane; t < npairs; t += 32) {
        int c = rr + dd;
        if (c >= n) c -= n;
        double r2 = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            double tt = xi[rr * DIM + a] - xi[c * DIM + a];
            r2 = fma(tt, tt, r2);
        }
        double v = phs(r2, k);
        K[rr * pitch + c] = v;
        K[c * pitch + rr] = v;
        amax_bits = max(amax_bits, (unsigned long long)__double_as_longlong(v));
        rr += 32;
        while (rr >= n) {
            rr -= n;
            ++dd;
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
            amax_bits = max(amax_bits, (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull);
        }
    }
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
            } else if (op >= 5) {
                v = phs_d2(op, k, r2, rk2, xi + j * DIM);
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
            } else if (op >= 5) {
                v = (double)d2_of_monomial(di, b, op);
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
#pragma unroll
    for (int o = 16; o; o >>= 1) amax_bits = max(amax_bits, __shfl_xor_sync(kFull, amax_bits, o));
    return fmax(__longlong_as_double((long long)amax_bits), 1.0);
}

// Unscaled store of the first n rows of columns M..M+R-1 of X (pitch xp).
template <class T>
__device__ void store_weights(const WParams &P, int64_t rb, int n, double s, const T *X, int xp,
                              int col0) {
    const int lane = threadIdx.x & 31;
    const double inv_s = recip_nr(s);
    for (int cI = 0; cI < P.R; ++cI) {
        double sc = op_order(P.opcode[cI]) == 2 ? inv_s * inv_s : inv_s;
        double *out = P.vals[cI] + rb;
        for (int j = lane; j < n; j += 32) out[j] = (double)X[j * xp + col0 + cI] * sc;
    }
}

// ------------------------------------------------------------ FP64 solver
// Pivot key of an FP64 value in row r (< 128): the high word of |v| (sign,
// exponent, 20 mantissa bits) with its 7 lowest bits replaced by 127 - r, so
// the largest key is the largest |v| to 13 mantissa bits, the lowest row on
// ties.  Keys compare as integers: the search runs on the integer pipe and
// one redux.sync, not on the FP64 pipe (1/74 of the FP32 rate on GB300).
__device__ __forceinline__ unsigned pivot_key64(double v, int r) {
    const unsigned hi = (unsigned)((unsigned long long)__double_as_longlong(v) >> 32) & 0x7FFFFFFFu;
    return (hi & 0xFFFFFF80u) | (unsigned)(127 - r);
}

// Gaussian elimination with row partial pivoting on [K | B] (M rows, M+R
// columns), then back substitution; solution overwrites columns M..M+R-1.
// Each pivot row is scaled by 1/pivot as it is swapped into place (one pass
// over its W entries), so the elimination uses the rows' own column entries
// as multipliers and the back substitution needs no division or scaling:
// fewer partially filled FP64 warp instructions than a multiplier column
// and a per-row scaling of the solution.
// Returns false if a pivot is not larger than M * u * amax.
__device__ bool lu_solve_fp64(double *K, int pitch, int M, int R, double amax) {
    const int lane = threadIdx.x & 31;
    const double tiny = (double)M * (DBL_EPSILON * 0.5) * amax;
    const int W_all = M + R;
    for (int kk = 0; kk < M; ++kk) {
        unsigned key = 0;
        for (int r = kk + lane; r < M; r += 32) key = max(key, pivot_key64(K[r * pitch + kk], r));
        const int prow = 127 - (int)(__reduce_max_sync(kFull, key) & 0x7Fu);
        const double piv = K[prow * pitch + kk];
        if (!abs_gt(piv, tiny)) return false;
        const double ip = recip_nr(piv);
        // row kk <- row prow / pivot (columns kk+1 ..); row prow <- row kk
        // (its column kk is the multiplier the elimination reads)
        if (lane == 0 && prow != kk) K[prow * pitch + kk] = K[kk * pitch + kk];
        for (int c = kk + 1 + lane; c < W_all; c += 32) {
            const double a = K[prow * pitch + c];
            if (prow != kk) K[prow * pitch + c] = K[kk * pitch + c];
            K[kk * pitch + c] = a * ip;
        }
        __syncwarp();
        const int W = W_all - kk - 1, H = M - kk - 1;
        if (H > 0) {
            const int q32 = 32 / W, r32 = 32 % W;
            int r = lane / W, c = lane % W;
            const double *Uk = K + kk * pitch + kk + 1;
            for (; r < H;) {
                double *dst = K + (kk + 1 + r) * pitch + kk + 1 + c;
                *dst = fma(-K[(kk + 1 + r) * pitch + kk], Uk[c], *dst);
                c += r32;
                r += q32;
                if (c >= W) { c -= W; ++r; }
            }
        }
        __syncwarp();
    }
    // back substitution, R columns at once (unit diagonal)
    for (int kk = M - 1; kk >= 0; --kk) {
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
    return (size_t)M_max * pitch64 + (size_t)n_max * dim + 2;
}

// One stencil (row) with the FP64 solver; `base` is the warp's shared memory.
// from_fallback: the row was handed over by the mixed-precision solver.
template <int DIM>
__device__ __noinline__ void fp64_row(const WParams &P, int64_t row, double *base, bool from_fallback) {
    const int lane = threadIdx.x & 31;
    double *K = base;
    double *xi = K + (size_t)P.M_max * P.pitch64;
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
    if (!lu_solve_fp64(K, P.pitch64, M, P.R, amax)) {
        reject_row(P, row, rb, n, MM_ST_SINGULAR);
        __syncwarp();
        return;
    }
    store_weights(P, rb, n, s, K, P.pitch64, M);
    if (P.status && lane == 0) P.status[row] = from_fallback ? MM_ST_FALLBACK : MM_ST_OK;
    __syncwarp();
}

// ------------------------------------------------------------ mixed solver
// FP32 Gauss-Jordan inversion with implicit partial pivoting.  Rows are never
// exchanged: the row chosen at step kk is marked (step = kk, perm[kk] = row).
// Lane t owns rows t, t+32, ... (RPL of them).  S [M x p32] (row-major, p32 a
// multiple of 4 with p32/4 odd, so float4 accesses of 8 consecutive rows hit
// distinct banks) holds K on entry, with zeros in the padding columns
// M .. 4*ceil(M/4)-1.  In-place elimination of column kk from every other row
// leaves, in that column, the matching column of the inverse; at the end
//     (K^-1)[i][j] = S[perm[i]][step of row j].
// Columns are eliminated two at a time: the second pivot is chosen from
// column kk+1 as updated by the first step (one column only), then every
// other row takes both rank-1 updates in one pass over its entries.
// Returns false if a pivot is not larger than `tiny`.
constexpr int kBig = 1 << 30;

// d = a * b + c on two FP32 lanes at once (Blackwell packed FP32 FMA)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long *>(&a)), "l"(*reinterpret_cast<unsigned long long *>(&b)),
          "l"(*reinterpret_cast<unsigned long long *>(&c)));
    return *reinterpret_cast<float2 *>(&d);
}

// Warp-wide argmax of |v| over the lanes' candidate rows (row < 96): one
// redux of the key |v| (low 7 mantissa bits dropped) : (127 - row), so ties
// go to the lower row.  Returns the row (kBig if there is no candidate).
__device__ __forceinline__ int pivot_row(unsigned key) {
    const unsigned best = __reduce_max_sync(kFull, key);
    return best ? 127 - (int)(best & 0x7Fu) : kBig;
}
__device__ __forceinline__ unsigned pivot_key(float v, int r) {
    return (__float_as_uint(fabsf(v)) & 0xFFFFFF80u) | (unsigned)(127 - r);
}

template <int RPL>
__device__ __forceinline__ bool gj32_invert(float *__restrict__ S, int p32, int M, int *step, int *perm,
                            float *__restrict__ ubuf, float tiny) {
    const int lane = threadIdx.x & 31;
    const int C4 = (M + 3) >> 2, W4 = 4 * C4;
    float *__restrict__ ubuf2 = ubuf + W4;
    bool ok = true;
    int kk = 0;
    for (; kk + 1 < M; kk += 2) {
        // first pivot: column kk
        unsigned key = 0;
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            if (step[q] == kBig) key = max(key, pivot_key(S[(lane + 32 * q) * p32 + kk], lane + 32 * q));
        int p1 = pivot_row(key);
        if (p1 == kBig) p1 = 0;                    // only when every row is exhausted (not reached)
        const float piv1 = S[p1 * p32 + kk];
        const bool good1 = fabsf(piv1) > tiny;
        const float ip1 = good1 ? __frcp_rn(piv1) : 0.0f;
        const float u1n = S[p1 * p32 + kk + 1] * ip1;          // u1 at column kk+1
        // own rows: multiplier of step 1 and column kk+1 after step 1
        float m1[RPL], c1[RPL];
        unsigned key2 = 0;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int r = lane + 32 * q;
            m1[q] = 0.0f;
            c1[q] = 0.0f;
            if (r < M) {
                if (r == p1) {
                    step[q] = kk;
                    c1[q] = u1n;
                } else {
                    m1[q] = S[r * p32 + kk];
                    c1[q] = fmaf(-m1[q], u1n, S[r * p32 + kk + 1]);
                    if (step[q] == kBig) key2 = max(key2, pivot_key(c1[q], r));
                }
            }
        }
        // second pivot: column kk+1 after step 1
        int p2 = pivot_row(key2);
        if (p2 == kBig) p2 = p1 == 0 ? 1 : 0;      // not reached
        const float m1p2 = S[p2 * p32 + kk];
        const float piv2 = fmaf(-m1p2, u1n, S[p2 * p32 + kk + 1]);
        const bool good2 = fabsf(piv2) > tiny;
        ok &= good1 && good2;
        const float ip2 = good2 ? __frcp_rn(piv2) : 0.0f;
        const float u2k = -m1p2 * ip1 * ip2;                   // u2 at column kk
        const float m2p1 = u1n;                                // step-2 multiplier of row p1
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            if (lane + 32 * q == p2) step[q] = kk + 1;
        __syncwarp();
        // the two scaled pivot rows (0 at columns kk, kk+1) and rows p1, p2 themselves
        float *P1 = S + p1 * p32, *P2 = S + p2 * p32;
        for (int c = lane; c < W4; c += 32) {
            const float a1 = P1[c], a2 = P2[c];
            const float u1 = a1 * ip1;
            const float u2 = fmaf(-m1p2, u1, a2) * ip2;
            const bool piv_col = c == kk || c == kk + 1;
            ubuf[c] = piv_col ? 0.0f : u1;
            ubuf2[c] = piv_col ? 0.0f : u2;
            P2[c] = c == kk ? u2k : (c == kk + 1 ? ip2 : u2);
            P1[c] = c == kk ? fmaf(-m2p1, u2k, ip1) : (c == kk + 1 ? -m2p1 * ip2 : fmaf(-m2p1, u2, u1));
        }
        if (lane == 0) {
            perm[kk] = p1;
            perm[kk + 1] = p2;
        }
        __syncwarp();
        bool live[RPL];
        float2 n1[RPL], n2[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int r = lane + 32 * q;
            live[q] = r < M && r != p1 && r != p2;
            n1[q] = make_float2(-m1[q], -m1[q]);
            n2[q] = make_float2(-c1[q], -c1[q]);
        }
        const float4 *u4 = reinterpret_cast<const float4 *>(ubuf);
        const float4 *v4 = reinterpret_cast<const float4 *>(ubuf2);
#pragma unroll 2
        for (int c4 = 0; c4 < C4; ++c4) {
            const float4 u = u4[c4], v = v4[c4];
#pragma unroll
            for (int q = 0; q < RPL; ++q)
                if (live[q]) {
                    float4 *dst = reinterpret_cast<float4 *>(S + (lane + 32 * q) * p32) + c4;
                    const float4 a = *dst;
                    float2 lo = ffma2(n1[q], make_float2(u.x, u.y), make_float2(a.x, a.y));
                    float2 hi = ffma2(n1[q], make_float2(u.z, u.w), make_float2(a.z, a.w));
                    lo = ffma2(n2[q], make_float2(v.x, v.y), lo);
                    hi = ffma2(n2[q], make_float2(v.z, v.w), hi);
                    *dst = make_float4(lo.x, lo.y, hi.x, hi.y);
                }
        }
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            if (live[q]) {
                float *Sr = S + (lane + 32 * q) * p32;
                Sr[kk] = fmaf(-c1[q], u2k, -m1[q] * ip1);
                Sr[kk + 1] = -c1[q] * ip2;
            }
        __syncwarp();
    }
    if (kk < M) {
        // last column of an odd-sized system: one rank-1 step
        unsigned key = 0;
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            if (step[q] == kBig) key = max(key, pivot_key(S[(lane + 32 * q) * p32 + kk], lane + 32 * q));
        int p1 = pivot_row(key);
        if (p1 == kBig) p1 = 0;
        const float piv = S[p1 * p32 + kk];
        const bool good = fabsf(piv) > tiny;
        ok &= good;
        const float ip = good ? __frcp_rn(piv) : 0.0f;
        float2 mm[RPL];
        bool live[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int r = lane + 32 * q;
            live[q] = r < M && r != p1;
            const float m = live[q] ? S[r * p32 + kk] : 0.0f;
            mm[q] = make_float2(-m, -m);
            if (r == p1) step[q] = kk;
        }
        __syncwarp();
        float *Pr = S + p1 * p32;
        for (int c = lane; c < W4; c += 32) {
            const float v = Pr[c] * ip;
            ubuf[c] = c == kk ? 0.0f : v;
            Pr[c] = c == kk ? ip : v;
        }
        if (lane == 0) perm[kk] = p1;
        __syncwarp();
        const float4 *u4 = reinterpret_cast<const float4 *>(ubuf);
        for (int c4 = 0; c4 < C4; ++c4) {
            const float4 u = u4[c4];
#pragma unroll
            for (int q = 0; q < RPL; ++q)
                if (live[q]) {
                    float4 *dst = reinterpret_cast<float4 *>(S + (lane + 32 * q) * p32) + c4;
                    const float4 a = *dst;
                    const float2 lo = ffma2(mm[q], make_float2(u.x, u.y), make_float2(a.x, a.y));
                    const float2 hi = ffma2(mm[q], make_float2(u.z, u.w), make_float2(a.z, a.w));
                    *dst = make_float4(lo.x, lo.y, hi.x, hi.y);
                }
        }
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            if (live[q]) S[(lane + 32 * q) * p32 + kk] = mm[q].x * ip;
        __syncwarp();
    }
    return ok;
}

// The same elimination with the rows held in registers, for systems of
// 33..W unknowns (W = 40 or 48 = 4 ceil(M_max / 4)).  Lane L holds row L in
// full and one of PARTS = 32 / (W - 32) consecutive pieces (PC = W / PARTS
// columns) of row 32 + L / PARTS, so the second rows cost every lane PC
// columns instead of W.  Every pass shifts the rows left by the number of
// columns it eliminates and appends the new inverse columns at the right,
// so the pivot columns are always registers 0 and 1 and every register index
// is static; a piece's last columns come from the next piece by a shuffle.
// After M steps the inverse sits in columns W - M .. W - 1 in step order and
// is written back to S in the layout the shared-memory form leaves.  Only
// the pivot rows pass through shared memory (buf: 4 W floats, 16-byte
// aligned: the raw pivot rows, then the scaled ones).  Each entry sees the
// same operations in the same order as the shared-memory form, so the two
// give identical inverses.
template <int W>
__device__ __forceinline__ bool gj32_invert_reg(float *__restrict__ S, int p32, int M, int *step, int *perm,
                                                float *__restrict__ buf, float tiny, float &nK, float &nKinv) {
    static_assert(W == 40 || W == 48, "register width");
    constexpr int W2 = W / 2, WC4 = W / 4;
    constexpr int PARTS = 32 / (W - 32), PC = W / PARTS, PC2 = PC / 2;
    const int lane = threadIdx.x & 31;
    const int C4 = (M + 3) >> 2, W4 = 4 * C4;
    const int pt = lane % PARTS, r1 = 32 + lane / PARTS, c1base = pt * PC;
    const int lead = lane - pt;                // lane holding columns 0.. of row r1
    const bool last = pt == PARTS - 1;
    float *__restrict__ P1 = buf;
    float *__restrict__ P2 = buf + W;
    float *__restrict__ U = buf + 2 * W;
    float *__restrict__ V = buf + 3 * W;
    const float2 zero2 = make_float2(0.0f, 0.0f);
    float2 A0[W2];                             // row lane
    float2 A1[PC2];                            // columns c1base .. c1base + PC - 1 of row r1
    int st0 = step[0];
    int st1 = r1 < M ? kBig : -1;
    {
        const float4 *src = reinterpret_cast<const float4 *>(S + (lane < M ? lane : 0) * p32);
#pragma unroll
        for (int c4 = 0; c4 < WC4; ++c4) {
            float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (lane < M && c4 < C4) a = src[c4];
            A0[2 * c4] = make_float2(a.x, a.y);
            A0[2 * c4 + 1] = make_float2(a.z, a.w);
        }
        const float2 *src1 = reinterpret_cast<const float2 *>(S + (r1 < M ? r1 : 0) * p32 + c1base);
#pragma unroll
        for (int j = 0; j < PC2; ++j) A1[j] = (r1 < M && c1base + 2 * j < W4) ? src1[j] : zero2;
    }
    // the raw pivot row p to dst (W floats): one lane for p < 32, the PARTS
    // lanes of the row otherwise
    auto put_row = [&](int p, float *dst) {
        if (p < 32) {
            if (lane == p) {
                float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
                for (int c4 = 0; c4 < WC4; ++c4)
                    d4[c4] = make_float4(A0[2 * c4].x, A0[2 * c4].y, A0[2 * c4 + 1].x, A0[2 * c4 + 1].y);
            }
        } else if (r1 == p) {
            float2 *d2 = reinterpret_cast<float2 *>(dst + c1base);
#pragma unroll
            for (int j = 0; j < PC2; ++j) d2[j] = A1[j];
        }
    };
    auto lead_of = [](int p) { return p < 32 ? p : (p - 32) * PARTS; };
    // max over rows of the row sums of |entries| of the frame (columns past
    // the matrix hold zeros); row r1's pieces are added in column order, lane
    // to lane, so every sum is formed in the order of the shared-memory form
    auto rows_norm = [&]() {
        float rs0 = 0.0f;
#pragma unroll
        for (int j = 0; j < W2; ++j) {
            rs0 += fabsf(A0[j].x);
            rs0 += fabsf(A0[j].y);
        }
        float rs1 = 0.0f;
#pragma unroll
        for (int t = 0; t < PARTS; ++t) {
            const float in = __shfl_up_sync(kFull, rs1, 1);
            if (pt == t) {
                rs1 = t == 0 ? 0.0f : in;
#pragma unroll
                for (int j = 0; j < PC2; ++j) {
                    rs1 += fabsf(A1[j].x);
                    rs1 += fabsf(A1[j].y);
                }
            }
        }
        float v = lane < M ? rs0 : 0.0f;
        if (last && r1 < M) v = fmaxf(v, rs1);
        return warp_maxf(v);
    };
    nK = rows_norm();
    // The two pivots of the pass that eliminates the frame's columns 0 and 1
    // (the pivot rows' steps are recorded when that pass runs).  Each pass
    // chooses the next pass's pivots as soon as its own update has produced
    // the new columns 0 and 1, so the choice overlaps the rest of the update.
    struct Piv {
        int p1, p2;
        float ip1, ip2, u1n, m1p2, u2k, m10, c10, m11, c11;
        bool good;
    };
    auto choose = [&]() {
        Piv v;
        // first pivot: column 0
        unsigned key = 0;
        if (st0 == kBig) key = pivot_key(A0[0].x, lane);
        if (pt == 0 && st1 == kBig) key = max(key, pivot_key(A1[0].x, r1));
        int p1 = pivot_row(key);
        if (p1 == kBig) p1 = 0;                    // only when every row is exhausted (not reached)
        const float2 h1 = p1 < 32 ? A0[0] : A1[0];
        const float piv1 = __shfl_sync(kFull, h1.x, lead_of(p1));
        const float p1c1 = __shfl_sync(kFull, h1.y, lead_of(p1));
        const bool good1 = fabsf(piv1) > tiny;
        const float ip1 = good1 ? __frcp_rn(piv1) : 0.0f;
        const float u1n = p1c1 * ip1;              // u1 at column 1
        // multiplier of step 1 and column 1 after step 1 (row r1's from its lead lane)
        const float m10 = A0[0].x, c10 = fmaf(-m10, u1n, A0[0].y);
        float m11 = A1[0].x, c11 = fmaf(-m11, u1n, A1[0].y);
        m11 = __shfl_sync(kFull, m11, lead);
        c11 = __shfl_sync(kFull, c11, lead);
        // second pivot: column 1 after step 1, among the rows other than p1
        unsigned key2 = 0;
        if (lane != p1 && lane < M && st0 == kBig) key2 = pivot_key(c10, lane);
        if (r1 != p1 && pt == 0 && r1 < M && st1 == kBig) key2 = max(key2, pivot_key(c11, r1));
        int p2 = pivot_row(key2);
        if (p2 == kBig) p2 = p1 == 0 ? 1 : 0;      // not reached
        const float m1p2 = __shfl_sync(kFull, p2 < 32 ? m10 : m11, lead_of(p2));
        const float piv2 = __shfl_sync(kFull, p2 < 32 ? c10 : c11, lead_of(p2));
        const bool good2 = fabsf(piv2) > tiny;
        const float ip2 = good2 ? __frcp_rn(piv2) : 0.0f;
        v.p1 = p1;
        v.p2 = p2;
        v.ip1 = ip1;
        v.ip2 = ip2;
        v.u1n = u1n;
        v.m1p2 = m1p2;
        v.u2k = -m1p2 * ip1 * ip2;                 // u2 at column 0
        v.m10 = m10;
        v.c10 = c10;
        v.m11 = m11;
        v.c11 = c11;
        v.good = good1 && good2;
        return v;
    };
    bool ok = true;
    int kk = 0;
    Piv pv = choose();
    for (; kk + 1 < M; kk += 2) {
        const int p1 = pv.p1, p2 = pv.p2;
        const float ip1 = pv.ip1, ip2 = pv.ip2, u1n = pv.u1n, m1p2 = pv.m1p2, u2k = pv.u2k;
        const float m10 = pv.m10, c10 = pv.c10, m11 = pv.m11, c11 = pv.c11;
        ok &= pv.good;
        if (lane == p1) st0 = kk;
        if (r1 == p1) st1 = kk;
        if (lane == p2) st0 = kk + 1;
        if (r1 == p2) st1 = kk + 1;
        put_row(p1, P1);
        put_row(p2, P2);
        if (lane == 0) {
            perm[kk] = p1;
            perm[kk + 1] = p2;
        }
        __syncwarp();
        // the two scaled pivot rows in the shifted frame, with the new inverse
        // columns (u1: ip1, 0; u2: u2k, ip2) appended
        for (int c = lane; c < W; c += 32) {
            float u, v;
            if (c < W - 2) {
                const float a1 = P1[c + 2], a2 = P2[c + 2];
                u = a1 * ip1;
                v = fmaf(-m1p2, u, a2) * ip2;
            } else if (c == W - 2) {
                u = ip1;
                v = u2k;
            } else {
                u = 0.0f;
                v = ip2;
            }
            U[c] = u;
            V[c] = v;
        }
        // row <- a * row + b1 * u1 + b2 * u2, shifted by two: other rows take
        // both rank-1 updates (a = 1), row p1 becomes u1 - u1n u2, row p2 u2
        auto coef = [&](int r, float m, float c, float2 &al, float2 &b1, float2 &b2) {
            const bool live = r < M && r != p1 && r != p2;
            const float a = live ? 1.0f : 0.0f;
            const float x1 = live ? -m : (r == p1 ? 1.0f : 0.0f);
            const float x2 = live ? -c : (r == p1 ? -u1n : (r == p2 ? 1.0f : 0.0f));
            al = make_float2(a, a);
            b1 = make_float2(x1, x1);
            b2 = make_float2(x2, x2);
        };
        float2 al0, b10, b20, al1, b11, b21;
        coef(lane, m10, c10, al0, b10, b20);
        coef(r1, m11, c11, al1, b11, b21);
        // first columns of the next piece (zero past the end of the row)
        float2 nxt = make_float2(__shfl_down_sync(kFull, A1[0].x, 1), __shfl_down_sync(kFull, A1[0].y, 1));
        if (last) nxt = zero2;
        __syncwarp();
        const float4 *U4 = reinterpret_cast<const float4 *>(U);
        const float4 *V4 = reinterpret_cast<const float4 *>(V);
        const float2 *U2 = reinterpret_cast<const float2 *>(U + c1base);
        const float2 *V2 = reinterpret_cast<const float2 *>(V + c1base);
        auto update0 = [&](int c4) {
            const float4 u = U4[c4], v = V4[c4];
            const float2 o0 = A0[2 * c4 + 1];
            const float2 o1v = 2 * c4 + 2 < W2 ? A0[2 * c4 + 2] : zero2;
            float2 lo = ffma2(al0, o0, zero2);
            float2 hi = ffma2(al0, o1v, zero2);
            lo = ffma2(b10, make_float2(u.x, u.y), lo);
            hi = ffma2(b10, make_float2(u.z, u.w), hi);
            A0[2 * c4] = ffma2(b20, make_float2(v.x, v.y), lo);
            A0[2 * c4 + 1] = ffma2(b20, make_float2(v.z, v.w), hi);
        };
        auto update1 = [&](int j) {
            const float2 o = j + 1 < PC2 ? A1[j + 1] : nxt;
            const float2 t = ffma2(b11, U2[j], ffma2(al1, o, zero2));
            A1[j] = ffma2(b21, V2[j], t);
        };
        // the next frame's columns 0 and 1, then the next pass's pivots, then the rest
        update0(0);
        update1(0);
        pv = choose();
#pragma unroll
        for (int c4 = 1; c4 < WC4; ++c4) update0(c4);
#pragma unroll
        for (int j = 1; j < PC2; ++j) update1(j);
    }
    if (kk < M) {
        // last column of an odd-sized system: one rank-1 step, shift by one
        unsigned key = 0;
        if (st0 == kBig) key = pivot_key(A0[0].x, lane);
        if (pt == 0 && st1 == kBig) key = max(key, pivot_key(A1[0].x, r1));
        int p1 = pivot_row(key);
        if (p1 == kBig) p1 = 0;
        const float piv = __shfl_sync(kFull, p1 < 32 ? A0[0].x : A1[0].x, lead_of(p1));
        const bool good = fabsf(piv) > tiny;
        ok &= good;
        const float ip = good ? __frcp_rn(piv) : 0.0f;
        const float m0 = A0[0].x;
        const float m1 = __shfl_sync(kFull, A1[0].x, lead);
        auto coef1 = [&](int r, float m, float2 &al, float2 &bb) {
            const bool live = r < M && r != p1;
            const float a = live ? 1.0f : 0.0f;
            const float x = live ? -m : (r == p1 ? 1.0f : 0.0f);
            al = make_float2(a, a);
            bb = make_float2(x, x);
        };
        float2 al0, bb0, al1, bb1;
        coef1(lane, m0, al0, bb0);
        coef1(r1, m1, al1, bb1);
        if (lane == p1) st0 = kk;
        if (r1 == p1) st1 = kk;
        put_row(p1, P1);
        if (lane == 0) perm[kk] = p1;
        __syncwarp();
        for (int c = lane; c < W; c += 32) U[c] = c < W - 1 ? P1[c + 1] * ip : ip;
        float nx = __shfl_down_sync(kFull, A1[0].x, 1);
        if (last) nx = 0.0f;
        __syncwarp();
        const float4 *U4 = reinterpret_cast<const float4 *>(U);
#pragma unroll
        for (int c4 = 0; c4 < WC4; ++c4) {
            const float4 u = U4[c4];
            const float2 o0 = make_float2(A0[2 * c4].y, A0[2 * c4 + 1].x);
            const float2 o1v = make_float2(A0[2 * c4 + 1].y, 2 * c4 + 2 < W2 ? A0[2 * c4 + 2].x : 0.0f);
            A0[2 * c4] = ffma2(bb0, make_float2(u.x, u.y), ffma2(al0, o0, zero2));
            A0[2 * c4 + 1] = ffma2(bb0, make_float2(u.z, u.w), ffma2(al0, o1v, zero2));
        }
        const float2 *U2 = reinterpret_cast<const float2 *>(U + c1base);
#pragma unroll
        for (int j = 0; j < PC2; ++j) {
            const float2 o = make_float2(A1[j].y, j + 1 < PC2 ? A1[j + 1].x : nx);
            A1[j] = ffma2(bb1, U2[j], ffma2(al1, o, zero2));
        }
    }
    nKinv = rows_norm();
    // the inverse: columns W - M .. W - 1 of the registers -> columns 0 .. M-1 of S
    const int off = W - M;
    if (lane < M) {
        float *dst = S + lane * p32;
        if (off == 0) {
            float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
            for (int c4 = 0; c4 < WC4; ++c4)
                d4[c4] = make_float4(A0[2 * c4].x, A0[2 * c4].y, A0[2 * c4 + 1].x, A0[2 * c4 + 1].y);
        } else {
#pragma unroll
            for (int j = 0; j < W2; ++j) {
                if (2 * j >= off) dst[2 * j - off] = A0[j].x;
                if (2 * j + 1 >= off) dst[2 * j + 1 - off] = A0[j].y;
            }
        }
    }
    if (r1 < M) {
        float *dst = S + r1 * p32;
#pragma unroll
        for (int j = 0; j < PC2; ++j) {
            const int c = c1base + 2 * j - off;
            if (c >= 0) dst[c] = A1[j].x;
            if (c + 1 >= 0) dst[c + 1] = A1[j].y;
        }
    }
    // pivot steps in the row-per-lane layout of the apply (row 32 + lane)
    step[0] = st0;
    const int s1 = __shfl_sync(kFull, st1, (lane * PARTS) & 31);
    if (lane < W - 32) step[1] = s1;
    __syncwarp();
    return ok;
}

// x = K^-1 b for R right-hand sides with the inverse above.  V [M x R]
// (shared, natural row order) holds b on entry and x on exit; Bp [4*ceil(M/4)
// x R] (shared, 16-byte aligned) is scratch for b in pivot order.
template <int RPL, int R>
__device__ void gj32_apply(const float *S, int p32, int M, const int *step, const int *perm, float *V,
                           float *Bp) {
    const int lane = threadIdx.x & 31;
    const int C4 = (M + 3) >> 2;
    for (int e = lane; e < 4 * C4 * R; e += 32) {
        const int k = e / R, c = e - k * R;
        Bp[e] = k < M ? V[perm[k] * R + c] : 0.0f;
    }
    __syncwarp();
    float y[RPL][R];
#pragma unroll
    for (int q = 0; q < RPL; ++q)
#pragma unroll
        for (int c = 0; c < R; ++c) y[q][c] = 0.0f;
    const float4 *B4 = reinterpret_cast<const float4 *>(Bp);
    for (int c4 = 0; c4 < C4; ++c4) {
        float b[4 * R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const float4 v = B4[c4 * R + t];
            b[4 * t] = v.x; b[4 * t + 1] = v.y; b[4 * t + 2] = v.z; b[4 * t + 3] = v.w;
        }
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            if (lane + 32 * q < M) {
                const float4 sv = reinterpret_cast<const float4 *>(S + (lane + 32 * q) * p32)[c4];
#pragma unroll
                for (int c = 0; c < R; ++c) {
                    float acc = y[q][c];
                    acc = fmaf(sv.x, b[c], acc);
                    acc = fmaf(sv.y, b[R + c], acc);
                    acc = fmaf(sv.z, b[2 * R + c], acc);
                    acc = fmaf(sv.w, b[3 * R + c], acc);
                    y[q][c] = acc;
                }
            }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < RPL; ++q)
        if (lane + 32 * q < M)
#pragma unroll
            for (int c = 0; c < R; ++c) V[step[q] * R + c] = y[q][c];
    __syncwarp();
}

// Per-warp shared memory of the mixed kernel (byte offsets, 16-aligned).
struct MixedLayout {
    int pA, p32;
    size_t a64, q64, b64, x64, xi, a32, u32, v32, bp, perm, bytes;
};

__host__ __device__ inline MixedLayout mixed_layout(int n_max, int l, int R, int dim) {
    MixedLayout L{};
    const int M = n_max + l, C4 = (M + 3) / 4;
    L.pA = n_max | 1;
    L.p32 = 4 * (C4 | 1);              // 4 * odd >= 4 * ceil(M/4)
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
    L.u32 = take((size_t)2 * 4 * C4 * 4);
    L.v32 = take((size_t)M * R * 4);
    L.bp = take((size_t)4 * C4 * R * 4);
    // u32 .. bp double as the 4 * (4 C4) floats of the register-resident
    // inverse's scratch (v32 and bp are used only after the inverse)
    if (o - L.u32 < (size_t)4 * 4 * C4 * 4) o = L.u32 + (size_t)4 * 4 * C4 * 4;
    L.perm = take((size_t)M * 4);
    L.bytes = o;
    return L;
}

// ------------------------------------------------ double-FP32 arithmetic
// A value is the unevaluated sum hi + lo of two floats (float2 {hi, lo},
// |lo| <= ulp(hi)), about 48 significant bits, computed on the FP32 pipe
// (GB300 issues FP32 at ~70x its FP64 rate).  Built from the error-free
// transformations TwoSum (Knuth), Fast2Sum (Dekker) and the FMA-based exact
// product; the _rn intrinsics keep the compiler from contracting them.
__device__ __forceinline__ float2 ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
// |a| >= |b| or a == 0
__device__ __forceinline__ float2 ff_fast_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    const float2 t = ff_two_sum(a.x, b.x);
    return ff_fast_sum(t.x, __fadd_rn(t.y, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 ff_sub(float2 a, float2 b) { return ff_add(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    return ff_fast_sum(p, e);
}
__device__ __forceinline__ float2 ff_scale(float2 a, float b) {
    const float p = __fmul_rn(a.x, b);
    return ff_fast_sum(p, fmaf(a.y, b, fmaf(a.x, b, -p)));
}
// square root by one Newton correction of the FP32 root: (a - h^2) / (2h)
__device__ __forceinline__ float2 ff_sqrt(float2 a) {
    if (!(a.x > 0.0f)) return make_float2(0.0f, 0.0f);
    const float h = __fsqrt_rn(a.x);
    const float p = __fmul_rn(h, h);
    const float t = __fadd_rn(__fsub_rn(__fsub_rn(a.x, p), fmaf(h, h, -p)), a.y);
    return ff_fast_sum(h, __fmul_rn(t, __fmul_rn(0.5f, __frcp_rn(h))));
}
__device__ __forceinline__ float2 ff_from_double(double d) {
    const float h = __double2float_rn(d);
    return make_float2(h, __double2float_rn(d - (double)h));
}
// r^k for odd k >= 1 from r^2
__device__ __forceinline__ float2 ff_phs(float2 r2, int k) {
    float2 v = ff_sqrt(r2);
    for (int i = 1; i < k; i += 2) v = ff_mul(v, r2);
    return v;
}
// r^(k-2) for odd k >= 3 from r^2
__device__ __forceinline__ float2 ff_phs_km2(float2 r2, int k) {
    float2 v = ff_sqrt(r2);
    for (int i = 3; i < k; i += 2) v = ff_mul(v, r2);
    return v;
}
// 1/a by one Newton correction of the FP32 reciprocal (a != 0)
__device__ __forceinline__ float2 ff_recip(float2 a) {
    const float h = __frcp_rn(a.x);
    const float e = __fsub_rn(fmaf(-a.x, h, 1.0f), __fmul_rn(a.y, h));   // 1 - a h
    return ff_fast_sum(h, __fmul_rn(h, e));
}
// the double-FP32 counterpart of phs_d2 (xf: this node's offsets)
__device__ inline float2 ff_phs_d2(int op, int k, float2 r2, float2 rk2, const float2 *xf) {
    const int a = d2_a(op), c = d2_c(op);
    float2 v = a == c ? ff_scale(rk2, (float)k) : make_float2(0.0f, 0.0f);
    if (r2.x > 0.0f) {
        // r^(k-4): r^-1 for k = 3, else r (r^2)^((k-5)/2)
        const float2 rk4 = k == 3 ? ff_recip(ff_sqrt(r2)) : ff_phs_km2(r2, k - 2);
        v = ff_add(v, ff_scale(ff_mul(rk4, ff_mul(xf[a], xf[c])), (float)(k * (k - 2))));
    }
    return v;
}

// The system for the residuals in double-FP32: A [n x pA] (diagonal 0), Q
// [n x l], B [M x R] (rows < n: l_phi, rows n + b: l_q), from the scaled
// offsets xf [n x DIM] (double-FP32).  The leading FP32 parts of A, Q and Q^T
// go to the FP32 system S [rows x p32] as they are formed (its zero block and
// padding are the caller's).  Returns max |K| over A and Q (FP32).
template <int DIM>
__device__ __forceinline__ float assemble_ff(const WParams &P, int64_t row, int n, const float2 *xf, float2 *A, int pA,
                             float2 *Q, float2 *B, int R, float *S, int p32) {
    const int lane = threadIdx.x & 31;
    const int l = P.l, k = P.k, di = DIM - 2;
    float amax = 0.0f;
    // the n (n - 1) / 2 unordered pairs (r, (r + d) mod n), d = 1 .. n/2 (r < n/2
    // for d = n/2), numbered t = (d - 1) n + r and dealt to the lanes in turn
    const int npairs = n * (n - 1) / 2;
    int d = 1 + lane / max(n, 1), r = lane % max(n, 1);
#pragma unroll 2
    for (int t = lane; t < npairs; t += 32) {
        int c = r + d;
        if (c >= n) c -= n;
        float2 r2 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const float2 dx = ff_sub(xf[r * DIM + a], xf[c * DIM + a]);
            r2 = ff_add(r2, ff_mul(dx, dx));
        }
        const float2 v = ff_phs(r2, k);
        A[r * pA + c] = v;
        A[c * pA + r] = v;
        S[r * p32 + c] = v.x;
        S[c * p32 + r] = v.x;
        amax = fmaxf(amax, v.x);
        r += 32;
        while (r >= n) {
            r -= n;
            ++d;
        }
    }
    for (int r = lane; r < n; r += 32) {
        A[r * pA + r] = make_float2(0.0f, 0.0f);
        S[r * p32 + r] = 0.0f;
        float2 *Qr = Q + r * l;
        Qr[0] = make_float2(1.0f, 0.0f);
        S[r * p32 + n] = 1.0f;
        S[n * p32 + r] = 1.0f;
        for (int b = 1; b < l; ++b) {
            const float2 v = ff_mul(Qr[c_mono.parent[di][b]], xf[r * DIM + c_mono.var[di][b]]);
            Qr[b] = v;
            S[r * p32 + n + b] = v.x;
            S[(n + b) * p32 + r] = v.x;
            amax = fmaxf(amax, fabsf(v.x));
        }
        float2 r2 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int a = 0; a < DIM; ++a) r2 = ff_add(r2, ff_mul(xf[r * DIM + a], xf[r * DIM + a]));
        const float2 rk2 = ff_phs_km2(r2, k);
        for (int cI = 0; cI < R; ++cI) {
            const int op = P.opcode[cI];
            float2 v;
            if (cI >= P.R) {
                v = make_float2(0.0f, 0.0f);      // unused solver column
            } else if (op == 0) {
                v = ff_scale(rk2, (float)(k * (k + DIM - 2)));
            } else if (op >= 5) {
                v = ff_phs_d2(op, k, r2, rk2, xf + r * DIM);
            } else {
                float2 dot;
                if (op == 4) {
                    dot = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int a = 0; a < DIM; ++a)
                        dot = ff_add(dot, ff_mul(ff_from_double(P.normals[row * DIM + a]), xf[r * DIM + a]));
                } else {
                    dot = xf[r * DIM + (op - 1)];
                }
                v = ff_scale(ff_mul(rk2, dot), -(float)k);
            }
            B[r * R + cI] = v;
        }
    }
    for (int b = lane; b < l; b += 32) {
        for (int cI = 0; cI < R; ++cI) {
            const int op = P.opcode[cI];
            float2 v = make_float2(0.0f, 0.0f);
            if (cI < P.R) {
                if (op == 0) {
                    v.x = (float)c_mono.lap[di][b];
                } else if (op >= 5) {
                    v.x = (float)d2_of_monomial(di, b, op);
                } else {
                    const int a = c_mono.lin[di][b];
                    if (a >= 0) v = op == 4 ? ff_from_double(P.normals[row * DIM + a])
                                            : make_float2((a == op - 1) ? 1.0f : 0.0f, 0.0f);
                }
            }
            B[(n + b) * R + cI] = v;
        }
    }
    __syncwarp();
    return warp_maxf(fmaxf(amax, 1.0f));
}

// The same system in native FP64: A64 [n x pA] (diagonal 0), Q64 [n x l],
// B64 [M x R] (rows < n: l_phi, rows n + b: l_q).  Returns max |K| (FP32).
template <int DIM>
__device__ __noinline__ float assemble_f64(const WParams &P, int64_t row, int n, const double *xi, double *A64, int pA,
                              double *Q64, double *B64, int R) {
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
            } else if (op >= 5) {
                v = phs_d2(op, k, r2, rk2, xi + r * DIM);
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
            if (cI < P.R) {
                if (op == 0) {
                    v = (double)c_mono.lap[di][b];
                } else if (op >= 5) {
                    v = (double)d2_of_monomial(di, b, op);
                } else {
                    const int a = c_mono.lin[di][b];
                    if (a >= 0) v = op == 4 ? P.normals[row * DIM + a] : ((a == op - 1) ? 1.0 : 0.0);
                }
            }
            B64[(n + b) * R + cI] = v;
        }
    }
    __syncwarp();
    return warp_maxf(fmaxf((float)amax, 1.0f));
}

// Compensated dot product (Ogita, Rump & Oishi) in double-FP32: acc -= kx * xx.
// The product of the high parts is split exactly and subtracted from hi with
// TwoSum; the rounding errors go to lo and the cross terms to la and lb (three
// independent chains, so consecutive terms overlap).  The value is
// hi + (lo + (la + lb)).
struct FFAcc {
    float hi, lo, la, lb;
    __device__ __forceinline__ explicit FFAcc(float2 b) : hi(b.x), lo(b.y), la(0.0f), lb(0.0f) {}
    __device__ __forceinline__ void sub(float2 kx, float2 xx) {
        const float p = __fmul_rn(kx.x, xx.x);
        const float pe = fmaf(kx.x, xx.x, -p);
        const float2 t = ff_two_sum(hi, -p);
        hi = t.x;
        lo = __fadd_rn(lo, __fsub_rn(t.y, pe));
        la = fmaf(-kx.x, xx.y, la);
        lb = fmaf(-kx.y, xx.x, lb);
    }
    __device__ __forceinline__ float value() const { return __fadd_rn(hi, __fadd_rn(lo, __fadd_rn(la, lb))); }
};

// The wide arithmetic of the refinement: the system (A, Q, b) and the
// solution x as double-FP32 pairs (WideFF, on the FP32 pipe) or as FP64
// (Wide64); the residual of row i, column c over the nonzero blocks of K.
struct WideFF {
    using T = float2;
    static __device__ __forceinline__ float hi(T v) { return v.x; }
    static __device__ __forceinline__ T from_f(float d) { return make_float2(d, 0.0f); }
    static __device__ __forceinline__ T add_f(T x, float d) {
        const float2 t = ff_two_sum(x.x, d);
        return ff_fast_sum(t.x, __fadd_rn(t.y, x.y));
    }
    static __device__ __forceinline__ double to_d(T x) { return (double)x.x + (double)x.y; }
    // rows i < n: A row i then Q row i; rows n + b: column b of Q.  One loop
    // serves both kinds (base and stride per lane), so lanes of a warp on
    // different kinds do not run both loops.
    static __device__ __forceinline__ float residual(const T *A, int pA, const T *Q, int l, const T *B,
                                                     const T *X, int n, int R, int i, int c) {
        FFAcc acc(B[i * R + c]);
        const bool arow = i < n;
        const T *p1 = arow ? A + i * pA : Q + (i - n);
        const int s1 = arow ? 1 : l;
        for (int j = 0; j < n; ++j) acc.sub(p1[j * s1], X[j * R + c]);
        const T *p2 = arow ? Q + i * l : Q;
        const int n2 = arow ? l : 0;
        for (int b = 0; b < n2; ++b) acc.sub(p2[b], X[(n + b) * R + c]);
        return acc.value();
    }
};

struct Wide64 {
    using T = double;
    static __device__ __forceinline__ float hi(T v) { return (float)v; }
    static __device__ __forceinline__ T from_f(float d) { return (double)d; }
    static __device__ __forceinline__ T add_f(T x, float d) { return x + (double)d; }
    static __device__ __forceinline__ double to_d(T x) { return x; }
    static __device__ __forceinline__ float residual(const T *A, int pA, const T *Q, int l, const T *B,
                                                     const T *X, int n, int R, int i, int c) {
        double acc = B[i * R + c];
        if (i < n) {
            const T *Ai = A + i * pA;
            const T *Qi = Q + i * l;
            for (int j = 0; j < n; ++j) acc = fma(-Ai[j], X[j * R + c], acc);
            for (int b = 0; b < l; ++b) acc = fma(-Qi[b], X[(n + b) * R + c], acc);
        } else {
            const int b = i - n;
            for (int j = 0; j < n; ++j) acc = fma(-Q[j * l + b], X[j * R + c], acc);
        }
        return (float)acc;
    }
};

// Refinement after the FP32 inverse: x0 = K^-1 b, then x <- x + K^-1 (b - K x)
// for at least two steps and until the observed contraction shows the
// remaining error below the tolerance; then one correction from the
// constraint rows alone.  Returns false if it did not converge.
template <int RPL, int R, class Wd>
__device__ __forceinline__ bool mixed_refine(const WParams &P, int n, int M, const float *S, int p32, const int *step,
                             const int *perm, const typename Wd::T *Aw, int pA, const typename Wd::T *Qw,
                             const typename Wd::T *Bw, typename Wd::T *Xw, float *V32, float *Bp) {
    const int lane = threadIdx.x & 31, l = P.l;
    for (int e = lane; e < M * R; e += 32) V32[e] = Wd::hi(Bw[e]);
    __syncwarp();
    gj32_apply<RPL, R>(S, p32, M, step, perm, V32, Bp);
    float dmax = 0.0f;
    for (int e = lane; e < M * R; e += 32) {
        const float d = V32[e];
        Xw[e] = Wd::from_f(d);
        dmax = fmaxf(dmax, fabsf(d));
    }
    float dprev = warp_maxf(dmax);
    __syncwarp();
    bool conv = false;
    for (int it = 1; it <= P.ir_max_steps; ++it) {
        for (int e = lane; e < M * R; e += 32) {
            const int i = e / R, c = e - i * R;
            V32[e] = Wd::residual(Aw, pA, Qw, l, Bw, Xw, n, R, i, c);
        }
        __syncwarp();
        gj32_apply<RPL, R>(S, p32, M, step, perm, V32, Bp);
        float dmx = 0.0f, xmax = 0.0f;
        for (int e = lane; e < M * R; e += 32) {
            const float d = V32[e];
            const typename Wd::T xn = Wd::add_f(Xw[e], d);
            Xw[e] = xn;
            dmx = fmaxf(dmx, fabsf(d));
            if (e < n * R) xmax = fmaxf(xmax, fabsf(Wd::hi(xn)));
        }
        dmx = warp_maxf(dmx);
        xmax = warp_maxf(xmax);
        // the observed contraction of the last step bounds the error left;
        // it is taken from two corrections (the first step's ratio compares
        // a correction with the solution itself and can underestimate it)
        const float theta = dmx / fmaxf(dprev, 1e-30f);
        if (it >= 2 && theta < 0.5f && theta / (1.0f - theta) * dmx <= (float)P.ir_tol * xmax) {
            conv = true;
            break;
        }
        dprev = dmx;
        __syncwarp();
    }
    if (!conv) return false;
    // Constraint rows Q^T w = l_q: one more residual on those rows only,
    // corrected through the FP32 inverse, so the monomials are reproduced to
    // the residual's precision rather than to the refinement tolerance.
    __syncwarp();
    for (int e = lane; e < M * R; e += 32) {
        const int i = e / R, c = e - i * R;
        V32[e] = i >= n ? Wd::residual(Aw, pA, Qw, l, Bw, Xw, n, R, i, c) : 0.0f;
    }
    __syncwarp();
    gj32_apply<RPL, R>(S, p32, M, step, perm, V32, Bp);
    for (int e = lane; e < n * R; e += 32) Xw[e] = Wd::add_f(Xw[e], V32[e]);
    __syncwarp();
    return true;
}

// One stencil (row) with the FP32 + refinement solver; `base` is the warp's
// shared memory.  Returns true if the row must go to the FP64 solver (its
// status is then MM_ST_NONCONVERGED and its weights are not written).
//
// K is inverted once in FP32 (Gauss-Jordan above); every solve is then a
// product with that inverse.  The 1-norm condition number of K follows from
// ||K||_1 and the exact infinity norm of the computed inverse (K is
// symmetric, so both norms agree); a stencil with ||K|| ||K^-1|| u32 above
// the bound goes to the FP64 solver.  The refinement (mixed_refine) keeps K,
// b and x in double-FP32 with compensated residuals, or in FP64 (P.wide64).
// W > 0 (= 4 ceil(M_max / 4)) selects the register-resident inverse.
template <int DIM, int RPL, int R, int W = 0>
__device__ __noinline__ bool mixed_row(const WParams &P, int64_t row, char *base) {
    const int lane = threadIdx.x & 31;
    const MixedLayout Ly = mixed_layout(P.n_max, P.l, R, DIM);
    double *xi = (double *)(base + Ly.xi);
    float *S = (float *)(base + Ly.a32);
    float *U32 = (float *)(base + Ly.u32);
    float *V32 = (float *)(base + Ly.v32);
    float *Bp = (float *)(base + Ly.bp);
    int *perm = (int *)(base + Ly.perm);
    const int pA = Ly.pA, p32 = Ly.p32, l = P.l;
    const float u32 = FLT_EPSILON * 0.5f;
    int n;
    int64_t rb;
    double s;
    if (!load_stencil<DIM>(P, row, n, rb, xi, s)) {
        reject_row(P, row, rb, n, MM_ST_BADARG);
        __syncwarp();
        return false;
    }
    const int M = n + l, W4 = 4 * ((M + 3) >> 2);
    // the system in wide arithmetic (A [n x pA], Q [n x l], b [M x R]; 8 bytes per entry)
    float amax;
    if (P.wide64) {
        amax = assemble_f64<DIM>(P, row, n, xi, (double *)(base + Ly.a64), pA, (double *)(base + Ly.q64),
                                 (double *)(base + Ly.b64), R);
    } else {
        // scaled offsets to double-FP32, in place (same 8 bytes per coordinate)
        float2 *xf = reinterpret_cast<float2 *>(xi);
        for (int j = lane; j < n * DIM; j += 32) xf[j] = ff_from_double(xi[j]);
        __syncwarp();
        amax = assemble_ff<DIM>(P, row, n, xf, (float2 *)(base + Ly.a64), pA, (float2 *)(base + Ly.q64),
                                (float2 *)(base + Ly.b64), R, S, p32);
    }
    // FP32 system: the leading parts (own rows; Q^T entries written by the row's owner)
    int step[RPL];
    const double *A64 = (const double *)(base + Ly.a64), *Q64 = (const double *)(base + Ly.q64);
    const float2 *Af = (const float2 *)(base + Ly.a64), *Qf = (const float2 *)(base + Ly.q64);
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        const int r = lane + 32 * q;
        step[q] = r < M ? kBig : -1;
        if (r < n) {
            // (the double-FP32 assembly wrote its leading parts as it went)
            if (P.wide64) {
                float *Sr = S + r * p32;
                for (int c = 0; c < n; ++c) Sr[c] = (float)A64[r * pA + c];
                for (int b = 0; b < l; ++b) {
                    const float v = (float)Q64[r * l + b];
                    Sr[n + b] = v;
                    S[(n + b) * p32 + r] = v;
                }
            }
        } else if (r < M) {
            for (int c = n; c < M; ++c) S[r * p32 + c] = 0.0f;
        }
        if (r < M)
            for (int c = M; c < W4; ++c) S[r * p32 + c] = 0.0f;
    }
    __syncwarp();
    // ||K||_1 and ||K^-1||_1 as max row sums (K and its inverse are symmetric)
    float n1 = 0.0f, ninv = 0.0f;
    bool queue;
    if constexpr (W > 0) {
        queue = !gj32_invert_reg<W>(S, p32, M, step, perm, U32, (float)M * u32 * amax, n1, ninv);
    } else {
        auto rows_norm = [&]() {
            float v = 0.0f;
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const int r = lane + 32 * q;
                if (r < M) {
                    float rs = 0.0f;
                    for (int c = 0; c < M; ++c) rs += fabsf(S[r * p32 + c]);
                    v = fmaxf(v, rs);
                }
            }
            return warp_maxf(v);
        };
        n1 = rows_norm();
        queue = !gj32_invert<RPL>(S, p32, M, step, perm, U32, (float)M * u32 * amax);
        if (!queue) ninv = rows_norm();
    }
    if (!queue) queue = !((double)n1 * (double)ninv * u32 <= P.kappa_max);
    bool conv = false;
    if (!queue) {
        if (P.wide64)
            conv = mixed_refine<RPL, R, Wide64>(P, n, M, S, p32, step, perm, A64, pA, Q64,
                                                (const double *)(base + Ly.b64), (double *)(base + Ly.x64),
                                                V32, Bp);
        else
            conv = mixed_refine<RPL, R, WideFF>(P, n, M, S, p32, step, perm, Af, pA, Qf,
                                                (const float2 *)(base + Ly.b64), (float2 *)(base + Ly.x64),
                                                V32, Bp);
    }
    if (!conv) {
        if (P.status && lane == 0) P.status[row] = MM_ST_NONCONVERGED;
        __syncwarp();
        return true;
    }
    // unscaled store
    const double inv_s = recip_nr(s);
    for (int cI = 0; cI < P.R; ++cI) {
        const double sc = op_order(P.opcode[cI]) == 2 ? inv_s * inv_s : inv_s;
        double *out = P.vals[cI] + rb;
        if (P.wide64) {
            const double *X = (const double *)(base + Ly.x64);
            for (int j = lane; j < n; j += 32) out[j] = X[j * R + cI] * sc;
        } else {
            const float2 *X = (const float2 *)(base + Ly.x64);
            for (int j = lane; j < n; j += 32) out[j] = WideFF::to_d(X[j * R + cI]) * sc;
        }
    }
    if (P.status && lane == 0) P.status[row] = MM_ST_OK;
    __syncwarp();
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
    for (int b = 0; b < 11 && R < 5; ++b)      // callers pass at most 5 operator bits
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
    P.wide64 = ctx->wide64;
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
            t.d2[di][b] = -1;
            if (deg == 2) {
                int a0 = -1, a1 = -1;
                for (int a = 0; a < 3; ++a)
                    for (int r = 0; r < exps[b][a]; ++r) (a0 < 0 ? a0 : a1) = a;
                t.d2[di][b] = (signed char)(3 * a0 + a1);
            }
        }
        for (int b = cnt; b < kMaxMono; ++b) {
            t.parent[di][b] = t.var[di][b] = t.lap[di][b] = 0;
            t.lin[di][b] = -1;
            t.d2[di][b] = -1;
        }
    }
}

}  // namespace
