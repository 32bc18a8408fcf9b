// The implicit solve of Section 2.3.2: the PDE is discretised by replacing
// every differential operator with its RBF-FD weights, which gives one sparse
// row per node (interior: the operator's weights; Dirichlet: the identity;
// Neumann: the d/dn weights), and the system M u = r is solved with BiCGSTAB
// preconditioned by an incomplete LU factorisation (the paper uses ILUT; this
// is ILU(0), the factorisation restricted to the pattern of M).
//
// Kernels:
//   k_assemble     one warp per row: the row's entries sorted by column (ILU
//                  needs sorted rows), Dirichlet rows replaced by the identity.
//   k_ilu0         one warp per row, rows taken in increasing order from an
//                  atomic ticket; row i waits for the rows k < i of its lower
//                  part (a per-row flag, release/acquire) and eliminates them
//                  in increasing k, each entry updated in the same order and
//                  with the same roundings (no fused multiply-add) as the
//                  plain row-by-row algorithm, so the factors are bit-exact.
//   k_lower/k_upper  sync-free triangular solves: rows in ticket order
//                  (increasing for L, decreasing for U), every row waits only
//                  for the unknowns it needs.  An unknown's own value is its
//                  readiness flag: the output vector is filled with a
//                  signalling-NaN pattern that arithmetic never produces, a
//                  row polls the entries it needs until they differ from it,
//                  so a dependency costs one L2 round trip.
//   k_spmv_dot, k_update, k_scalars  BiCGSTAB's products, vector updates and
//                  dot products (block partial sums reduced in a fixed order
//                  by one block: deterministic), all scalars kept on the GPU.
// Every wait is bounded: after kSpinMax polls the warp records an error and
// goes on with the value it has (the call then fails with MM_ECUDA).
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "mm_internal.cuh"

namespace {

constexpr uint64_t kPending = 0x7FF4DEADBEEF0001ull;   // signalling NaN: "not computed yet"
constexpr uint32_t kSpinMax = 1u << 22;
constexpr int kRowMax = 64;                              // entries per row
constexpr int kTickets = 4;                              // ticket counters, used round-robin

__device__ __forceinline__ uint64_t ld_relaxed_u64(const void *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(void *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until x[k] holds a computed value and returns it (bounded).
__device__ __forceinline__ double wait_value(const double *x, int64_t k, int *err) {
    uint64_t v = ld_relaxed_u64(x + k);
    for (uint32_t i = 0; v == kPending; ++i) {
        if (i >= kSpinMax) {
            atomicExch(err, 1);
            return 0.0;
        }
        if (i > 32) __nanosleep(32);
        v = ld_relaxed_u64(x + k);
    }
    return __longlong_as_double((long long)v);
}

// Next ticket of this launch (lane 0 draws, the warp shares it).
__device__ __forceinline__ int64_t next_ticket(unsigned long long *counter) {
    unsigned long long t = 0;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(counter, 1ull);
    return (int64_t)__shfl_sync(0xffffffffu, t, 0);
}

// The launch's ticket counter is tickets[slot]; it zeroes the next slot for
// the next launch on the stream (launches on one stream do not overlap).
__device__ __forceinline__ void reset_next_ticket(unsigned long long *tickets, int slot) {
    if (blockIdx.x == 0 && threadIdx.x == 0) tickets[(slot + 1) % kTickets] = 0ull;
}

// ------------------------------------------------------------------ assembly
// Row i of the implicit matrix: the stencil row's entries sorted by column;
// rows with kind MM_ROW_DIRICHLET become the identity row on the same
// pattern (1 on the diagonal, explicit zeros elsewhere).  A row without its
// own index, with a repeated column or longer than kRowMax sets *err.
__global__ void __launch_bounds__(256) k_assemble(int64_t nrows, const int64_t *__restrict__ rp,
                                                  const int32_t *__restrict__ col,
                                                  const double *__restrict__ val,
                                                  const uint8_t *__restrict__ kind, int32_t *__restrict__ ocol,
                                                  double *__restrict__ oval, int *err) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < nrows; i += nw) {
        const int64_t b = rp[i];
        const int n = (int)(rp[i + 1] - b);
        if (n < 1 || n > kRowMax) {
            if (lane == 0) atomicExch(err, 2);
            continue;
        }
        const bool dir = kind && kind[i] == MM_ROW_DIRICHLET;
        int c[2];
        double v[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int j = lane + 32 * s;
            c[s] = j < n ? col[b + j] : 0x7FFFFFFF;
            v[s] = j < n ? val[b + j] : 0.0;
            if (j < n && (c[s] < 0 || (int64_t)c[s] >= nrows)) atomicExch(err, 6);
        }
        // rank of each entry = entries with a smaller column (or the same
        // column at a lower position, which is reported as an error)
        int rank[2] = {0, 0}, dup = 0, has_diag = 0;
        for (int j = 0; j < n; ++j) {
            const int cj = __shfl_sync(0xffffffffu, c[j >> 5], j & 31);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int me = lane + 32 * s;
                if (me < n) {
                    rank[s] += cj < c[s] || (cj == c[s] && j < me);
                    dup |= cj == c[s] && j != me;
                }
            }
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int me = lane + 32 * s;
            if (me < n) {
                has_diag |= c[s] == (int)i;
                ocol[b + rank[s]] = c[s];
                oval[b + rank[s]] = dir ? (c[s] == (int)i ? 1.0 : 0.0) : v[s];
            }
        }
        if (__any_sync(0xffffffffu, dup) && lane == 0) atomicExch(err, 3);
        if (!__any_sync(0xffffffffu, has_diag) && lane == 0) atomicExch(err, 4);
    }
}

// ------------------------------------------------------------------ ILU(0)
// In-place ILU(0) of the sorted matrix F (a copy of M): row i, for every k <
// i of its pattern in increasing order, l_ik = f_ik / u_kk, then
// f_ij -= l_ik u_kj for every j > k present in both rows (the IKJ order of
// the plain algorithm; updates outside the pattern are dropped).  diag[i]
// receives the position of (i, i).  Row k is read only after flag[k] ==
// epoch (row k's warp writes its factors, fences, then releases the flag).
__global__ void __launch_bounds__(256) k_ilu0(int64_t nrows, const int64_t *__restrict__ rp,
                                              const int32_t *__restrict__ col, double *F,
                                              int64_t *diag, uint32_t *flag, uint32_t epoch,
                                              unsigned long long *tickets, int slot, int *err) {
    reset_next_ticket(tickets, slot);
    const int lane = threadIdx.x & 31;
    for (;;) {
        const int64_t i = next_ticket(tickets + slot);
        if (i >= nrows) break;
        const int64_t b = rp[i];
        int n = (int)(rp[i + 1] - b);
        if (n > kRowMax) {   // not factored (the call fails); the flag is still released
            if (lane == 0) atomicExch(err, 2);
            n = kRowMax;
        }
        int c[2];
        double a[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int j = lane + 32 * s;
            c[s] = j < n ? col[b + j] : 0x7FFFFFFF;
            a[s] = j < n ? F[b + j] : 0.0;
        }
        int d = -1;   // position of the diagonal within the row
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const unsigned m = __ballot_sync(0xffffffffu, c[s] == (int)i);
            if (m && d < 0) d = 32 * s + __ffs(m) - 1;
        }
        // columns in range and increasing (else the row is not factored)
        bool bad = false;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int j = lane + 32 * s;
            const int nxt = __shfl_down_sync(0xffffffffu, c[s], 1);       // entry j + 1 (lanes 0..30)
            const int wrap = __shfl_sync(0xffffffffu, c[1], 0);           // entry 32
            const int succ = lane < 31 ? nxt : (s == 0 ? wrap : 0x7FFFFFFF);
            if (j < n) bad |= c[s] < 0 || (int64_t)c[s] >= nrows || (j + 1 < n && succ <= c[s]);
        }
        bad = __any_sync(0xffffffffu, bad);
        if (d < 0 || bad) {
            if (lane == 0) atomicExch(err, bad ? 6 : 4);
            d = 0;   // no elimination: the row is stored as it is and released
        }
        for (int j = 0; j < d; ++j) {
            const int k = __shfl_sync(0xffffffffu, c[j >> 5], j & 31);
            int ready = 1;
            if (lane == 0) {
                uint32_t f = ld_acquire_u32(flag + k);
                for (uint32_t t = 0; f != epoch; ++t) {
                    if (t >= kSpinMax) {
                        atomicExch(err, 1);
                        ready = 0;
                        break;
                    }
                    if (t > 32) __nanosleep(64);
                    f = ld_acquire_u32(flag + k);
                }
            }
            // a row that never finished is not read (its diag entry is unset)
            if (!__shfl_sync(0xffffffffu, ready, 0)) continue;
            (void)ld_acquire_u32(flag + k);   // every lane acquires the row's release
            const int64_t dk = (int64_t)__ldcg((const long long *)diag + k);
            const int64_t ek = __ldcg(rp + k + 1);
            const double ukk = __ldcg(F + dk);
            double lik = 0.0;
            if (lane == (j & 31)) {
                const int s = j >> 5;
                if (ukk == 0.0) {
                    atomicExch(err, 5);
                } else {
                    lik = __ddiv_rn(a[s], ukk);
                }
                a[s] = lik;
            }
            lik = __shfl_sync(0xffffffffu, lik, j & 31);
            // U part of row k: positions dk+1 .. ek-1 (at most 63)
            const int m = (int)(ek - dk - 1 < kRowMax - 1 ? ek - dk - 1 : kRowMax - 1);
            int uc[2];
            double uv[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int q = lane + 32 * s;
                uc[s] = q < m ? __ldcg(col + dk + 1 + q) : -1;
                uv[s] = q < m ? __ldcg(F + dk + 1 + q) : 0.0;
            }
            for (int q = 0; q < m; ++q) {
                const int cq = __shfl_sync(0xffffffffu, uc[q >> 5], q & 31);
                const double vq = __shfl_sync(0xffffffffu, uv[q >> 5], q & 31);
#pragma unroll
                for (int s = 0; s < 2; ++s)
                    if (c[s] == cq) a[s] = __dsub_rn(a[s], __dmul_rn(lik, vq));
            }
        }
        if (lane == (d & 31) && a[d >> 5] == 0.0) atomicExch(err, 5);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int j = lane + 32 * s;
            if (j < n) F[b + j] = a[s];
        }
        if (lane == 0) diag[i] = b + d;
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release_u32(flag + i, epoch);
    }
}

__global__ void k_fill_pending(int64_t n, double *x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        reinterpret_cast<unsigned long long *>(x)[i] = kPending;
}

// ------------------------------------------------------- dependency levels
// Level of every row in a substitution: 0 without dependencies, else 1 + the
// largest level of the rows it reads (lower: columns < i of its row, upper:
// columns > i).  Sync-free like the substitutions (ticket order, each level a
// readiness flag: -1 until written); *maxlev receives the largest level.
template <bool LOWER>
__global__ void __launch_bounds__(256) k_levels(int64_t nrows, const int64_t *__restrict__ rp,
                                                const int32_t *__restrict__ col,
                                                const int64_t *__restrict__ diag, int32_t *lev, int32_t *maxlev,
                                                unsigned long long *tickets, int slot, int *err) {
    reset_next_ticket(tickets, slot);
    const int lane = threadIdx.x & 31;
    for (;;) {
        const int64_t t = next_ticket(tickets + slot);
        if (t >= nrows) break;
        const int64_t i = LOWER ? t : nrows - 1 - t;
        const int64_t b = LOWER ? __ldg(rp + i) : __ldg(diag + i) + 1;
        const int64_t e = LOWER ? __ldg(diag + i) : __ldg(rp + i + 1);
        int m = -1;
        for (int64_t p = b + lane; p < e; p += 32) {
            const int k = __ldg(col + p);
            int v;
            asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(lev + k) : "memory");
            for (uint32_t it = 0; v < 0; ++it) {
                if (it >= kSpinMax) {
                    atomicExch(err, 1);
                    v = 0;
                    break;
                }
                if (it > 32) __nanosleep(32);
                asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(lev + k) : "memory");
            }
            m = max(m, v);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) {
            asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(lev + i), "r"(m + 1) : "memory");
            atomicMax(maxlev, m + 1);
        }
    }
}

// Counting sort of the rows by level: counts, exclusive prefix (one block),
// scatter (the order inside a level is arbitrary: each row's arithmetic does
// not depend on it).
__global__ void k_level_count(int64_t nrows, const int32_t *__restrict__ lev, int32_t *count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(count + lev[i], 1);
}
__global__ void __launch_bounds__(1024) k_level_scan(const int32_t *maxlev, int32_t *count) {
    __shared__ int32_t part[32];
    const int nl = *maxlev + 1;
    int32_t carry = 0;
    for (int base = 0; base < nl; base += 1024) {
        const int i = base + threadIdx.x;
        const int32_t v = i < nl ? count[i] : 0;
        int32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) part[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            int32_t w = part[threadIdx.x];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (threadIdx.x >= o) w += y;
            }
            part[threadIdx.x] = w;
        }
        __syncthreads();
        const int32_t before = (threadIdx.x >= 32 ? part[(threadIdx.x >> 5) - 1] : 0) + x - v;
        if (i < nl) count[i] = carry + before;   // exclusive start of level i
        const int32_t tot = part[31];
        __syncthreads();
        carry += tot;
    }
}
__global__ void k_level_scatter(int64_t nrows, const int32_t *__restrict__ lev, int32_t *start, int32_t *order) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x)
        order[atomicAdd(start + lev[i], 1)] = (int32_t)i;
}

// ------------------------------------------------------- BiCGSTAB scalars
struct KrylovScalars {
    double rho, rho1, alpha, omega, beta, nb, res, tol;
    int it, maxit, stop;   // stop: 0 running, 1 converged, 2 breakdown, 3 iteration limit
    int pad;
};

// How the lower solve gets its right-hand side b_i
enum { kRhsPlain = 0, kRhsP = 1, kRhsS = 2 };

// Sync-free forward substitution with the unit lower factor: y = L^-1 b.
// y must hold kPending on entry; x_reset (optional) is set to kPending row by
// row (the output of the upper solve that follows).  kRhsP forms b = p = r +
// beta (p - omega v) and kRhsS b = s = r - alpha v, storing p or s.
template <int RHS>
__global__ void __launch_bounds__(256) k_lower(int64_t nrows, const int64_t *__restrict__ rp,
                                               const int32_t *__restrict__ col,
                                               const double *__restrict__ F,
                                               const int64_t *__restrict__ diag, const double *bvec,
                                               double *pv, const double *__restrict__ r,
                                               const double *__restrict__ v, const KrylovScalars *sc,
                                               double *y, double *x_reset, const int32_t *__restrict__ order,
                                               unsigned long long *tickets, int slot, int *err) {
    reset_next_ticket(tickets, slot);
    if (sc && sc->stop) return;
    const int lane = threadIdx.x & 31;
    double c1 = 0.0, c2 = 0.0;
    if (RHS == kRhsP) { c1 = sc->beta; c2 = sc->omega; }
    if (RHS == kRhsS) c1 = sc->alpha;
    for (;;) {
        const int64_t t = next_ticket(tickets + slot);
        if (t >= nrows) break;
        const int64_t i = order ? (int64_t)__ldg(order + t) : t;
        const int64_t b = __ldg(rp + i), dg = __ldg(diag + i);
        const int nl = (int)(dg - b);
        double acc = 0.0;
        for (int j = lane; j < nl; j += 32) {
            const int k = __ldg(col + b + j);
            acc = fma(__ldg(F + b + j), wait_value(y, k, err), acc);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            double bi;
            if (RHS == kRhsP) {
                bi = fma(c1, fma(-c2, v[i], pv[i]), r[i]);
                pv[i] = bi;
            } else if (RHS == kRhsS) {
                bi = fma(-c1, v[i], r[i]);
                pv[i] = bi;
            } else {
                bi = bvec[i];
            }
            st_relaxed_u64(y + i, (uint64_t)__double_as_longlong(bi - acc));
            if (x_reset) reinterpret_cast<unsigned long long *>(x_reset)[i] = kPending;
        }
    }
}

// Sync-free back substitution with the upper factor: x = U^-1 y, rows in
// decreasing order.  x must hold kPending on entry; y_reset (optional, may be
// y itself) is set to kPending row by row once the row has read y_i.
__global__ void __launch_bounds__(256) k_upper(int64_t nrows, const int64_t *__restrict__ rp,
                                               const int32_t *__restrict__ col,
                                               const double *__restrict__ F,
                                               const int64_t *__restrict__ diag, double *y, double *x,
                                               bool reset_y, const KrylovScalars *sc,
                                               const int32_t *__restrict__ order,
                                               unsigned long long *tickets, int slot, int *err) {
    reset_next_ticket(tickets, slot);
    if (sc && sc->stop) return;
    const int lane = threadIdx.x & 31;
    for (;;) {
        const int64_t t = next_ticket(tickets + slot);
        if (t >= nrows) break;
        const int64_t i = order ? (int64_t)__ldg(order + t) : nrows - 1 - t;
        const int64_t dg = __ldg(diag + i), e = __ldg(rp + i + 1);
        const int nu = (int)(e - dg - 1);
        double acc = 0.0;
        for (int j = lane; j < nu; j += 32) {
            const int k = __ldg(col + dg + 1 + j);
            acc = fma(__ldg(F + dg + 1 + j), wait_value(x, k, err), acc);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const double yi = y[i];
            st_relaxed_u64(x + i, (uint64_t)__double_as_longlong((yi - acc) / __ldg(F + dg)));
            if (reset_y) reinterpret_cast<unsigned long long *>(y)[i] = kPending;
        }
    }
}

// -------------------------------------------------- products and updates
constexpr int kVecThreads = 256;

// Sum of `v` over the block (fixed shuffle/shared-memory tree), valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    return t;
}

// Row dot product of a 4-lane group (lanes sub = 0..3 read every 4th entry).
__device__ __forceinline__ double row4(int64_t i, int sub, const int64_t *__restrict__ rp,
                                       const int32_t *__restrict__ col, const double *__restrict__ val,
                                       const double *__restrict__ x) {
    double acc = 0.0;
    const int64_t e = __ldg(rp + i + 1);
    for (int64_t p = __ldg(rp + i) + sub; p < e; p += 4) acc = fma(__ldg(val + p), __ldg(x + __ldg(col + p)), acc);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2, 4);
    return acc;
}

// MODE 0 (start): r = b - A x, rh = r, p = v = 0; partials ||b||^2, ||r||^2.
// MODE 1: v = A ph; partial rh.v.   MODE 2: t = A sh; partials t.s, t.t.
template <int MODE>
__global__ void __launch_bounds__(kVecThreads) k_spmv_dot(int64_t n, const int64_t *__restrict__ rp,
                                                          const int32_t *__restrict__ col,
                                                          const double *__restrict__ val,
                                                          const double *__restrict__ x, double *y,
                                                          const double *__restrict__ a, double *rh,
                                                          double *p, double *v, const KrylovScalars *sc,
                                                          double *partials) {
    __shared__ double sh[kVecThreads / 32];
    if (sc->stop) return;
    const int sub = threadIdx.x & 3;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) >> 2;
    double d0 = 0.0, d1 = 0.0;
    const int64_t steps = (n + ngroups - 1) / ngroups;
    for (int64_t s = 0; s < steps; ++s) {
        const int64_t i = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 2) + s * ngroups;
        const bool in = i < n;
        const double ax = row4(in ? i : 0, sub, rp, col, val, x);
        if (in && sub == 0) {
            if (MODE == 0) {
                const double bi = a[i], ri = bi - ax;
                y[i] = ri;
                rh[i] = ri;
                p[i] = 0.0;
                v[i] = 0.0;
                d0 += bi * bi;
                d1 += ri * ri;
            } else if (MODE == 1) {
                y[i] = ax;
                d0 += a[i] * ax;
            } else {
                y[i] = ax;
                d0 += ax * a[i];
                d1 += ax * ax;
            }
        }
    }
    d0 = block_sum(d0, sh);
    d1 = block_sum(d1, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = d0;
        partials[2 * blockIdx.x + 1] = d1;
    }
}

// x += alpha ph + omega sh; r = s - omega t; partials ||r||^2, rh.r.
__global__ void __launch_bounds__(kVecThreads) k_update(int64_t n, double *x, const double *__restrict__ ph,
                                                        const double *__restrict__ shv,
                                                        const double *__restrict__ s,
                                                        const double *__restrict__ t, double *r,
                                                        const double *__restrict__ rh,
                                                        const KrylovScalars *sc, double *partials) {
    __shared__ double sh[kVecThreads / 32];
    if (sc->stop) return;
    const double alpha = sc->alpha, omega = sc->omega;
    double d0 = 0.0, d1 = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = fma(omega, shv[i], fma(alpha, ph[i], x[i]));
        const double ri = fma(-omega, t[i], s[i]);
        r[i] = ri;
        d0 += ri * ri;
        d1 += rh[i] * ri;
    }
    d0 = block_sum(d0, sh);
    d1 = block_sum(d1, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = d0;
        partials[2 * blockIdx.x + 1] = d1;
    }
}

// Without a preconditioner: p = r + beta (p - omega v) (kRhsP) or
// s = r - alpha v (kRhsS), the "solve" being the identity.
template <int RHS>
__global__ void __launch_bounds__(kVecThreads) k_axpy_rhs(int64_t n, double *pv, const double *__restrict__ r,
                                                          const double *__restrict__ v,
                                                          const KrylovScalars *sc) {
    if (sc->stop) return;
    const double c1 = RHS == kRhsP ? sc->beta : sc->alpha, c2 = sc->omega;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pv[i] = RHS == kRhsP ? fma(c1, fma(-c2, v[i], pv[i]), r[i]) : fma(-c1, v[i], r[i]);
}

// Scalars from the partial sums (one block, fixed order).
//   kStart: nb = ||b||, res = ||r||/nb, rho1 = rh.r (= ||r||^2), beta = rho1.
//   kAlpha: alpha = rho1 / rh.v (rh.v == 0: breakdown).
//   kOmega: omega = t.s / t.t (0 if t = 0).
//   kNext:  res = ||r||/nb, it += 1; converged if res <= tol; else the next
//           iteration's rho1 = rh.r and beta = (rho1 / rho)(alpha / omega)
//           (rho1 == 0 or omega == 0: breakdown); iteration limit.
enum { kStart = 0, kAlpha = 1, kOmega = 2, kNext = 3 };
template <int STAGE>
__global__ void __launch_bounds__(kVecThreads) k_scalars(const double *partials, int nparts, KrylovScalars *sc) {
    __shared__ double sh[kVecThreads / 32];
    if (sc->stop) return;
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        s0 += partials[2 * i];
        s1 += partials[2 * i + 1];
    }
    s0 = block_sum(s0, sh);
    s1 = block_sum(s1, sh);
    if (threadIdx.x != 0) return;
    if (STAGE == kStart) {
        sc->nb = sqrt(s0);
        sc->res = sqrt(s1) / (sc->nb > 0.0 ? sc->nb : 1.0);
        sc->rho = sc->alpha = sc->omega = 1.0;
        sc->it = 0;
        if (sc->res <= sc->tol) { sc->stop = 1; return; }
        if (sc->maxit <= 0) { sc->stop = 3; return; }
        sc->rho1 = s1;
        if (s1 == 0.0) { sc->stop = 2; return; }
        sc->beta = s1;
    } else if (STAGE == kAlpha) {
        if (s0 == 0.0) { sc->stop = 2; return; }
        sc->alpha = sc->rho1 / s0;
    } else if (STAGE == kOmega) {
        sc->omega = s1 > 0.0 ? s0 / s1 : 0.0;
    } else {
        sc->it += 1;
        sc->res = sqrt(s0) / (sc->nb > 0.0 ? sc->nb : 1.0);
        if (sc->res <= sc->tol) { sc->stop = 1; return; }
        if (sc->it >= sc->maxit) { sc->stop = 3; return; }
        sc->rho = sc->rho1;
        sc->rho1 = s1;
        if (s1 == 0.0 || sc->omega == 0.0) { sc->stop = 2; return; }
        sc->beta = (sc->rho1 / sc->rho) * (sc->alpha / sc->omega);
    }
}

}  // namespace

// ======================================================================== host
namespace {

int bad_pattern(mm_ctx *ctx, const mm_csr_pattern *A) {
    if (!A || !A->d_row_ptr || !A->d_col || A->nrows < 1 || A->nrows >= (int64_t(1) << 31) || A->nnz < A->nrows)
        return mm_fail(ctx, MM_EBADARG, "bad matrix pattern (square CSR with a diagonal entry in every row)");
    return MM_OK;
}

int vec_blocks(const mm_ctx *ctx, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kVecThreads - 1) / kVecThreads, (int64_t)ctx->num_sms * 4));
}

// Blocks of 256 threads for a ticketed kernel: at most `per_sm_cap` per SM
// (and what fits at once).  The rows that can proceed at a time are one
// wavefront of the dependency graph (a few hundred to a few thousand rows),
// so more warps would only poll for their dependencies.
int ticket_blocks(mm_ctx *ctx, const void *kernel, int64_t rows, int per_sm_cap = 2) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    per_sm = std::min(per_sm, per_sm_cap);
    const int64_t want = (rows + 7) / 8;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)per_sm * ctx->num_sms));
}

int read_err(mm_ctx *ctx, const int *d_err, const char *what) {
    int e = 0;
    MM_CUDA_CHECK(ctx, cudaMemcpyAsync(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    MM_CUDA_CHECK(ctx, cudaStreamSynchronize(ctx->stream));
    switch (e) {
        case 0: return MM_OK;
        case 1: return mm_fail(ctx, MM_ECUDA, "%s: a wait for another row timed out", what);
        case 2: return mm_fail(ctx, MM_EUNSUPPORTED, "%s: a row has more than %d entries", what, kRowMax);
        case 3: return mm_fail(ctx, MM_EBADARG, "%s: a row lists a column twice", what);
        case 4: return mm_fail(ctx, MM_EBADARG, "%s: a row has no diagonal entry", what);
        case 5: return mm_fail(ctx, MM_ESINGULAR, "%s: zero pivot", what);
        case 6: return mm_fail(ctx, MM_EBADARG, "%s: a row's columns are out of range or not increasing", what);
    }
    return mm_fail(ctx, MM_ECUDA, "%s: error %d", what, e);
}

// Workspace of the solves: err, tickets, scalars, partials, flags, vectors,
// and (with levels) the rows of the two substitutions sorted by dependency level.
struct KrylovWs {
    int *err;
    unsigned long long *tickets;
    KrylovScalars *sc;
    double *partials;
    uint32_t *flag;
    double *vec[9];   // r, rh, p, v, ph, s, sh, t, Y
    int32_t *lev, *count, *maxlev, *ordL, *ordU;
};

int krylov_ws(mm_ctx *ctx, int64_t n, int nparts, int nvec, bool flags, KrylovWs *w, bool levels = false) {
    WsCarve c;
    const size_t o_err = c.take<int>(1), o_tk = c.take<unsigned long long>(kTickets),
                 o_sc = c.take<KrylovScalars>(1), o_part = c.take<double>(2 * (size_t)nparts),
                 o_flag = c.take<uint32_t>(flags ? (size_t)n : 1);
    size_t o_vec[9];
    for (int i = 0; i < nvec; ++i) o_vec[i] = c.take<double>((size_t)n);
    const size_t nl = levels ? (size_t)n : 1;
    const size_t o_lev = c.take<int32_t>(nl), o_cnt = c.take<int32_t>(nl + 1), o_max = c.take<int32_t>(1),
                 o_ordL = c.take<int32_t>(nl), o_ordU = c.take<int32_t>(nl);
    char *ws = mm_workspace(ctx, c.off);
    if (!ws) return mm_fail(ctx, MM_ENOMEM, "solver workspace of %zu bytes", c.off);
    w->err = (int *)(ws + o_err);
    w->tickets = (unsigned long long *)(ws + o_tk);
    w->sc = (KrylovScalars *)(ws + o_sc);
    w->partials = (double *)(ws + o_part);
    w->flag = (uint32_t *)(ws + o_flag);
    for (int i = 0; i < nvec; ++i) w->vec[i] = (double *)(ws + o_vec[i]);
    w->lev = (int32_t *)(ws + o_lev);
    w->count = (int32_t *)(ws + o_cnt);
    w->maxlev = (int32_t *)(ws + o_max);
    w->ordL = levels ? (int32_t *)(ws + o_ordL) : nullptr;
    w->ordU = levels ? (int32_t *)(ws + o_ordU) : nullptr;
    MM_CUDA_CHECK(ctx, cudaMemsetAsync(ws, 0, o_part, ctx->stream));   // err, tickets, scalars
    if (flags) MM_CUDA_CHECK(ctx, cudaMemsetAsync(w->flag, 0, (size_t)n * sizeof(uint32_t), ctx->stream));
    return MM_OK;
}

void fill_pending(mm_ctx *ctx, double *x, int64_t n) {
    k_fill_pending<<<vec_blocks(ctx, n), kVecThreads, 0, ctx->stream>>>(n, x);
}

// One application of (L U)^-1: y = L^-1 b (b formed by RHS), x = U^-1 y.
// On entry Y is all kPending; on exit again (the upper solve resets it).
template <int RHS>
void precond(mm_ctx *ctx, const mm_csr_pattern *A, const double *F, const int64_t *diag, const double *b,
             double *pv, const double *r, const double *v, const KrylovScalars *sc, double *Y, double *x,
             const KrylovWs &w, int &seq, int lblocks, int ublocks) {
    const int64_t n = A->nrows;
    k_lower<RHS><<<lblocks, 256, 0, ctx->stream>>>(n, A->d_row_ptr, A->d_col, F, diag, b, pv, r, v, sc, Y, x,
                                                   w.ordL, w.tickets, seq % kTickets, w.err);
    ++seq;
    k_upper<<<ublocks, 256, 0, ctx->stream>>>(n, A->d_row_ptr, A->d_col, F, diag, Y, x, true, sc, w.ordU,
                                              w.tickets, seq % kTickets, w.err);
    ++seq;
}

// The rows of both substitutions sorted by dependency level (ordL, ordU), so
// the tickets hand out the rows of one wavefront together.
template <bool LOWER>
void sort_by_level(mm_ctx *ctx, const mm_csr_pattern *A, const int64_t *diag, const KrylovWs &w, int &seq,
                   int32_t *order) {
    const int64_t n = A->nrows;
    cudaStream_t st = ctx->stream;
    cudaMemsetAsync(w.lev, 0xFF, sizeof(int32_t) * (size_t)n, st);
    cudaMemsetAsync(w.count, 0, sizeof(int32_t) * (size_t)(n + 1), st);
    cudaMemsetAsync(w.maxlev, 0, sizeof(int32_t), st);
    const int lb = ticket_blocks(ctx, (const void *)k_levels<LOWER>, n);
    k_levels<LOWER><<<lb, 256, 0, st>>>(n, A->d_row_ptr, A->d_col, diag, w.lev, w.maxlev, w.tickets,
                                        seq % kTickets, w.err);
    ++seq;
    k_level_count<<<vec_blocks(ctx, n), kVecThreads, 0, st>>>(n, w.lev, w.count);
    k_level_scan<<<1, 1024, 0, st>>>(w.maxlev, w.count);
    k_level_scatter<<<vec_blocks(ctx, n), kVecThreads, 0, st>>>(n, w.lev, w.count, order);
}

void sort_levels(mm_ctx *ctx, const mm_csr_pattern *A, const int64_t *diag, const KrylovWs &w, int &seq) {
    sort_by_level<true>(ctx, A, diag, w, seq, w.ordL);
    sort_by_level<false>(ctx, A, diag, w, seq, w.ordU);
}

}  // namespace

extern "C" int mm_implicit_assemble(mm_ctx *ctx, const mm_csr_pattern *stencils, const double *d_vals,
                                    const uint8_t *d_kind, int32_t *d_col_out, double *d_vals_out) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (int rc = bad_pattern(ctx, stencils)) return rc;
    if (!d_vals || !d_col_out || !d_vals_out)
        return mm_fail(ctx, MM_EBADARG, "values and outputs are required");
    DeviceGuard g(ctx);
    KrylovWs w{};
    if (int rc = krylov_ws(ctx, stencils->nrows, 1, 0, false, &w)) return rc;
    const int64_t n = stencils->nrows;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, (int64_t)ctx->num_sms * 16));
    k_assemble<<<blocks, 256, 0, ctx->stream>>>(n, stencils->d_row_ptr, stencils->d_col, d_vals, d_kind, d_col_out,
                                                d_vals_out, w.err);
    MM_LAUNCH_CHECK(ctx);
    return read_err(ctx, w.err, "mm_implicit_assemble");
}

extern "C" int mm_ilu0(mm_ctx *ctx, const mm_csr_pattern *A, const double *d_vals, double *d_factors,
                       int64_t *d_diag) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (int rc = bad_pattern(ctx, A)) return rc;
    if (!d_vals || !d_factors || !d_diag) return mm_fail(ctx, MM_EBADARG, "values, factors and diag are required");
    DeviceGuard g(ctx);
    KrylovWs w{};
    if (int rc = krylov_ws(ctx, A->nrows, 1, 0, true, &w)) return rc;
    if (d_factors != d_vals)
        MM_CUDA_CHECK(ctx, cudaMemcpyAsync(d_factors, d_vals, (size_t)A->nnz * sizeof(double),
                                           cudaMemcpyDeviceToDevice, ctx->stream));
    const int blocks = ticket_blocks(ctx, (const void *)k_ilu0, A->nrows);
    k_ilu0<<<blocks, 256, 0, ctx->stream>>>(A->nrows, A->d_row_ptr, A->d_col, d_factors, d_diag, w.flag, 1u,
                                            w.tickets, 0, w.err);
    MM_LAUNCH_CHECK(ctx);
    return read_err(ctx, w.err, "mm_ilu0");
}

extern "C" int mm_ilu0_solve(mm_ctx *ctx, const mm_csr_pattern *A, const double *d_factors,
                             const int64_t *d_diag, const double *d_b, double *d_x) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (int rc = bad_pattern(ctx, A)) return rc;
    if (!d_factors || !d_diag || !d_b || !d_x || d_b == d_x)
        return mm_fail(ctx, MM_EBADARG, "factors, diag, b and a distinct x are required");
    DeviceGuard g(ctx);
    KrylovWs w{};
    if (int rc = krylov_ws(ctx, A->nrows, 1, 1, false, &w, true)) return rc;
    double *Y = w.vec[0];
    fill_pending(ctx, Y, A->nrows);
    int seq = 0;
    sort_levels(ctx, A, d_diag, w, seq);
    const int lb = ticket_blocks(ctx, (const void *)k_lower<kRhsPlain>, A->nrows);
    const int ub = ticket_blocks(ctx, (const void *)k_upper, A->nrows);
    precond<kRhsPlain>(ctx, A, d_factors, d_diag, d_b, nullptr, nullptr, nullptr, nullptr, Y, d_x, w, seq, lb, ub);
    MM_LAUNCH_CHECK(ctx);
    return read_err(ctx, w.err, "mm_ilu0_solve");
}

extern "C" int mm_bicgstab(mm_ctx *ctx, const mm_csr_pattern *A, const double *d_vals,
                           const double *d_factors, const int64_t *d_diag, const double *d_b, double *d_x,
                           double tol, int maxit, int *iters, double *relres) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (int rc = bad_pattern(ctx, A)) return rc;
    if (!d_vals || !d_b || !d_x || (d_factors && !d_diag))
        return mm_fail(ctx, MM_EBADARG, "values, b and x (and diag with factors) are required");
    if (!(tol >= 0.0) || maxit < 0) return mm_fail(ctx, MM_EBADARG, "tol >= 0 and maxit >= 0 required");
    DeviceGuard g(ctx);
    const int64_t n = A->nrows;
    const int nb = vec_blocks(ctx, n);
    KrylovWs w{};
    if (int rc = krylov_ws(ctx, n, nb, 9, false, &w, d_factors != nullptr)) return rc;
    double *r = w.vec[0], *rh = w.vec[1], *p = w.vec[2], *v = w.vec[3], *ph = w.vec[4], *s = w.vec[5],
           *shv = w.vec[6], *t = w.vec[7], *Y = w.vec[8];
    const bool pre = d_factors != nullptr;
    if (!pre) { ph = p; shv = s; }
    KrylovScalars init{};
    init.tol = tol;
    init.maxit = maxit;
    MM_CUDA_CHECK(ctx, cudaMemcpyAsync(w.sc, &init, sizeof init, cudaMemcpyHostToDevice, ctx->stream));
    if (pre) fill_pending(ctx, Y, n);
    const int64_t *rp = A->d_row_ptr;
    const int32_t *col = A->d_col;
    cudaStream_t st = ctx->stream;
    k_spmv_dot<0><<<nb, kVecThreads, 0, st>>>(n, rp, col, d_vals, d_x, r, d_b, rh, p, v, w.sc, w.partials);
    k_scalars<kStart><<<1, kVecThreads, 0, st>>>(w.partials, nb, w.sc);
    MM_LAUNCH_CHECK(ctx);
    const int lb = pre ? ticket_blocks(ctx, (const void *)k_lower<kRhsP>, n) : 0;
    const int ub = pre ? ticket_blocks(ctx, (const void *)k_upper, n) : 0;
    int seq = 0;
    if (pre) sort_levels(ctx, A, d_diag, w, seq);
    constexpr int kCheck = 16;   // iterations enqueued between two looks at the scalars
    KrylovScalars h{};
    for (int done = 0; done < maxit; done += kCheck) {
        for (int j = 0; j < kCheck && done + j < maxit; ++j) {
            if (pre) precond<kRhsP>(ctx, A, d_factors, d_diag, nullptr, p, r, v, w.sc, Y, ph, w, seq, lb, ub);
            else k_axpy_rhs<kRhsP><<<nb, kVecThreads, 0, st>>>(n, p, r, v, w.sc);
            k_spmv_dot<1><<<nb, kVecThreads, 0, st>>>(n, rp, col, d_vals, ph, v, rh, nullptr, nullptr, nullptr,
                                                      w.sc, w.partials);
            k_scalars<kAlpha><<<1, kVecThreads, 0, st>>>(w.partials, nb, w.sc);
            if (pre) precond<kRhsS>(ctx, A, d_factors, d_diag, nullptr, s, r, v, w.sc, Y, shv, w, seq, lb, ub);
            else k_axpy_rhs<kRhsS><<<nb, kVecThreads, 0, st>>>(n, s, r, v, w.sc);
            k_spmv_dot<2><<<nb, kVecThreads, 0, st>>>(n, rp, col, d_vals, shv, t, s, nullptr, nullptr, nullptr,
                                                      w.sc, w.partials);
            k_scalars<kOmega><<<1, kVecThreads, 0, st>>>(w.partials, nb, w.sc);
            k_update<<<nb, kVecThreads, 0, st>>>(n, d_x, ph, shv, s, t, r, rh, w.sc, w.partials);
            k_scalars<kNext><<<1, kVecThreads, 0, st>>>(w.partials, nb, w.sc);
        }
        MM_LAUNCH_CHECK(ctx);
        MM_CUDA_CHECK(ctx, cudaMemcpyAsync(&h, w.sc, sizeof h, cudaMemcpyDeviceToHost, st));
        MM_CUDA_CHECK(ctx, cudaStreamSynchronize(st));
        if (h.stop) break;
    }
    if (maxit == 0 || !h.stop) {
        MM_CUDA_CHECK(ctx, cudaMemcpyAsync(&h, w.sc, sizeof h, cudaMemcpyDeviceToHost, st));
        MM_CUDA_CHECK(ctx, cudaStreamSynchronize(st));
    }
    if (int rc = read_err(ctx, w.err, "mm_bicgstab")) return rc;
    if (iters) *iters = h.it;
    if (relres) *relres = h.res;
    if (h.stop == 1) return MM_OK;
    return mm_fail(ctx, MM_ENOCONV, "BiCGSTAB stopped after %d iterations at relative residual %.3e (%s)", h.it,
                   h.res, h.stop == 2 ? "breakdown" : "iteration limit");
}
