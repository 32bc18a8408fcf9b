// Stencil selection: the n closest nodes of every query node (Section 2.1 of
// the paper: stencils of closest neighbours, each node first in its own).
//
// Ranking: ascending (squared distance, node index).  The squared distance is
// computed in FP64 exactly as sum_a (p_a - c_a)^2 in dimension order with
// round-to-nearest and no fused multiply-add (__dsub_rn/__dmul_rn/__dadd_rn),
// so any exact implementation of the same ranking gives bit-identical rows.
// Keys are compared as integers: for d2 >= 0 the IEEE bit pattern orders like
// the value, so the top list needs no FP64 compare.
//
// FP64 is scarce on this GPU, so everything that only has to be conservative
// runs in FP32 with an explicit error bound delta on FP32 distances (from the
// largest coordinate magnitude): cell pruning, the stop test, and a candidate
// filter that rejects a node when even its distance minus delta cannot beat
// the current n-th best.  Only candidates that pass get the exact FP64 key.
//
// Two search strategies, one warp per query, both exact:
//  * grid: nodes are counting-sorted into a uniform grid (cell edge chosen
//    from the mean density so a cell holds ~ppc nodes); the warp visits the
//    query's cell and then Chebyshev rings of cells around it, skipping cells
//    whose (slightly enlarged) box lies farther than the current n-th best,
//    and stops once the ring boundary is farther than the n-th best.
//  * brute: every node is a candidate (for small N).
// The top n-1 list lives in registers across the warp (two slots per lane,
// up to 64 entries) and is kept sorted by warp-wide insertion, or by a bitonic merge
// when a batch brings many new entries.
#include <float.h>
#include <math.h>

#include <algorithm>

#include "mm_internal.cuh"

namespace {

constexpr int kWarpsPerBlock = 8;
constexpr unsigned kFull = 0xffffffffu;

struct GridParams {
    double lo[3];
    double cell;
    double inv_cell;
    int dims[3];
    int ncells;
    float lo32[3];     // FP32 copies for the conservative tests
    float cell32;
    float inv_cell32;  // FP32 1/cell: ring centre of a query (any cell is a valid centre)
    float delta32;     // bound on |FP32 distance - exact distance| for any two nodes
};

// ------------------------------------------------------------------ binning
template <int DIM>
__global__ void k_bbox_partial(const double *__restrict__ pts, int64_t N, double *partial) {
    double mn[DIM], mx[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) { mn[a] = DBL_MAX; mx[a] = -DBL_MAX; }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            double v = pts[i * DIM + a];
            mn[a] = fmin(mn[a], v);
            mx[a] = fmax(mx[a], v);
        }
    }
    __shared__ double smn[DIM][32], smx[DIM][32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        for (int o = 16; o; o >>= 1) {
            mn[a] = fmin(mn[a], __shfl_xor_sync(kFull, mn[a], o));
            mx[a] = fmax(mx[a], __shfl_xor_sync(kFull, mx[a], o));
        }
        if (lane == 0) { smn[a][w] = mn[a]; smx[a][w] = mx[a]; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = blockDim.x >> 5;
        for (int a = 0; a < DIM; ++a) {
            double a0 = smn[a][0], a1 = smx[a][0];
            for (int j = 1; j < nw; ++j) { a0 = fmin(a0, smn[a][j]); a1 = fmax(a1, smx[a][j]); }
            partial[blockIdx.x * 2 * DIM + a] = a0;
            partial[blockIdx.x * 2 * DIM + DIM + a] = a1;
        }
    }
}

// One block: reduce the block partials (every thread a stride of them, then
// the warps, then the first warp), then one thread chooses the cell edge so a
// cell holds about `ppc` nodes on average and caps the cell count at `cap`.
template <int DIM>
__global__ void k_grid_params(const double *partial, int nparts, int64_t N, double ppc,
                              int64_t cap, GridParams *gp) {
    __shared__ double s_lo[DIM][32], s_hi[DIM][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double lo[DIM], hi[DIM], ext[DIM], emax = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        lo[a] = DBL_MAX; hi[a] = -DBL_MAX;
        for (int j = threadIdx.x; j < nparts; j += blockDim.x) {
            lo[a] = fmin(lo[a], partial[j * 2 * DIM + a]);
            hi[a] = fmax(hi[a], partial[j * 2 * DIM + DIM + a]);
        }
        for (int o = 16; o; o >>= 1) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(kFull, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(kFull, hi[a], o));
        }
        if (lane == 0) { s_lo[a][w] = lo[a]; s_hi[a][w] = hi[a]; }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int a = 0; a < DIM; ++a) {
        lo[a] = s_lo[a][0]; hi[a] = s_hi[a][0];
        for (int j = 1; j < nw; ++j) { lo[a] = fmin(lo[a], s_lo[a][j]); hi[a] = fmax(hi[a], s_hi[a][j]); }
        ext[a] = hi[a] - lo[a];
        emax = fmax(emax, ext[a]);
    }
    if (!(emax > 0)) emax = 1.0;
    double vol = 1.0;
    for (int a = 0; a < DIM; ++a) {
        ext[a] = fmax(ext[a], 1e-9 * emax);
        vol *= ext[a];
    }
    double cells_target = fmax(1.0, (double)N / ppc);
    double c = pow(vol / cells_target, 1.0 / DIM);
    int dims[DIM];
    for (int it = 0; it < 64; ++it) {
        double prod = 1.0;
        for (int a = 0; a < DIM; ++a) {
            double d = ceil(ext[a] / c);
            if (d < 1) d = 1;
            if (d > 1 << 20) d = 1 << 20;
            dims[a] = (int)d;
            prod *= d;
        }
        if (prod <= (double)cap) break;
        c *= pow(prod / (double)cap, 1.0 / DIM) * 1.01;
    }
    // Grid origin slightly below the box so no node sits on the low face.
    for (int a = 0; a < 3; ++a) {
        gp->lo[a] = a < DIM ? lo[a] - 1e-7 * c : 0.0;
        gp->dims[a] = a < DIM ? dims[a] : 1;
    }
    gp->cell = c;
    gp->inv_cell = 1.0 / c;
    double amax = 0.0;
    for (int a = 0; a < DIM; ++a) amax = fmax(amax, fmax(fabs(lo[a]), fabs(hi[a])));
    for (int a = 0; a < 3; ++a) gp->lo32[a] = (float)gp->lo[a];
    gp->cell32 = (float)c;
    gp->inv_cell32 = (float)(1.0 / c);
    // each coordinate rounds by <= u32*amax, the difference by <= 2*u32*amax,
    // the FP32 square, sum and root by a few u32 of the distance (<= 2*amax*sqrt(d))
    gp->delta32 = (float)(16.0 * (FLT_EPSILON * 0.5) * amax * sqrt((double)DIM)) + 1e-30f;
    long long nc = 1;
    for (int a = 0; a < DIM; ++a) nc *= dims[a];
    gp->ncells = (int)nc;
}

template <int DIM>
__device__ __forceinline__ int cell_coord(double x, int a, const GridParams &g) {
    int i = (int)floor((x - g.lo[a]) * g.inv_cell);
    return min(max(i, 0), g.dims[a] - 1);
}

template <int DIM>
__global__ void k_cell_count(const double *__restrict__ pts, int64_t N, const GridParams *gp,
                             int *cell_of, int *rank, int *count) {
    GridParams g = *gp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int cid = 0;
#pragma unroll
        for (int a = DIM - 1; a >= 0; --a) cid = cid * g.dims[a] + cell_coord<DIM>(pts[i * DIM + a], a, g);
        cell_of[i] = cid;
        rank[i] = atomicAdd(&count[cid], 1);
    }
}

// Exclusive scan of count[0..n) into start[0..n] in three passes.
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ int block_exclusive_scan(int v, int *sh, int *total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < (blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    int base = w > 0 ? sh[w - 1] : 0;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void k_scan_tiles(const int *count, const GridParams *gp, int *start, int *tile_sum) {
    __shared__ int sh[32];
    int n = gp->ncells;
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems], s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = base + j < n ? count[base + j] : 0;
        s += v[j];
    }
    int total;
    int ex = block_exclusive_scan(s, sh, &total);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) start[base + j] = ex;
        ex += v[j];
    }
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void k_scan_sums(int *tile_sum, int ntiles, const GridParams *gp, int *start) {
    __shared__ int sh[32];
    int carry = 0;
    for (int b = 0; b < ntiles; b += blockDim.x) {
        int v = b + threadIdx.x < ntiles ? tile_sum[b + threadIdx.x] : 0;
        int total;
        int ex = block_exclusive_scan(v, sh, &total);
        if (b + threadIdx.x < ntiles) tile_sum[b + threadIdx.x] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) start[gp->ncells] = carry;
}

__global__ void k_scan_add(const int *tile_sum, const GridParams *gp, int *start) {
    int n = gp->ncells;
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int add = tile_sum[blockIdx.x];
    for (int j = threadIdx.x; j < kScanTile; j += blockDim.x)
        if (base + j < n) start[base + j] += add;
}

template <int DIM>
__global__ void k_scatter(const double *__restrict__ pts, int64_t N, const int *cell_of,
                          const int *rank, const int *start, double *spts, float *spts32,
                          int *sidx, float *pts32) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int d = start[cell_of[i]] + rank[i];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const double v = pts[i * DIM + a];
            spts[(int64_t)d * DIM + a] = v;
            spts32[(int64_t)d * DIM + a] = (float)v;
            pts32[i * DIM + a] = (float)v;
        }
        sidx[d] = (int)i;
    }
}

template <int DIM>
__global__ void k_to_fp32(const double *__restrict__ pts, int64_t N, float *pts32) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N * DIM;
         i += (int64_t)gridDim.x * blockDim.x)
        pts32[i] = (float)pts[i];
}

// Delta for the brute-force search (no grid): from the largest coordinate.
template <int DIM>
__global__ void k_brute_delta(const double *partial, int nparts, float *delta) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double amax = 0.0;
    for (int j = 0; j < nparts * 2 * DIM; ++j) amax = fmax(amax, fabs(partial[j]));
    *delta = (float)(16.0 * (FLT_EPSILON * 0.5) * amax * sqrt((double)DIM)) + 1e-30f;
}

// ------------------------------------------------------------- the top list
typedef unsigned long long u64;
constexpr u64 kInfBits = 0x7ff0000000000000ULL;    // +inf: empty slot

__device__ __forceinline__ bool key_lt(u64 da, int ia, u64 db, int ib) {
    return da < db || (da == db && ia < ib);
}

// Sorted list of the K best (d2 bits, index) keys; slot s on lane s (lo) and
// on lane s-32 (hi).  Empty slots hold (+inf, INT_MAX).
struct TopList {
    u64 dlo, dhi;
    int ilo, ihi;
    int K;

    __device__ void init(int k) {
        K = k;
        dlo = dhi = kInfBits;
        ilo = ihi = 0x7fffffff;
    }
    // Key of slot K-1 (the worst kept), broadcast to all lanes.
    __device__ void worst(u64 &d, int &i) const {
        if (K == 0) { d = 0; i = -1; return; }
        const int s = K - 1, src = s & 31;
        const u64 dv = s < 32 ? dlo : dhi;
        const int iv = s < 32 ? ilo : ihi;
        d = __shfl_sync(kFull, dv, src);
        i = __shfl_sync(kFull, iv, src);
    }
    // Insert a warp-uniform key known to be better than the worst.  With K
    // <= 32 the second slots are never used (warp-uniform branch).
    __device__ void insert(u64 d, int idx) {
        const int lane = threadIdx.x & 31;
        const unsigned blo = __ballot_sync(kFull, key_lt(dlo, ilo, d, idx));
        int pos = __popc(blo);
        const u64 pdlo = __shfl_up_sync(kFull, dlo, 1);
        const int pilo = __shfl_up_sync(kFull, ilo, 1);
        if (K > 32) {
            const unsigned bhi = __ballot_sync(kFull, key_lt(dhi, ihi, d, idx));
            pos += __popc(bhi);
            u64 pdhi = __shfl_up_sync(kFull, dhi, 1);
            int pihi = __shfl_up_sync(kFull, ihi, 1);
            const u64 d31 = __shfl_sync(kFull, dlo, 31);
            const int i31 = __shfl_sync(kFull, ilo, 31);
            if (lane == 0) { pdhi = d31; pihi = i31; }
            const int shi = lane + 32;
            if (shi > pos) { dhi = pdhi; ihi = pihi; }
            if (shi == pos) { dhi = d; ihi = idx; }
        }
        const int slo = lane;
        if (slo > pos) { dlo = pdlo; ilo = pilo; }
        if (slo == pos) { dlo = d; ilo = idx; }
    }
};

// One compare-exchange stage over the warp for sorted order of (key, index)
// pairs: lane and lane ^ j exchange so that the lane with the lower position
// in the pair's direction keeps the smaller pair (`up`: this lane's pair
// sorts ascending).
__device__ __forceinline__ void cmpx(u64 &k, int &i, int j, bool up) {
    const int lane = threadIdx.x & 31;
    const u64 ok = __shfl_xor_sync(kFull, k, j);
    const int oi = __shfl_xor_sync(kFull, i, j);
    const bool lower = (lane & j) == 0;
    const bool other_smaller = key_lt(ok, oi, k, i);
    // keep the smaller one if (lower == up), else the larger one
    if ((lower == up) == other_smaller) { k = ok; i = oi; }
}

// Bitonic sort of 32 pairs (one per lane) into ascending lane order.
__device__ __forceinline__ void sort32(u64 &k, int &i) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int w = 2; w <= 32; w <<= 1)
#pragma unroll
        for (int j = w >> 1; j; j >>= 1) cmpx(k, i, j, (lane & w) == 0 || w == 32);
}
// A bitonic sequence of 32 pairs into ascending lane order.
__device__ __forceinline__ void bitonic32(u64 &k, int &i) {
#pragma unroll
    for (int j = 16; j; j >>= 1) cmpx(k, i, j, true);
}

// Merge of up to 32 new pairs (one per lane, +inf for none) into a list of
// K <= 32 slots held one per lane in ascending order: bitonic sort of the new
// pairs, the elementwise smaller of the list and the reversed new pairs (the
// 32 smallest of both, as a bitonic sequence), bitonic merge.  ~21 exchange
// stages, whatever the number of new pairs.
__device__ __forceinline__ void merge_batch(TopList &tl, u64 k, int i) {
    const int lane = threadIdx.x & 31;
    sort32(k, i);
    const u64 rk = __shfl_sync(kFull, k, 31 - lane);
    const int ri = __shfl_sync(kFull, i, 31 - lane);
    if (key_lt(rk, ri, tl.dlo, tl.ilo)) { tl.dlo = rk; tl.ilo = ri; }
    bitonic32(tl.dlo, tl.ilo);
}

// The same for a list of 33 <= K <= 64 slots (lo: slots 0..31, hi: 32..63).
// With the new pairs B sorted and reversed, min(lo, B) are the 32 smallest of
// lo and B, all no larger than any hi slot (lo alone has 32 such), so they
// are the new lo; max(lo, B), the 32 largest of lo and B, merge with hi the
// same way for the new hi.  ~32 exchange stages.
__device__ __forceinline__ void merge_batch2(TopList &tl, u64 k, int i) {
    const int lane = threadIdx.x & 31;
    sort32(k, i);
    const u64 rk = __shfl_sync(kFull, k, 31 - lane);
    const int ri = __shfl_sync(kFull, i, 31 - lane);
    u64 yk = rk;
    int yi = ri;
    if (key_lt(rk, ri, tl.dlo, tl.ilo)) {
        yk = tl.dlo;
        yi = tl.ilo;
        tl.dlo = rk;
        tl.ilo = ri;
    }
    bitonic32(tl.dlo, tl.ilo);
    bitonic32(yk, yi);
    const u64 zk = __shfl_sync(kFull, yk, 31 - lane);
    const int zi = __shfl_sync(kFull, yi, 31 - lane);
    if (key_lt(zk, zi, tl.dhi, tl.ihi)) { tl.dhi = zk; tl.ihi = zi; }
    bitonic32(tl.dhi, tl.ihi);
}

template <int DIM>
__device__ __forceinline__ double dist2_rn(const double *p, const double *c) {
    double t = __dsub_rn(p[0], c[0]);
    double s = __dmul_rn(t, t);
#pragma unroll
    for (int a = 1; a < DIM; ++a) {
        double u = __dsub_rn(p[a], c[a]);
        s = __dadd_rn(s, __dmul_rn(u, u));
    }
    return s;
}

// Worst key as an FP32 upper bound of its squared distance (inf while the list
// is not full).
__device__ __forceinline__ float worst_f32(u64 wd) {
    return __double2float_ru(__longlong_as_double((long long)wd));
}

// One chunk of candidates (one per lane, `valid` lanes only): reject by the
// FP32 lower bound, compute exact keys for the rest, insert the ones that beat
// the current worst.  x32/c32: FP32 coordinates; pexact: FP64 coordinates of
// the candidate (read only if it passes).
template <int DIM>
__device__ __forceinline__ void consider(TopList &tl, bool valid, const float *x32, const float *c32,
                                         const double *pexact, const double *c, int idx,
                                         float delta, u64 &wd, int &wi, bool &dup) {
    bool pass = false;
    if (valid) {
        float d2f = 0.0f;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const float t = x32[a] - c32[a];
            d2f = fmaf(t, t, d2f);
        }
        const float lo = fmaxf(sqrtf(d2f) - delta, 0.0f);
        pass = lo * lo <= worst_f32(wd) * 1.000001f;
    }
    u64 key = kInfBits;
    if (__any_sync(kFull, pass) && pass) {
        const double d2 = dist2_rn<DIM>(pexact, c);
        key = (u64)__double_as_longlong(d2);
        if (d2 == 0.0) dup = true;
    }
    unsigned m = __ballot_sync(kFull, pass && key_lt(key, idx, wd, wi));
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const u64 ck = __shfl_sync(kFull, key, src);
        const int ci = __shfl_sync(kFull, idx, src);
        if (key_lt(ck, ci, wd, wi)) {
            tl.insert(ck, ci);
            tl.worst(wd, wi);
        }
    }
}

__device__ __forceinline__ void write_row(const TopList &tl, int64_t q, int n, int32_t *out_row,
                                          int32_t *status, bool dup) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) out_row[0] = (int32_t)q;
    const int K = n - 1;
    bool full = true;
    if (lane < K) {
        out_row[1 + lane] = tl.ilo == 0x7fffffff ? -1 : tl.ilo;
        full &= tl.ilo != 0x7fffffff;
    }
    if (lane + 32 < K) {
        out_row[33 + lane] = tl.ihi == 0x7fffffff ? -1 : tl.ihi;
        full &= tl.ihi != 0x7fffffff;
    }
    full = __all_sync(kFull, full);
    if (status && lane == 0) status[q] = dup ? MM_ST_DUPLICATE : (full ? MM_ST_OK : MM_ST_BADARG);
}

// ---------------------------------------------------------- grid ring search
// Candidates that pass the FP32 filter wait in a per-warp queue in shared
// memory and get their exact FP64 keys 32 at a time, so FP64 instructions
// (1/64 of the FP32 rate on this GPU, and issued for the whole warp however
// few lanes need them) run on full batches; the queue is also flushed at the
// end of every ring, before the stop test.  While candidates wait, the list's
// worst key is older (larger) than it would be, which only lets more
// candidates through the conservative tests; the final list is the same,
// because the ranking is a total order and every candidate that can enter it
// passes.
constexpr int kQueue = 64;

// (2D: 64 registers, no spills, four blocks of eight warps per SM; 3D: three)
template <int DIM>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, DIM == 2 ? 4 : 3)
k_knn_grid(const double *__restrict__ pts, const float *__restrict__ pts32, const GridParams *gp,
           const int *__restrict__ start, const double *__restrict__ spts, const float *__restrict__ spts32,
           const int *__restrict__ sidx, int64_t q_begin, int64_t q_end, int n,
           int32_t *__restrict__ out, int32_t *status) {
    __shared__ int s_sp[kWarpsPerBlock][kQueue];
    __shared__ int s_idx[kWarpsPerBlock][kQueue];
    const GridParams g = *gp;
    const int lane = threadIdx.x & 31;
    int *qsp = s_sp[threadIdx.x >> 5];
    int *qidx = s_idx[threadIdx.x >> 5];
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float delta = g.delta32;
    const float slack = 2.0f * delta + 1e-6f * g.cell32;
    int maxdim = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) maxdim = max(maxdim, g.dims[a]);
    for (int64_t q = q_begin + warp0; q < q_end; q += nwarps) {
        double c[DIM];
        float c32[DIM];
        int cq[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            c[a] = pts[q * DIM + a];
            c32[a] = pts32[q * DIM + a];
            // ring centre: the query's cell up to FP32 rounding (any cell is
            // a valid centre: the rings, the pruning and the stop test use
            // the query's own coordinates)
            const int i = __float2int_rd((c32[a] - g.lo32[a]) * g.inv_cell32);
            cq[a] = min(max(i, 0), g.dims[a] - 1);
        }
        TopList tl;
        tl.init(n - 1);
        u64 wd;
        int wi;
        tl.worst(wd, wi);
        // FP32 upper bound of the worst kept squared distance, and the
        // squared FP32 distance a candidate must not exceed to possibly beat
        // it (sqrt(d2f) - delta <= sqrt(worst), with a relative margin)
        float wf = 0.0f, thr = 0.0f;
        auto bounds = [&]() {
            wf = worst_f32(wd);
            const float r = sqrtf(wf * 1.000001f) + delta;
            thr = r * r * 1.00001f;
        };
        bounds();
        bool dup = false;
        int qn = 0;
        // exact keys of the first `cnt` queued candidates, insertion of those
        // that beat the worst kept
        auto flush = [&](int cnt) {
            const bool v = lane < cnt;
            const int sp = v ? qsp[lane] : 0;
            const int idx = v ? qidx[lane] : -1;
            u64 key = kInfBits;
            if (v) {
                const double d2 = dist2_rn<DIM>(spts + (int64_t)sp * DIM, c);
                key = (u64)__double_as_longlong(d2);
                if (d2 == 0.0) dup = true;
            }
            const bool better = v && key_lt(key, idx, wd, wi);
            unsigned m = __ballot_sync(kFull, better);
            if (tl.K <= 32 && __popc(m) >= 6) {
                // many new entries: one bitonic merge instead of one insertion each
                merge_batch(tl, better ? key : kInfBits, better ? idx : 0x7fffffff);
                tl.worst(wd, wi);
                m = 0;
            } else if (tl.K > 32 && __popc(m) >= 8) {
                merge_batch2(tl, better ? key : kInfBits, better ? idx : 0x7fffffff);
                tl.worst(wd, wi);
                m = 0;
            }
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1;
                const u64 ck = __shfl_sync(kFull, key, src);
                const int ci = __shfl_sync(kFull, idx, src);
                if (key_lt(ck, ci, wd, wi)) {
                    tl.insert(ck, ci);
                    tl.worst(wd, wi);
                }
            }
            bounds();
        };
        for (int t = 0; t <= maxdim; ++t) {
            const int side = 2 * t + 1;
            int ncube = side;
#pragma unroll
            for (int a = 1; a < DIM; ++a) ncube *= side;
            for (int u0 = 0; u0 < ncube; u0 += 32) {
                const int u = u0 + lane;
                int cstart = 0, ccount = 0;
                if (u < ncube) {
                    int off[DIM], rem = u, cheb = 0;
                    bool inside = true;
                    int cid = 0;
#pragma unroll
                    for (int a = 0; a < DIM; ++a) {
                        off[a] = rem % side - t;
                        rem /= side;
                        cheb = max(cheb, abs(off[a]));
                    }
                    float md2 = 0.0f;
#pragma unroll
                    for (int a = DIM - 1; a >= 0; --a) {
                        const int ca = cq[a] + off[a];
                        inside &= (ca >= 0 && ca < g.dims[a]);
                        cid = cid * g.dims[a] + ca;
                        const float blo = fmaf((float)ca, g.cell32, g.lo32[a]) - slack;
                        const float bhi = fmaf((float)(ca + 1), g.cell32, g.lo32[a]) + slack;
                        const float gap = fmaxf(0.0f, fmaxf(blo - c32[a], c32[a] - bhi));
                        md2 = fmaf(gap, gap, md2);
                    }
                    if (inside && cheb == t && !(md2 * 0.99999f > wf)) {
                        cstart = start[cid];
                        ccount = start[cid + 1] - cstart;
                    }
                }
                // inclusive scan of counts over the warp
                int incl = ccount;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                const int total = __shfl_sync(kFull, incl, 31);
                for (int p0 = 0; p0 < total; p0 += 32) {
                    const int p = p0 + lane;
                    int owner = 0;
#pragma unroll
                    for (int step = 16; step; step >>= 1) {
                        const int probe = __shfl_sync(kFull, incl, owner + step - 1);
                        if (probe <= p) owner += step;
                    }
                    const int os = __shfl_sync(kFull, cstart, owner);
                    const int oi = __shfl_sync(kFull, incl, owner);
                    const int oc = __shfl_sync(kFull, ccount, owner);
                    bool pass = false;
                    int sp = 0, idx = -1;
                    if (p < total) {
                        sp = os + (p - (oi - oc));
                        idx = sidx[sp];
                        float d2f = 0.0f;
#pragma unroll
                        for (int a = 0; a < DIM; ++a) {
                            const float tt = spts32[(int64_t)sp * DIM + a] - c32[a];
                            d2f = fmaf(tt, tt, d2f);
                        }
                        pass = idx != (int)q && d2f <= thr;
                    }
                    const unsigned pm = __ballot_sync(kFull, pass);
                    if (pm) {
                        const int at = qn + __popc(pm & lt_mask);
                        if (pass) {
                            qsp[at] = sp;
                            qidx[at] = idx;
                        }
                        qn += __popc(pm);
                        __syncwarp();
                        if (qn >= 32) {
                            flush(32);
                            __syncwarp();
                            if (lane < qn - 32) {
                                qsp[lane] = qsp[32 + lane];
                                qidx[lane] = qidx[32 + lane];
                            }
                            qn -= 32;
                            __syncwarp();
                        }
                    }
                }
            }
            if (qn > 0) {
                flush(qn);
                qn = 0;
                __syncwarp();
            }
            // stop once every unvisited cell is provably farther than the worst kept
            bool covers = true;
            float bd = 3.0e38f;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const bool lo_edge = cq[a] - t <= 0, hi_edge = cq[a] + t >= g.dims[a] - 1;
                covers &= lo_edge && hi_edge;
                if (!lo_edge) bd = fminf(bd, c32[a] - fmaf((float)(cq[a] - t), g.cell32, g.lo32[a]));
                if (!hi_edge) bd = fminf(bd, fmaf((float)(cq[a] + t + 1), g.cell32, g.lo32[a]) - c32[a]);
            }
            if (covers) break;
            bd = fmaxf(bd - slack, 0.0f);
            if (bd * bd * 0.99999f > wf) break;
        }
        dup = __any_sync(kFull, dup);
        write_row(tl, q, n, out + (q - q_begin) * n, status, dup);
    }
}

// ----------------------------------------------------------------- brute force
template <int DIM>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_knn_brute(const double *__restrict__ pts, const float *__restrict__ pts32, const float *dptr,
            int64_t N, int64_t q_begin, int64_t q_end, int n, int32_t *__restrict__ out,
            int32_t *status) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float delta = *dptr;
    for (int64_t q = q_begin + warp0; q < q_end; q += nwarps) {
        double c[DIM];
        float c32[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            c[a] = pts[q * DIM + a];
            c32[a] = (float)c[a];
        }
        TopList tl;
        tl.init(n - 1);
        u64 wd;
        int wi;
        tl.worst(wd, wi);
        bool dup = false;
        for (int64_t j0 = 0; j0 < N; j0 += 32) {
            const int64_t j = j0 + lane;
            const bool valid = j < N && j != q;
            const int64_t jj = j < N ? j : 0;
            float x32[DIM];
#pragma unroll
            for (int a = 0; a < DIM; ++a) x32[a] = pts32[jj * DIM + a];
            consider<DIM>(tl, valid, x32, c32, pts + jj * DIM, c, (int)j, delta, wd, wi, dup);
        }
        dup = __any_sync(kFull, dup);
        write_row(tl, q, n, out + (q - q_begin) * n, status, dup);
    }
}

template <int DIM>
int knn_impl(mm_ctx *ctx, int64_t N, const double *d_pts, int nranges, const mm_knn_range *ranges,
             int method, int32_t *d_status) {
    int nmax = 0;
    for (int r = 0; r < nranges; ++r) nmax = max(nmax, (int)ranges[r].n);
    cudaStream_t st = ctx->stream;
    const int qblocks = ctx->num_sms * 16;
    if (method == MM_KNN_AUTO) method = N <= 4096 ? MM_KNN_BRUTE : MM_KNN_GRID;
    const int bb_blocks = std::min(ctx->num_sms * 2, (int)((N + 255) / 256) + 1);
    const int eb = (int)std::min<int64_t>((N + 255) / 256, (int64_t)ctx->num_sms * 8);
    if (method == MM_KNN_BRUTE) {
        WsCarve wc;
        const size_t o_part = wc.take<double>((size_t)bb_blocks * 2 * DIM);
        const size_t o_delta = wc.take<float>(1);
        const size_t o_p32 = wc.take<float>((size_t)N * DIM);
        char *ws = mm_workspace(ctx, wc.off);
        if (!ws) return mm_fail(ctx, MM_ENOMEM, "knn workspace of %zu bytes", wc.off);
        double *part = (double *)(ws + o_part);
        float *delta = (float *)(ws + o_delta);
        float *p32 = (float *)(ws + o_p32);
        k_bbox_partial<DIM><<<bb_blocks, 256, 0, st>>>(d_pts, N, part);
        k_brute_delta<DIM><<<1, 32, 0, st>>>(part, bb_blocks, delta);
        k_to_fp32<DIM><<<eb, 256, 0, st>>>(d_pts, N, p32);
        MM_LAUNCH_CHECK(ctx);
        for (int r = 0; r < nranges; ++r) {
            const mm_knn_range &R = ranges[r];
            if (R.q_end <= R.q_begin) continue;
            const int64_t warps = R.q_end - R.q_begin;
            const int blocks = (int)std::min<int64_t>((warps + kWarpsPerBlock - 1) / kWarpsPerBlock, qblocks);
            k_knn_brute<DIM><<<blocks, kWarpsPerBlock * 32, 0, st>>>(d_pts, p32, delta, N, R.q_begin,
                                                                     R.q_end, R.n, R.d_idx, d_status);
            MM_LAUNCH_CHECK(ctx);
        }
        return MM_OK;
    }
    // ---- grid build
    const double ppc = fmax(2.0, nmax / double(1 << DIM));
    const int64_t cap = (int64_t)(4.0 * N / ppc) + 64;
    const int ntiles = (int)((cap + kScanTile - 1) / kScanTile);
    WsCarve wc;
    const size_t o_part = wc.take<double>((size_t)bb_blocks * 2 * DIM);
    const size_t o_gp = wc.take<GridParams>(1);
    const size_t o_count = wc.take<int>((size_t)cap + 1);
    const size_t o_start = wc.take<int>((size_t)cap + 1);
    const size_t o_cellof = wc.take<int>((size_t)N);
    const size_t o_rank = wc.take<int>((size_t)N);
    const size_t o_spts = wc.take<double>((size_t)N * DIM);
    const size_t o_spts32 = wc.take<float>((size_t)N * DIM);
    const size_t o_sidx = wc.take<int>((size_t)N);
    const size_t o_pts32 = wc.take<float>((size_t)N * DIM);
    const size_t o_tiles = wc.take<int>((size_t)ntiles + 1);
    char *ws = mm_workspace(ctx, wc.off);
    if (!ws) return mm_fail(ctx, MM_ENOMEM, "knn workspace of %zu bytes", wc.off);
    double *part = (double *)(ws + o_part);
    GridParams *gp = (GridParams *)(ws + o_gp);
    int *count = (int *)(ws + o_count), *start = (int *)(ws + o_start);
    int *cellof = (int *)(ws + o_cellof), *rank = (int *)(ws + o_rank);
    double *spts = (double *)(ws + o_spts);
    float *spts32 = (float *)(ws + o_spts32);
    int *sidx = (int *)(ws + o_sidx), *tiles = (int *)(ws + o_tiles);
    float *pts32 = (float *)(ws + o_pts32);
    k_bbox_partial<DIM><<<bb_blocks, 256, 0, st>>>(d_pts, N, part);
    k_grid_params<DIM><<<1, 256, 0, st>>>(part, bb_blocks, N, ppc, cap, gp);
    MM_CUDA_CHECK(ctx, cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(cap + 1), st));
    k_cell_count<DIM><<<eb, 256, 0, st>>>(d_pts, N, gp, cellof, rank, count);
    k_scan_tiles<<<ntiles, kScanThreads, 0, st>>>(count, gp, start, tiles);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(tiles, ntiles, gp, start);
    k_scan_add<<<ntiles, kScanThreads, 0, st>>>(tiles, gp, start);
    k_scatter<DIM><<<eb, 256, 0, st>>>(d_pts, N, cellof, rank, start, spts, spts32, sidx, pts32);
    MM_LAUNCH_CHECK(ctx);
    for (int r = 0; r < nranges; ++r) {
        const mm_knn_range &R = ranges[r];
        if (R.q_end <= R.q_begin) continue;
        const int64_t warps = R.q_end - R.q_begin;
        const int blocks = (int)std::min<int64_t>((warps + kWarpsPerBlock - 1) / kWarpsPerBlock, qblocks);
        k_knn_grid<DIM><<<blocks, kWarpsPerBlock * 32, 0, st>>>(d_pts, pts32, gp, start, spts, spts32,
                                                                sidx, R.q_begin, R.q_end, R.n, R.d_idx,
                                                                d_status);
        MM_LAUNCH_CHECK(ctx);
    }
    return MM_OK;
}

}  // namespace

int knn_launch(mm_ctx *ctx, int dim, int64_t N, const double *d_pts, int nranges,
               const mm_knn_range *ranges, int method, int32_t *d_status) {
    if (dim == 2) return knn_impl<2>(ctx, N, d_pts, nranges, ranges, method, d_status);
    return knn_impl<3>(ctx, N, d_pts, nranges, ranges, method, d_status);
}
