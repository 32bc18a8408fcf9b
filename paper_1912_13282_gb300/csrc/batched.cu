// Persistent batched weights: all stencil classes of a call in one launch.
//
// The class descriptors travel by value in a __grid_constant__ kernel
// parameter (no host memory is read when a captured graph replays).  Work
// items are chunks of consecutive rows of one class; warps take them from an
// atomic counter until the counter passes the total, so the loop is bounded
// by the number of items.  The FP32 + FP64-refinement variant hands rows it
// cannot finish to a second launch, the FP64 solver, through a queue of
// (class, row) pairs.
//
// Classes need different amounts of shared memory per stencil.  A CTA gets
// room for W stencils of the smallest class (at least one of the largest);
// classes are grouped into phases by how many stencils of them fit at once,
// and in each phase only that many warps of the CTA take work (from the
// phase's own counter), each with a slot of the CTA's memory divided by that
// number.  CTAs move from phase to phase on their own (a CTA barrier between
// phases, no inter-CTA waiting).
//
// The autotuner times launch shapes on a sample of each class and keeps the
// fastest per batch signature in the context (saved/loaded as a text table).
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "rbffd_dev.cuh"

namespace {

constexpr int kMaxBatchClasses = 96;
typedef unsigned long long u64;

struct BatchParams {
    WParams cls[kMaxBatchClasses];          // in phase order
    int64_t prefix[kMaxBatchClasses + 1];   // first work item of each class
    signed char variant[kMaxBatchClasses];  // mixed-kernel shape per class
    int nclasses;
    int nphases;
    int phase_end[kMaxBatchClasses];        // one past the last class of each phase
    int phase_warps[kMaxBatchClasses];      // warps of a CTA working in the phase
    int phase_slot[kMaxBatchClasses];       // shared-memory bytes per working warp
    int chunk_rows;
    int64_t total_items;
    int *queue;                             // [nphases] work counters
    u64 *fb_list;                           // (class << 32) | row
    int *fb_count;
    int fb_slot;                            // FP64 slot bytes of the fallback launch
};

static_assert(sizeof(BatchParams) <= 32000, "batched kernel parameters exceed the 32 KB limit");

// Variant of a class for the mixed kernel: (dim, rows per lane, column count)
// with the shared-memory inverse (0..11), or (dim, register width, column
// count) with the register-resident inverse (12..19), which the per-class
// launch also takes for systems of 33..48 unknowns padded to 40 or 48
// columns.  Both inverses give the same bits.  Classes with 2..4 operators
// run on the 4-column solver (the unused columns carry a zero right-hand
// side and are not stored).
__host__ __device__ inline int mixed_cols(int R) { return R == 1 ? 1 : 4; }
__host__ __device__ inline int mixed_variant(int dim, int rpl, int R, int wreg) {
    const int rsel = R == 1 ? 0 : 1;
    if (wreg) return 12 + ((dim - 2) * 2 + (wreg == 48 ? 1 : 0)) * 2 + rsel;
    return ((dim - 2) * 3 + (rpl - 1)) * 2 + rsel;
}

template <int DIM, int RPL, int W = 0>
__device__ bool mixed_dispatch_r(int rsel, const WParams &P, int64_t row, char *base) {
    if (rsel == 0) return mixed_row<DIM, RPL, 1, W>(P, row, base);
    return mixed_row<DIM, RPL, 4, W>(P, row, base);
}

template <int DIM>
__device__ bool mixed_dispatch_d(int v, const WParams &P, int64_t row, char *base) {
    const int rsel = v % 2;
    if (v >= 12) {
        if (((v - 12) >> 1) & 1) return mixed_dispatch_r<DIM, 2, 48>(rsel, P, row, base);
        return mixed_dispatch_r<DIM, 2, 40>(rsel, P, row, base);
    }
    const int rpl = (v / 2) % 3 + 1;
    if (rpl == 1) return mixed_dispatch_r<DIM, 1>(rsel, P, row, base);
    if (rpl == 2) return mixed_dispatch_r<DIM, 2>(rsel, P, row, base);
    return mixed_dispatch_r<DIM, 3>(rsel, P, row, base);
}

__device__ int class_of(const BatchParams &B, int64_t item, int cb, int ce) {
    int lo = cb, hi = ce - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.prefix[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <bool MIXED>
__device__ __forceinline__ void batched_body(const BatchParams &B) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int cb = 0;
    for (int p = 0; p < B.nphases; ++p) {
        const int ce = B.phase_end[p];
        if (wib < B.phase_warps[p]) {
            char *base = (char *)smem + (size_t)wib * B.phase_slot[p];
            const int64_t ib = B.prefix[cb], ie = B.prefix[ce];
            for (;;) {
                long long item = 0;
                if (lane == 0) item = ib + atomicAdd(&B.queue[p], 1);
                item = __shfl_sync(kFull, item, 0);
                if (item >= ie) break;            // every item of the phase is taken once
                const int c = class_of(B, item, cb, ce);
                const WParams &P = B.cls[c];
                const int64_t r0 = P.row_begin + (item - B.prefix[c]) * (int64_t)B.chunk_rows;
                const int64_t r1 = min(r0 + (int64_t)B.chunk_rows, P.row_end);
                const int v = B.variant[c];
                for (int64_t row = r0; row < r1; ++row) {
                    if (MIXED) {
                        const bool q = P.dim == 2 ? mixed_dispatch_d<2>(v, P, row, base)
                                                  : mixed_dispatch_d<3>(v, P, row, base);
                        if (q && lane == 0) {
                            const int slot = atomicAdd(B.fb_count, 1);
                            B.fb_list[slot] = ((u64)c << 32) | (u64)row;
                        }
                        __syncwarp();
                    } else {
                        if (P.dim == 2) fp64_row<2>(P, row, (double *)base, false);
                        else fp64_row<3>(P, row, (double *)base, false);
                    }
                }
            }
        }
        __syncthreads();
        cb = ce;
    }
}

// The FP32 + refinement kernel is held to 168 registers (the register-resident
// inverse's budget in the per-class launch: 12 warps per SM); 8-warp CTAs
// still fit (168 x 256 registers).
__global__ void __maxnreg__(168) k_weights_batched_mixed(const __grid_constant__ BatchParams B) {
    batched_body<true>(B);
}

__global__ void __launch_bounds__(256) k_weights_batched_fp64(const __grid_constant__ BatchParams B) {
    batched_body<false>(B);
}

__global__ void __launch_bounds__(256) k_weights_batched_fallback(const __grid_constant__ BatchParams B) {
    extern __shared__ double smem[];
    const int wib = threadIdx.x >> 5;
    double *base = (double *)((char *)smem + (size_t)wib * B.fb_slot);
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t count = *B.fb_count;
    for (int64_t t = gw; t < count; t += nw) {
        const u64 e = B.fb_list[t];
        const int c = (int)(e >> 32);
        const int64_t row = (int64_t)(e & 0xffffffffULL);
        const WParams &P = B.cls[c];
        if (P.dim == 2) fp64_row<2>(P, row, base, true);
        else fp64_row<3>(P, row, base, true);
    }
}

// ------------------------------------------------------------------ host
struct Prepared {
    std::vector<WParams> cls;        // classes of the persistent launch (call order)
    std::vector<size_t> foot;        // shared-memory bytes per stencil of each
    size_t fb_slot = 0;              // FP64 bytes per stencil, largest class
    std::vector<int> separate;       // classes launched on their own
    int64_t rows = 0;
    bool mixed = false;
    std::string signature;
};

std::string signature_of(const std::vector<WParams> &cls, int precision) {
    std::string s = precision == MM_FP64 ? "fp64" : "fp32ir";
    char buf[96];
    for (const WParams &P : cls) {
        snprintf(buf, sizeof buf, ";d%d n%d m%d k%d R%d", P.dim, P.n_max, P.m, P.k, P.R);
        s += buf;
    }
    return s;
}

mm_launch_config default_config() {
    mm_launch_config c;
    c.warps_per_block = 4;
    c.blocks_per_sm = 0;   // from the occupancy calculator
    c.chunk_rows = 16;
    return c;
}

size_t round16(size_t b) { return (b + 15) & ~size_t(15); }

// Validates the classes and computes their footprints; classes the
// persistent kernel cannot take (mixed precision with 5 operators) are
// listed in `separate`.
int prepare(mm_ctx *ctx, int nclasses, const mm_weights_class *classes, int precision,
            int64_t row_cap, Prepared &out, std::vector<WeightsJob> &jobs) {
    out.mixed = precision == MM_FP32_IR;
    jobs.clear();
    for (int i = 0; i < nclasses; ++i) {
        const mm_weights_class &C = classes[i];
        if (__builtin_popcount(C.ops) > 5)
            return mm_fail(ctx, MM_EUNSUPPORTED, "class %d: at most 5 operator bits per class", i);
        WeightsJob job{};
        int rc = weights_job_from_args(ctx, C.ops, C.k, C.m, C.dim, C.N, C.d_pts, C.d_normals,
                                       &C.stencils, C.row_begin, C.row_end, C.n_max, C.d_vals,
                                       C.d_status, &job);
        if (rc != MM_OK) return mm_fail(ctx, rc, "class %d: %s", i, ctx->err.c_str());
        if (row_cap > 0 && job.row_end - job.row_begin > row_cap) job.row_end = job.row_begin + row_cap;
        jobs.push_back(job);
        WParams P = wparams_from_job(ctx, job);
        if (out.mixed && P.R > 4) {
            out.separate.push_back(i);
            continue;
        }
        const size_t f64 = round16(fp64_warp_doubles(P.M_max, P.pitch64, P.n_max, P.dim) * sizeof(double));
        const size_t fm = out.mixed ? round16(mixed_layout(P.n_max, P.l, mixed_cols(P.R), P.dim).bytes) : f64;
        out.cls.push_back(P);
        out.foot.push_back(fm);
        out.fb_slot = std::max(out.fb_slot, f64);
        out.rows += P.row_end - P.row_begin;
    }
    out.signature = signature_of(out.cls, precision);
    return MM_OK;
}

// Phase plan for W warps per CTA: shared memory S = max(W * smallest
// footprint, largest footprint) (capped by the device), grown to the most
// that keeps as many CTAs resident per SM (whole KB), so a class of larger
// stencils runs as many of them per CTA as that room allows (3 of the 3D
// refined class in one 8-warp CTA per SM instead of 2); classes ordered by
// the number of stencils that fit in S at once, descending.
int build_params(mm_ctx *ctx, const Prepared &pr, const mm_launch_config &cfg, BatchParams &B,
                 size_t &smem) {
    const int W = cfg.warps_per_block;
    const int nc = (int)pr.cls.size();
    size_t fmin = ~size_t(0), fmax = 0;
    for (size_t f : pr.foot) { fmin = std::min(fmin, f); fmax = std::max(fmax, f); }
    if (fmax > ctx->smem_optin) return mm_fail(ctx, MM_EUNSUPPORTED, "batched: %zu bytes of shared memory per stencil", fmax);
    smem = std::min(std::max((size_t)W * fmin, fmax), (size_t)ctx->smem_optin);
    if (ctx->smem_per_sm > smem + ctx->smem_reserved) {
        const size_t ncta = ctx->smem_per_sm / (smem + ctx->smem_reserved);
        const size_t room = (ctx->smem_per_sm / ncta - ctx->smem_reserved) & ~size_t(1023);
        smem = std::max(smem, std::min(room, (size_t)ctx->smem_optin));
    }
    std::vector<int> order(nc), fit(nc);
    for (int i = 0; i < nc; ++i) {
        order[i] = i;
        fit[i] = (int)std::min<size_t>(W, smem / pr.foot[i]);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return fit[a] > fit[b]; });
    memset(&B, 0, sizeof(BatchParams));
    B.nclasses = nc;
    B.nphases = 0;
    B.chunk_rows = cfg.chunk_rows;
    int64_t items = 0;
    for (int j = 0; j < nc; ++j) {
        const int i = order[j];
        const WParams &P = pr.cls[i];
        B.cls[j] = P;
        if (pr.mixed) {
            const int rpl = (P.M_max + 31) / 32, w4 = 4 * ((P.M_max + 3) / 4);
            const int wreg = rpl == 2 && !ctx->gj_shared && (w4 == 40 || w4 == 48) ? w4 : 0;
            B.variant[j] = (signed char)mixed_variant(P.dim, rpl, P.R, wreg);
        }
        B.prefix[j] = items;
        items += (P.row_end - P.row_begin + cfg.chunk_rows - 1) / cfg.chunk_rows;
        const bool new_phase = B.nphases == 0 || B.phase_warps[B.nphases - 1] != fit[i];
        if (new_phase) {
            B.phase_warps[B.nphases] = fit[i];
            B.phase_slot[B.nphases] = (int)(smem / fit[i] & ~size_t(15));
            ++B.nphases;
        }
        B.phase_end[B.nphases - 1] = j + 1;
    }
    B.prefix[nc] = items;
    B.total_items = items;
    B.fb_slot = (int)pr.fb_slot;
    if (items >= (int64_t(1) << 31)) return mm_fail(ctx, MM_EUNSUPPORTED, "batched: too many work items");
    return MM_OK;
}

// Occupancy query, cached per (device, kernel, block, shared memory) so a
// warmed-up call makes no such query inside a stream capture.
cudaError_t occupancy(const mm_ctx *ctx, const void *kern, int threads, size_t sm, int *out) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_tuple(ctx->device, kern, threads, sm);
    auto it = cache.find(key);
    if (it != cache.end()) { *out = it->second; return cudaSuccess; }
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kern, threads, sm);
    if (e == cudaSuccess) cache[key] = *out;
    return e;
}

int launch_prepared(mm_ctx *ctx, const Prepared &pr, const mm_launch_config &cfg) {
    if (pr.cls.empty()) return MM_OK;
    if (cfg.warps_per_block < 1 || cfg.warps_per_block > 8 || cfg.chunk_rows < 1)
        return mm_fail(ctx, MM_EBADARG, "bad launch config");
    BatchParams *Bp = new BatchParams();
    BatchParams &B = *Bp;
    size_t sm = 0;
    int rc = build_params(ctx, pr, cfg, B, sm);
    if (rc != MM_OK) { delete Bp; return rc; }
    WsCarve wc;
    const size_t o_q = wc.take<int>((size_t)B.nphases + 1);
    const size_t o_fb = pr.mixed ? wc.take<u64>((size_t)pr.rows + 1) : 0;
    char *ws = mm_workspace(ctx, wc.off);
    if (!ws) { delete Bp; return mm_fail(ctx, MM_ENOMEM, "batched workspace of %zu bytes", wc.off); }
    B.queue = (int *)(ws + o_q);
    B.fb_count = B.queue + B.nphases;
    B.fb_list = pr.mixed ? (u64 *)(ws + o_fb) : nullptr;
    cudaStream_t st = ctx->stream;
    const void *kern = pr.mixed ? (const void *)k_weights_batched_mixed : (const void *)k_weights_batched_fp64;
    cudaError_t e = cudaMemsetAsync(B.queue, 0, sizeof(int) * (B.nphases + 1), st);
    if (e == cudaSuccess) e = mm_set_smem(ctx, kern, sm);
    int per_sm = cfg.blocks_per_sm;
    if (e == cudaSuccess && per_sm <= 0) {
        int occ = 0;
        e = occupancy(ctx, kern, cfg.warps_per_block * 32, sm, &occ);
        per_sm = std::max(occ, 1);
    }
    if (e != cudaSuccess) { delete Bp; return mm_fail(ctx, MM_ECUDA, "batched launch setup: %s", cudaGetErrorString(e)); }
    const int blocks = per_sm * ctx->num_sms;
    if (pr.mixed) k_weights_batched_mixed<<<blocks, cfg.warps_per_block * 32, sm, st>>>(B);
    else k_weights_batched_fp64<<<blocks, cfg.warps_per_block * 32, sm, st>>>(B);
    e = cudaGetLastError();
    if (e == cudaSuccess && pr.mixed) {
        const int wpb = (int)std::max<size_t>(1, std::min<size_t>(4, (96 * 1024) / pr.fb_slot));
        const size_t fsm = pr.fb_slot * wpb;
        e = mm_set_smem(ctx, (const void *)k_weights_batched_fallback, fsm);
        if (e == cudaSuccess) {
            const int fb_blocks = (int)std::min<int64_t>((pr.rows + wpb - 1) / wpb, (int64_t)ctx->num_sms * 8);
            k_weights_batched_fallback<<<std::max(fb_blocks, 1), wpb * 32, fsm, st>>>(B);
            e = cudaGetLastError();
        }
    }
    delete Bp;
    if (e != cudaSuccess) return mm_fail(ctx, MM_ECUDA, "batched launch: %s", cudaGetErrorString(e));
    return MM_OK;
}

int run_separate(mm_ctx *ctx, const Prepared &pr, const std::vector<WeightsJob> &jobs, int precision) {
    for (int i : pr.separate) {
        int rc = weights_launch(ctx, jobs[i], precision);
        if (rc != MM_OK) return rc;
    }
    return MM_OK;
}

}  // namespace

int batched_init_device(mm_ctx *ctx) {
    MonoTable t;
    mono_table_host(t);
    MM_CUDA_CHECK(ctx, cudaMemcpyToSymbol(c_mono, &t, sizeof(t)));
    return MM_OK;
}

extern "C" {

int mm_rbffd_weights_batched(mm_ctx *ctx, int nclasses, const mm_weights_class *classes,
                             int precision, const mm_launch_config *config) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (nclasses < 1 || nclasses > kMaxBatchClasses || !classes)
        return mm_fail(ctx, MM_EBADARG, "nclasses must be in [1, %d]", kMaxBatchClasses);
    if (precision != MM_FP64 && precision != MM_FP32_IR)
        return mm_fail(ctx, MM_EBADARG, "unknown precision %d", precision);
    DeviceGuard g(ctx);
    Prepared pr;
    std::vector<WeightsJob> jobs;
    int rc = prepare(ctx, nclasses, classes, precision, 0, pr, jobs);
    if (rc == MM_OK) {
        mm_launch_config cfg;
        if (config) cfg = *config;
        else {
            auto it = ctx->tiles.find(pr.signature);
            cfg = it != ctx->tiles.end() ? it->second : default_config();
        }
        rc = launch_prepared(ctx, pr, cfg);
        if (rc == MM_OK) rc = run_separate(ctx, pr, jobs, precision);
    }
    return rc;
}

int mm_autotune_batched(mm_ctx *ctx, int nclasses, const mm_weights_class *classes, int precision,
                        int64_t sample_rows, mm_launch_config *best, double *best_ms) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (nclasses < 1 || nclasses > kMaxBatchClasses || !classes)
        return mm_fail(ctx, MM_EBADARG, "nclasses must be in [1, %d]", kMaxBatchClasses);
    if (precision != MM_FP64 && precision != MM_FP32_IR)
        return mm_fail(ctx, MM_EBADARG, "unknown precision %d", precision);
    if (sample_rows <= 0) sample_rows = 16384;
    DeviceGuard g(ctx);
    Prepared pr;
    std::vector<WeightsJob> jobs;
    int rc = prepare(ctx, nclasses, classes, precision, sample_rows, pr, jobs);
    if (rc != MM_OK) return rc;
    // full-size signature: the sample only truncates row ranges
    mm_launch_config best_cfg = default_config();
    double best_t = 1e300;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int wpbs[] = {1, 2, 4, 8};
    const int chunks[] = {4, 16, 64};
    for (int wpb : wpbs) {
        BatchParams *Bp = new BatchParams();
        size_t sm = 0;
        mm_launch_config probe{wpb, 1, 16};
        const bool fits = build_params(ctx, pr, probe, *Bp, sm) == MM_OK;
        delete Bp;
        ctx->err.clear();
        if (!fits || sm > ctx->smem_optin) continue;
        const void *kern = pr.mixed ? (const void *)k_weights_batched_mixed : (const void *)k_weights_batched_fp64;
        if (mm_set_smem(ctx, kern, sm) != cudaSuccess) { cudaGetLastError(); continue; }
        int occ = 0;
        if (occupancy(ctx, kern, wpb * 32, sm, &occ) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            continue;
        }
        for (int bps = std::max(1, occ / 2); bps <= occ; bps = bps == occ ? occ + 1 : std::min(occ, bps * 2)) {
            for (int ch : chunks) {
                mm_launch_config c{wpb, bps, ch};
                rc = launch_prepared(ctx, pr, c);           // warm-up
                if (rc != MM_OK) break;
                float total = 0.f;
                for (int rep = 0; rep < 3 && rc == MM_OK; ++rep) {
                    cudaEventRecord(e0, ctx->stream);
                    rc = launch_prepared(ctx, pr, c);
                    cudaEventRecord(e1, ctx->stream);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    total += ms;
                }
                if (rc != MM_OK) break;
                if (total / 3 < best_t) { best_t = total / 3; best_cfg = c; }
            }
            if (rc != MM_OK) break;
        }
        if (rc != MM_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MM_OK) return rc;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mm_fail(ctx, MM_ECUDA, "autotune: %s", cudaGetErrorString(e));
    // key the table by the full-size signature (row counts do not enter it)
    ctx->tiles[pr.signature] = best_cfg;
    if (best) *best = best_cfg;
    if (best_ms) *best_ms = best_t;
    return MM_OK;
}

int mm_tile_table_save(const mm_ctx *ctx, const char *path) {
    if (!ctx || !path) return MM_EBADARG;
    FILE *f = fopen(path, "w");
    if (!f) return MM_EBADARG;
    fprintf(f, "# libmm batched-weights launch shapes: signature|warps_per_block|blocks_per_sm|chunk_rows\n");
    for (const auto &kv : ctx->tiles)
        fprintf(f, "%s|%d|%d|%d\n", kv.first.c_str(), kv.second.warps_per_block, kv.second.blocks_per_sm,
                kv.second.chunk_rows);
    fclose(f);
    return MM_OK;
}

int mm_tile_table_load(mm_ctx *ctx, const char *path) {
    if (!ctx || !path) return MM_EBADARG;
    FILE *f = fopen(path, "r");
    if (!f) return mm_fail(ctx, MM_EBADARG, "cannot open %s", path);
    char line[4096];
    int rc = MM_OK;
    while (fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        std::string s(line);
        while (!s.empty() && (s.back() == '\n' || s.back() == '\r')) s.pop_back();
        size_t p3 = s.rfind('|');
        size_t p2 = p3 == std::string::npos ? p3 : s.rfind('|', p3 - 1);
        size_t p1 = p2 == std::string::npos || p2 == 0 ? std::string::npos : s.rfind('|', p2 - 1);
        if (p1 == std::string::npos) { rc = mm_fail(ctx, MM_EBADARG, "bad tile table line"); break; }
        mm_launch_config c;
        c.warps_per_block = atoi(s.substr(p1 + 1, p2 - p1 - 1).c_str());
        c.blocks_per_sm = atoi(s.substr(p2 + 1, p3 - p2 - 1).c_str());
        c.chunk_rows = atoi(s.substr(p3 + 1).c_str());
        if (c.warps_per_block < 1 || c.warps_per_block > 8 || c.chunk_rows < 1 || c.blocks_per_sm < 0) {
            rc = mm_fail(ctx, MM_EBADARG, "bad tile table entry");
            break;
        }
        ctx->tiles[s.substr(0, p1)] = c;
    }
    fclose(f);
    return rc;
}

}  // extern "C"
