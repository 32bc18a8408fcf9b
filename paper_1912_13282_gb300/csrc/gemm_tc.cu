// Training GEMMs of the surrogate MLP on the Blackwell tensor cores:
//     C[M x N] = A[M x K] * B[N x K]^T,   A and B BF16, both K-major,
// FP32 accumulators in tensor memory, one CTA of 4 warps per 128-row tile of
// C (all N columns of a tile up to 256 in one accumulator).  The K loop runs
// in blocks of 64: every thread copies its share of the A and B blocks into
// shared memory in the 128-byte-swizzled K-major layout (16-byte cp.async,
// zero-filled outside the matrix), the stage is fenced for the tensor core's
// (async) proxy, and one thread issues the four K = 16 tcgen05.mma of the
// block and commits them to the stage's mbarrier; two stages, so the copies
// of block k + 1 overlap the MMAs of block k.  K may be split across
// blockIdx.z (partial products, summed later in a fixed order).
//
// Epilogues (every thread holds one row of the tile = one tensor-memory lane,
// read 32 columns at a time): FP32 partial products; bias; bias + GELU with
// the pre-activation (FP32), the activation (BF16) and its transpose (BF16,
// [N x ldt]: for a fixed column the warp's 32 rows are consecutive
// addresses); the GELU derivative times the accumulator (the backward
// pass's dZ, again with its transpose).  Waits are bounded (tc::kSpin polls):
// on a timeout the kernel sets *err, writes nothing from that tile and frees
// its tensor memory.
#include <cuda_bf16.h>

#include "mm_internal.cuh"
#include "tc_common.cuh"

namespace {

using namespace tc;
typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ float tanh_hw(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float gelu_tc(float z) {
    const float c = 0.7978845608028654f;
    return 0.5f * z * (1.0f + tanh_hw(c * fmaf(0.044715f * z, z * z, z)));
}
__device__ __forceinline__ float gelu_grad_tc(float z) {
    const float c = 0.7978845608028654f;
    const float t = tanh_hw(c * fmaf(0.044715f * z, z * z, z));
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * c * (1.0f + 3.0f * 0.044715f * z * z);
}

// Copies rows [r0, r0 + rows) x K-block [k0, k0 + 64) of a K-major matrix
// (ld elements per row) into a 128B-swizzled tile at `dst`; entries outside
// [0, R) x [0, k_end) are zero (a chunk that straddles k_end copies only its
// leading bytes; cp.async fills the rest with zeros).
__device__ __forceinline__ void load_block(uint32_t dst, const bf16 *G, int64_t ld, int r0, int rows, int R,
                                           int k0, int k_end) {
    for (int i = threadIdx.x; i < rows * 8; i += blockDim.x) {
        const int r = i >> 3, c = i & 7;
        const int gr = r0 + r, gk = k0 + 8 * c;
        const bool in = gr < R && gk < k_end;
        const bf16 *src = in ? G + (int64_t)gr * ld + gk : G;
        const uint32_t bytes = in ? 2u * (uint32_t)min(8, k_end - gk) : 0u;
        cp_async16(dst + (uint32_t)r * 128u + ((uint32_t)(c ^ (r & 7)) << 4), src, bytes);
    }
}

template <int NT, int EPI>
__global__ void __launch_bounds__(128) k_gemm_tc(const __grid_constant__ TcGemmArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sb = smem_u32(sm);
    constexpr uint32_t kABytes = 16384, kBBytes = NT * 128, kStage = kABytes + kBBytes;
    const uint32_t bar = sb + 2 * kStage;          // [0], [1]: stages, [2]: all MMAs done
    const uint32_t tslot = bar + 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * 128, n0 = blockIdx.x * NT;
    const int k_begin = blockIdx.z * a.kslice;
    const int k_end = min(a.K, k_begin + a.kslice);
    const int nk = (k_end - k_begin + 63) / 64;   // >= 1 by the grid's construction
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) mbar_init(bar + 8u * i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tslot), "r"(NT)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(sm + (tslot - sb));
    constexpr uint32_t idesc = idesc_bf16(128, NT);
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
        const int s = kb & 1;
        // the stage's previous MMAs (block kb - 2) must be done before it is overwritten
        if (kb >= 2) ok = mbar_wait(bar + 8u * s, (uint32_t)(((kb >> 1) - 1) & 1)) && ok;
        ok = __syncthreads_and(ok);
        if (!ok) break;
        const uint32_t sa = sb + s * kStage, sbB = sa + kABytes;
        const int k0 = k_begin + 64 * kb;
        load_block(sa, a.A, a.lda, m0, 128, a.M, k0, k_end);
        load_block(sbB, a.B, a.ldb, n0, NT, a.N, k0, k_end);
        cp_async_wait_all();
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const int kk = min(64, k_end - k0);
            for (int j = 0; j < (kk + 15) / 16; ++j)
                umma(tmem, sdesc(sa + 32u * j), sdesc(sbB + 32u * j), idesc, (kb | j) != 0);
            umma_commit(bar + 8u * s);
        }
    }
    if (tid == 0) umma_commit(bar + 16u);          // arrives once every MMA above has completed
    ok = mbar_wait(bar + 16u, 0) && ok;
    ok = __syncthreads_and(ok);
    tc_fence_after();
    if (!ok) {
        if (tid == 0) atomicExch(a.err, 1);
    } else {
        const int row = m0 + 32 * warp + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16);
        const bool rin = row < a.M;
        for (int cc = 0; cc < NT; cc += 32) {
            float v[32];
            tmem_ld32(lane_addr + (uint32_t)cc, v);
            const int c0 = n0 + cc;
            if (c0 >= a.N) break;
            const int ncol = min(32, a.N - c0);
            if (EPI == kTcPartial) {
                if (rin) {
                    float *dst = a.c + ((int64_t)blockIdx.z * a.M + row) * a.ldc + c0;
                    for (int j = 0; j < ncol; ++j) dst[j] = v[j];
                }
            } else if (EPI == kTcBias) {
                if (rin) {
                    float *dst = a.c + (int64_t)row * a.ldc + c0;
                    for (int j = 0; j < ncol; ++j) dst[j] = v[j] + __ldg(a.bias + c0 + j);
                }
            } else {
                // kTcBiasGelu: z = acc + b, h = gelu(z);  kTcDGelu: h = acc * gelu'(z)
                bf16 hv[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float out = 0.0f;
                    if (rin && j < ncol) {
                        if (EPI == kTcBiasGelu) {
                            const float z = v[j] + __ldg(a.bias + c0 + j);
                            a.z[(int64_t)row * a.ldz + c0 + j] = z;
                            out = gelu_tc(z);
                        } else {
                            out = v[j] * gelu_grad_tc(a.z[(int64_t)row * a.ldz + c0 + j]);
                        }
                    }
                    hv[j] = __float2bfloat16(out);
                }
                if (rin) {
                    bf16 *dst = a.h + (int64_t)row * a.ldh + c0;
                    for (int j = 0; j < ncol; ++j) dst[j] = hv[j];
                    if (a.ht)
                        for (int j = 0; j < ncol; ++j) a.ht[(int64_t)(c0 + j) * a.ldht + row] = hv[j];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT) : "memory");
    }
}

template <int NT>
int launch_nt(mm_ctx *ctx, const TcGemmArgs &a) {
    constexpr uint32_t smem = 2 * (16384 + NT * 128) + 64 + 1024;
    const dim3 grid((a.N + NT - 1) / NT, (a.M + 127) / 128, (a.K + a.kslice - 1) / a.kslice);
    const void *k = nullptr;
    switch (a.epi) {
        case kTcPartial: k = (const void *)k_gemm_tc<NT, kTcPartial>; break;
        case kTcBias: k = (const void *)k_gemm_tc<NT, kTcBias>; break;
        case kTcBiasGelu: k = (const void *)k_gemm_tc<NT, kTcBiasGelu>; break;
        default: k = (const void *)k_gemm_tc<NT, kTcDGelu>; break;
    }
    MM_CUDA_CHECK(ctx, mm_set_smem(ctx, k, smem));
    switch (a.epi) {
        case kTcPartial: k_gemm_tc<NT, kTcPartial><<<grid, 128, smem, ctx->stream>>>(a); break;
        case kTcBias: k_gemm_tc<NT, kTcBias><<<grid, 128, smem, ctx->stream>>>(a); break;
        case kTcBiasGelu: k_gemm_tc<NT, kTcBiasGelu><<<grid, 128, smem, ctx->stream>>>(a); break;
        default: k_gemm_tc<NT, kTcDGelu><<<grid, 128, smem, ctx->stream>>>(a); break;
    }
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

}  // namespace

int tc_gemm(mm_ctx *ctx, const TcGemmArgs &a) {
    if (a.M <= 0 || a.N <= 0 || a.K <= 0) return MM_OK;
    if (a.lda % 8 || a.ldb % 8 || a.kslice <= 0 || a.kslice % 64 || a.N > 256)
        return mm_fail(ctx, MM_EUNSUPPORTED, "tensor-core GEMM: lda, ldb multiples of 8, kslice of 64, N <= 256");
    // 128 x 64 tiles unless that leaves fewer than two tiles per SM: the
    // training GEMMs are small (4,096 x 256 x 256), so parallelism matters
    // more than re-reading A once per 64 columns
    if (a.N <= 32) return launch_nt<32>(ctx, a);
    const int64_t tiles64 = ((a.M + 127) / 128) * (int64_t)((a.N + 63) / 64) * ((a.K + a.kslice - 1) / a.kslice);
    if (a.N <= 64 || tiles64 <= 2 * (int64_t)ctx->num_sms) return launch_nt<64>(ctx, a);
    return launch_nt<256>(ctx, a);
}
