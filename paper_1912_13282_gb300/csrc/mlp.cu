// Learned surrogate of the Laplacian stencil weights (no counterpart in the
// paper): a GELU multilayer perceptron 2n -> 256 -> 256 -> 256 -> n on the
// scaled stencil offsets, BF16 weights/activations with FP32 accumulation on
// the tensor cores (tcgen05: the training GEMMs in gemm_tc.cu, the fused
// inference in mlp_tc.cu), trained on weights the method itself produces.  Its predictions are projected (double-FP32, or FP64) onto the rows
// Q^T w = l_q of the augmented system (Section 2.2.2, eq. rbf-system-aug), then
// checked against the remaining rows' residual; rejected stencils get a solve.
//
// Layout: feature width padded to 64, outputs to 32 (zero weights and inputs in
// the padding), hidden width 256, 3 hidden layers.  Parameters are FP32
// "master" copies updated by Adam, with BF16 copies for the GEMMs.
#include <cuda_bf16.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <random>
#include <vector>

#include "rbffd_dev.cuh"

struct mm_mlp {
    int device = 0;
    int n_in = 0, n_out = 0, H = 256, L = 3;
    static constexpr int KIN = 64, KOUT = 32;   // padded widths
    int64_t bmax = 0;                           // rows per internal batch
    int step = 0;
    // device buffers
    float *p = nullptr, *g = nullptr, *am = nullptr, *av = nullptr;   // padded layout
    __nv_bfloat16 *wb = nullptr;                                       // bf16 weights
    float *Z = nullptr;                 // [3][bmax][256] pre-activations
    __nv_bfloat16 *Hb = nullptr;        // [3][bmax][256] activations
    __nv_bfloat16 *Xb = nullptr;        // [bmax][64]
    float *Y = nullptr;                 // [bmax][32]
    __nv_bfloat16 *dY = nullptr;        // [bmax][32]
    __nv_bfloat16 *dZa = nullptr, *dZb = nullptr;   // [bmax][256]
    // transposed copies for the tensor-core GEMMs, whose operands are K-major:
    // weights [in][out] (W2..W4), activations / input / output gradient / dZ
    // as [features][bmax]
    __nv_bfloat16 *WT = nullptr, *HT = nullptr, *XT = nullptr, *dYT = nullptr;
    __nv_bfloat16 *dZTa = nullptr, *dZTb = nullptr;
    float *loss = nullptr;              // [1]
    float *part = nullptr;              // [64][256][256] split-K / bias partial sums
    float *ymean = nullptr, *ystd = nullptr;   // [32] output scaling (device)
    __nv_bfloat16 *img = nullptr;       // weight image of the fused tensor-core inference
    int *tc_err = nullptr;              // its timeout flag
    std::vector<float> h_mean, h_std;
    int64_t np_pad = 0;
    // offsets into the padded parameter vector
    int64_t oW[4], ob[4];
};

namespace {

typedef __nv_bfloat16 bf16;
constexpr int kH = 256, kKIN = 64, kKOUT = 32;

// ------------------------------------------------------------ elementwise
__global__ void k_pack_x(const float *x, int64_t B, int n_in, bf16 *xb, bf16 *xt, int64_t ldt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B * kKIN;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / kKIN;
        const int c = (int)(i % kKIN);
        const bf16 v = __float2bfloat16(c < n_in ? x[r * n_in + c] : 0.f);
        xb[i] = v;
        if (xt) xt[(int64_t)c * ldt + r] = v;
    }
}

// dY = 2 (Y - (T - mean)/std) / (B n_out) on the n_out real columns (0 in the
// padding); loss += mean squared normalised error.
__global__ void k_loss(const float *Y, const float *T, int64_t B, int n_out, const float *mean,
                       const float *std, bf16 *dY, bf16 *dYT, int64_t ldt, float *loss) {
    float s = 0.f;
    const float scale = 2.0f / ((float)B * n_out);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B * kKOUT;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / kKOUT;
        const int c = (int)(i % kKOUT);
        float d = 0.f;
        if (c < n_out) {
            const float t = (T[r * n_out + c] - mean[c]) / std[c];
            const float e = Y[i] - t;
            d = scale * e;
            s += e * e;
        }
        dY[i] = __float2bfloat16(d);
        dYT[(int64_t)c * ldt + r] = __float2bfloat16(d);
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, s / ((float)B * n_out));
}

// Bias-gradient partial sums: block b sums rows b, b + nblocks, ... of dZ
// column by column into part[b][c].
__global__ void k_bias_partial(const bf16 *dZ, int64_t B, int N, float *part) {
    const int c = threadIdx.x;
    if (c >= N) return;
    float s = 0.f;
    for (int64_t r = blockIdx.x; r < B; r += gridDim.x) s += __bfloat162float(dZ[r * N + c]);
    part[(int64_t)blockIdx.x * N + c] = s;
}

// out[i] = sum_z part[z][i] in z order (deterministic), i < count.
__global__ void k_sum_parts(const float *part, int nparts, int64_t count, float *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < nparts; ++z) s += part[(int64_t)z * count + i];
        out[i] = s;
    }
}

// Adam (Kingma & Ba) on the FP32 master copy; refreshes the BF16 weights.
__global__ void k_adam(float *p, const float *g, float *m, float *v, int64_t np, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Transposed BF16 copies [in][out] of W2, W3 (256 x 256) and W4 (32 x 256),
// the B operands of the backward GEMMs.
__global__ void k_refresh_wt(const float *p, bf16 *wt, int64_t o2, int64_t o3, int64_t o4) {
    const int64_t n2 = (int64_t)kH * kH, tot = 2 * n2 + (int64_t)kH * kKOUT;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = i, off;
        int nout;
        if (e < n2) { off = o2; nout = kH; }
        else if ((e -= n2) < n2) { off = o3; nout = kH; }
        else { e -= n2; off = o4; nout = kKOUT; }
        const int64_t in = e / nout, out = e % nout;          // wt[in][out] = W[out][in]
        wt[i] = __float2bfloat16(p[off + out * kH + in]);
    }
}

// BF16 copies of the four weight matrices (not the biases).
__global__ void k_refresh_bf16(const float *p, bf16 *wb, int64_t o1, int64_t n1, int64_t o2, int64_t n2,
                               int64_t o3, int64_t n3, int64_t o4, int64_t n4) {
    const int64_t tot = n1 + n2 + n3 + n4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t src;
        if (i < n1) src = o1 + i;
        else if (i < n1 + n2) src = o2 + (i - n1);
        else if (i < n1 + n2 + n3) src = o3 + (i - n1 - n2);
        else src = o4 + (i - n1 - n2 - n3);
        wb[i] = __float2bfloat16(p[src]);
    }
}

__global__ void k_denorm(const float *Y, int64_t B, int n_out, const float *mean, const float *std,
                         float *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B * n_out;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / n_out;
        const int c = (int)(i % n_out);
        out[i] = Y[r * kKOUT + c] * std[c] + mean[c];
    }
}

int grid1(mm_ctx *ctx, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8));
}

// bf16 weight matrix i (0..3) inside wb
const bf16 *wmat(const mm_mlp *net, int i) {
    int64_t off = 0;
    const int64_t sz[4] = {(int64_t)kH * kKIN, (int64_t)kH * kH, (int64_t)kH * kH, (int64_t)kKOUT * kH};
    for (int j = 0; j < i; ++j) off += sz[j];
    return net->wb + off;
}

// Transposed weight matrix i (1..3) inside WT, [in][out]
const bf16 *wtmat(const mm_mlp *net, int i) {
    return net->WT + (int64_t)(i - 1) * kH * kH;
}

// dW = dZ^T H on the tensor cores: A = dZ^T [out x B], B = H^T [in x B]
// (both K-major, K = the B rows), split-K slices of `kslice` rows summed in
// slice order, and db = column sums of dZ; both deterministic.
int weight_grads(mm_ctx *ctx, mm_mlp *net, int out, int in, int64_t B, const bf16 *dZ, const bf16 *dZT,
                 const bf16 *HinT, float *dW, float *db, int splits) {
    TcGemmArgs a{};
    a.M = out; a.N = in; a.K = (int)B;
    a.kslice = (int)(((B + splits - 1) / splits + 63) / 64 * 64);
    a.A = dZT; a.lda = net->bmax;
    a.B = HinT; a.ldb = net->bmax;
    a.epi = kTcPartial;
    a.c = net->part; a.ldc = in;
    a.err = net->tc_err;
    int rc = tc_gemm(ctx, a);
    if (rc) return rc;
    const int slices = (int)((B + a.kslice - 1) / a.kslice);
    k_sum_parts<<<grid1(ctx, (int64_t)out * in), 256, 0, ctx->stream>>>(net->part, slices, (int64_t)out * in, dW);
    const int nb = (int)std::min<int64_t>(B, 256);
    k_bias_partial<<<nb, out, 0, ctx->stream>>>(dZ, B, out, net->part);
    k_sum_parts<<<grid1(ctx, out), 256, 0, ctx->stream>>>(net->part, nb, out, db);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

// Forward pass of `B` rows already packed in net->Xb; output in net->Y.  Each
// hidden layer writes its pre-activation, its activation and the transposed
// activation (for the weight gradients).
int forward(mm_ctx *ctx, mm_mlp *net, int64_t B) {
    const bf16 *in = net->Xb;
    int kin = kKIN;
    for (int l = 0; l < 3; ++l) {
        TcGemmArgs a{};
        a.M = (int)B; a.N = kH; a.K = kin; a.kslice = kin;
        a.A = in; a.lda = kin;
        a.B = wmat(net, l); a.ldb = kin;
        a.epi = kTcBiasGelu;
        a.bias = net->p + net->ob[l];
        a.z = net->Z + (int64_t)l * net->bmax * kH; a.ldz = kH;
        a.h = net->Hb + (int64_t)l * net->bmax * kH; a.ldh = kH;
        a.ht = net->HT + (int64_t)l * net->bmax * kH; a.ldht = net->bmax;
        a.err = net->tc_err;
        int rc = tc_gemm(ctx, a);
        if (rc != MM_OK) return rc;
        in = a.h;
        kin = kH;
    }
    TcGemmArgs o{};
    o.M = (int)B; o.N = kKOUT; o.K = kH; o.kslice = kH;
    o.A = in; o.lda = kH;
    o.B = wmat(net, 3); o.ldb = kH;
    o.epi = kTcBias;
    o.c = net->Y; o.ldc = kKOUT;
    o.bias = net->p + net->ob[3];
    o.err = net->tc_err;
    return tc_gemm(ctx, o);
}

// dZ_prev = (dZ W) * gelu'(Z_prev) on the tensor cores: A = dZ [B x out],
// B = W^T [in x out]; writes dZ_prev and its transpose.
int backward_data(mm_ctx *ctx, mm_mlp *net, int64_t B, const bf16 *dZ, int out, const bf16 *WT, float *Zprev,
                  bf16 *dZp, bf16 *dZpT) {
    TcGemmArgs a{};
    a.M = (int)B; a.N = kH; a.K = out; a.kslice = 64 * ((out + 63) / 64);
    a.A = dZ; a.lda = out;
    a.B = WT; a.ldb = out;
    a.epi = kTcDGelu;
    a.z = Zprev; a.ldz = kH;
    a.h = dZp; a.ldh = kH;
    a.ht = dZpT; a.ldht = net->bmax;
    a.err = net->tc_err;
    return tc_gemm(ctx, a);
}

// Gradients of the mean squared error w.r.t. all parameters into net->g
// (every entry written, in a fixed summation order), for B rows with targets T (raw, [B x n_out]).
int backward(mm_ctx *ctx, mm_mlp *net, int64_t B, const float *T) {
    cudaStream_t st = ctx->stream;
    k_loss<<<grid1(ctx, B * kKOUT), 256, 0, st>>>(net->Y, T, B, net->n_out, net->ymean, net->ystd,
                                                   net->dY, net->dYT, net->bmax, net->loss);
    MM_LAUNCH_CHECK(ctx);
    const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(64, B / 128));
    // output layer
    const bf16 *H3T = net->HT + 2 * net->bmax * kH;
    int rc = weight_grads(ctx, net, kKOUT, kH, B, net->dY, net->dYT, H3T, net->g + net->oW[3],
                          net->g + net->ob[3], splits);
    if (rc) return rc;
    rc = backward_data(ctx, net, B, net->dY, kKOUT, net->WT + 2 * (int64_t)kH * kH, net->Z + 2 * net->bmax * kH,
                       net->dZa, net->dZTa);
    if (rc) return rc;
    bf16 *dZ = net->dZa, *dZn = net->dZb, *dZT = net->dZTa, *dZTn = net->dZTb;
    for (int l = 2; l >= 0; --l) {
        const bf16 *HinT = l == 0 ? net->XT : net->HT + (int64_t)(l - 1) * net->bmax * kH;
        const int kin = l == 0 ? kKIN : kH;
        rc = weight_grads(ctx, net, kH, kin, B, dZ, dZT, HinT, net->g + net->oW[l], net->g + net->ob[l], splits);
        if (rc) return rc;
        if (l > 0) {
            rc = backward_data(ctx, net, B, dZ, kH, wtmat(net, l), net->Z + (int64_t)(l - 1) * net->bmax * kH,
                               dZn, dZTn);
            if (rc) return rc;
            std::swap(dZ, dZn);
            std::swap(dZT, dZTn);
        }
    }
    return MM_OK;
}

int refresh_bf16(mm_ctx *ctx, mm_mlp *net) {
    const int64_t n1 = (int64_t)kH * kKIN, n2 = (int64_t)kH * kH, n4 = (int64_t)kKOUT * kH;
    k_refresh_bf16<<<grid1(ctx, n1 + 2 * n2 + n4), 256, 0, ctx->stream>>>(
        net->p, net->wb, net->oW[0], n1, net->oW[1], n2, net->oW[2], n2, net->oW[3], n4);
    k_refresh_wt<<<grid1(ctx, 2 * n2 + n4), 256, 0, ctx->stream>>>(net->p, net->WT, net->oW[1], net->oW[2],
                                                                   net->oW[3]);
    MM_LAUNCH_CHECK(ctx);
    const int rc = mlp_tc_image(ctx, net->p, net->oW, net->img);
    if (rc != MM_OK) return rc;
    return MM_OK;
}

// ------------------------------------------------------ stencil features
// Scaled offsets xi_j = (x_j - x_c)/s, s = max distance, of the n stencil nodes
// in stencil order: feature row [xi_0x, xi_0y, xi_1x, ...] (FP32).  With
// `orient` (2D) the offsets are turned so the nearest other node lies on +x
// and mirrored so the next one has y >= 0: Laplacian weights do not change
// under rotations and reflections of the whole stencil, so the network sees
// one canonical frame per stencil.
template <int DIM>
__global__ void k_features(const double *pts, const int64_t *rp, const int32_t *col, int64_t r0,
                           int64_t r1, int n, int orient, float *x, double *scale) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = r0 + gw; row < r1; row += nw) {
        const int64_t b = rp[row];
        // offsets: the difference in FP64 (it may cancel), the rest in FP32
        // (the features feed a BF16 network)
        double d[DIM] = {};
        float f[DIM] = {};
        float r2 = 0.0f;
        if (lane < n) {
            const int j = col[b + lane];
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                d[a] = pts[(int64_t)j * DIM + a] - pts[row * DIM + a];
                f[a] = (float)d[a];
                r2 = fmaf(f[a], f[a], r2);
            }
        }
        for (int o = 16; o; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
        const float inv = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
#pragma unroll
        for (int a = 0; a < DIM; ++a) f[a] *= inv;
        if (DIM == 2 && orient && n >= 3) {
            const float ax = __shfl_sync(0xffffffffu, f[0], 1), ay = __shfl_sync(0xffffffffu, f[1], 1);
            const float an = sqrtf(ax * ax + ay * ay);
            const float c = an > 0.f ? ax / an : 1.f, sn = an > 0.f ? ay / an : 0.f;
            const float xr = c * f[0] + sn * f[1], yr = -sn * f[0] + c * f[1];
            const float y2 = __shfl_sync(0xffffffffu, yr, 2);
            f[0] = xr;
            f[1] = y2 < 0.f ? -yr : yr;
        }
        if (lane < n) {
#pragma unroll
            for (int a = 0; a < DIM; ++a) x[(row - r0) * (int64_t)n * DIM + lane * DIM + a] = f[a];
        }
        if (scale) {
            // s = max distance in FP64, as the weights solvers scale
            double q2 = 0.0;
#pragma unroll
            for (int a = 0; a < DIM; ++a) q2 = fma(d[a], d[a], q2);
            for (int o = 16; o; o >>= 1) q2 = fmax(q2, __shfl_xor_sync(0xffffffffu, q2, o));
            if (lane == 0) scale[row - r0] = sqrt(q2);
        }
    }
}

// ------------------------------------------------- projection and residual check
// One warp per stencil (n <= 32, l <= 16).  wt: predicted scaled Laplacian
// weights [n] (FP32).  Least-norm correction onto the monomial rows
// Q^T w = l_q of the augmented system:
//     w = wt + Q z,  (Q^T Q) z = l_q - Q^T w,
// repeated while the constraint rows are off by more than 1e-13 of their
// terms (at most 6 passes).  Q, w and the constraint residuals are carried in
// double-FP32 (compensated sums on the FP32 pipe), or in FP64 when the
// context asks for native FP64 (MM_OPT_WIDE); z comes from an FP32
// inverse of the Jacobi-scaled Gram matrix (in-place Gauss-Jordan, no
// pivoting: the matrix is symmetric positive definite).
// Residual check (FP32, A evaluated on the fly): r = l_phi - A w, lambda =
// (Q^T Q)^-1 Q^T r (least squares), rho = ||r - Q lambda||_inf /
// ||l_phi||_inf; accept if rho <= tau.  Up to 8 blocks of 4 warps per SM.
struct ProjParams {
    WParams P;              // LAP only, k, m, row range, output vals[0]
    const float *wt;        // [rows x n] predictions (scaled units), row - row_begin
    float tau;
    int *fb_list, *fb_count;
    float *rho_out;         // optional [rows]
};

__device__ __forceinline__ float phs32(float r2, int k) {
    float p = r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f;
    for (int i = 1; i < k; i += 2) p *= r2;
    return p;
}

template <int DIM, bool W64>
__global__ void __launch_bounds__(128, 8) k_project(const __grid_constant__ ProjParams J) {
    constexpr int NM = 32, LM = 16, QP = LM + 1, GP = LM + 1;   // odd pitches: conflict-free rows
    const WParams &P = J.P;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    __shared__ double s_xi[4][NM * DIM];          // offsets (FP64; double-FP32 in place unless W64)
    __shared__ double s_Q[4][NM][QP];             // Q (double-FP32 pairs, or FP64 if W64)
    __shared__ float s_G[4][LM][GP];              // Jacobi-scaled Gram matrix, then its inverse
    __shared__ double s_w[4][NM];                 // weights (double-FP32 pairs, or FP64 if W64)
    __shared__ float s_u[4][LM], s_d[4][LM], s_z[4][LM], s_r[4][NM];
    float2 (*Qf)[QP] = reinterpret_cast<float2 (*)[QP]>(s_Q[wib]);
    double (*Qd)[QP] = s_Q[wib];
    float (*G)[GP] = s_G[wib];
    float2 *wf = reinterpret_cast<float2 *>(s_w[wib]);
    double *wd = s_w[wib];
    float *u = s_u[wib], *dsc = s_d[wib], *zz = s_z[wib], *rr = s_r[wib];
    const int l = P.l, di = DIM - 2, k = P.k;
    const int bl = lane & 15, hl = lane >> 4;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = P.row_begin + gw; row < P.row_end; row += nw) {
        int n;
        int64_t rb;
        double s;
        double *xi = s_xi[wib];
        if (!load_stencil<DIM>(P, row, n, rb, xi, s) || n > NM || l > LM) {
            reject_row(P, row, rb, n, MM_ST_BADARG);
            __syncwarp();
            continue;
        }
        float2 *xf = reinterpret_cast<float2 *>(xi);
        if (!W64) {
            for (int j = lane; j < n * DIM; j += 32) xf[j] = ff_from_double(xi[j]);
            __syncwarp();
        }
        // leading FP32 parts of the offsets, Q and w
        auto x32 = [&](int j, int a) { return W64 ? (float)xi[j * DIM + a] : xf[j * DIM + a].x; };
        auto q32 = [&](int j, int b) { return W64 ? (float)Qd[j][b] : Qf[j][b].x; };
        auto w32 = [&](int j) { return W64 ? (float)wd[j] : __fadd_rn(wf[j].x, wf[j].y); };
        // Q by stencil node, predicted weights
        if (lane < n) {
            if (W64) {
                double *Qj = Qd[lane];
                Qj[0] = 1.0;
                for (int b = 1; b < l; ++b) Qj[b] = Qj[c_mono.parent[di][b]] * xi[lane * DIM + c_mono.var[di][b]];
                wd[lane] = (double)J.wt[(row - P.row_begin) * n + lane];
            } else {
                float2 *Qj = Qf[lane];
                Qj[0] = make_float2(1.0f, 0.0f);
                for (int b = 1; b < l; ++b) Qj[b] = ff_mul(Qj[c_mono.parent[di][b]], xf[lane * DIM + c_mono.var[di][b]]);
                wf[lane] = make_float2(J.wt[(row - P.row_begin) * n + lane], 0.0f);
            }
        }
        __syncwarp();
        // Gram matrix Q^T Q (FP32, upper triangle), Jacobi scaling
        for (int e = lane; e < l * (l + 1) / 2; e += 32) {
            int a = 0, t = e;
            while (t >= l - a) { t -= l - a; ++a; }
            const int b = a + t;
            float acc = 0.0f;
            for (int j = 0; j < n; ++j) acc = fmaf(q32(j, a), q32(j, b), acc);
            G[a][b] = acc;
            G[b][a] = acc;
        }
        __syncwarp();
        if (lane < l) dsc[lane] = rsqrtf(fmaxf(G[lane][lane], 1e-30f));
        __syncwarp();
        for (int e = lane; e < l * l; e += 32) {
            const int a = e / l, b = e - a * l;
            G[a][b] *= dsc[a] * dsc[b];
        }
        __syncwarp();
        // in-place Gauss-Jordan inverse; lanes (row bl, column half hl)
        bool ok = true;
        const int c0 = 8 * hl, c1 = min(l, c0 + 8);
        for (int c = 0; c < l; ++c) {
            const float piv = G[c][c];
            ok &= piv > 0.0f;
            const float ip = piv > 0.0f ? __frcp_rn(piv) : 0.0f;
            const bool live = bl < l && bl != c;
            const float m = live ? G[bl][c] : 0.0f;
            __syncwarp();
            if (lane < l) {
                const float v = G[c][lane] * ip;
                u[lane] = lane == c ? 0.0f : v;
                G[c][lane] = lane == c ? ip : v;
            }
            __syncwarp();
            if (live) {
                for (int j = c0; j < c1; ++j) G[bl][j] = fmaf(-m, u[j], G[bl][j]);
                if (c >= c0 && c < c1) G[bl][c] = -m * ip;
            }
            __syncwarp();
        }
        // projection passes; lanes (constraint bl, half hl of the nodes)
        const int jh = (n + 1) / 2, j0 = hl * jh, j1 = min(n, j0 + jh);
        for (int pass = 0; pass < 6; ++pass) {
            float c_b = 0.0f, mag = 0.0f;
            if (W64) {
                double cb = 0.0;
                if (bl < l) {
                    if (hl == 0) cb = (double)c_mono.lap[di][bl];
                    for (int j = j0; j < j1; ++j) {
                        cb = fma(-Qd[j][bl], wd[j], cb);
                        mag = fmaf(fabsf((float)Qd[j][bl]), fabsf((float)wd[j]), mag);
                    }
                }
                cb += __shfl_xor_sync(kFull, cb, 16);
                c_b = (float)cb;
            } else {
                float2 cb = make_float2(0.0f, 0.0f);
                if (bl < l) {
                    FFAcc acc(make_float2(hl == 0 ? (float)c_mono.lap[di][bl] : 0.0f, 0.0f));
                    for (int j = j0; j < j1; ++j) {
                        acc.sub(Qf[j][bl], wf[j]);
                        mag = fmaf(fabsf(Qf[j][bl].x), fabsf(wf[j].x), mag);
                    }
                    cb = make_float2(acc.hi, __fadd_rn(acc.lo, __fadd_rn(acc.la, acc.lb)));
                }
                const float oh = __shfl_xor_sync(kFull, cb.x, 16), ol = __shfl_xor_sync(kFull, cb.y, 16);
                const float2 t = ff_two_sum(cb.x, oh);
                c_b = __fadd_rn(t.x, __fadd_rn(t.y, __fadd_rn(cb.y, ol)));
            }
            mag += __shfl_xor_sync(kFull, mag, 16);
            if (bl < l && hl == 0) mag += fabsf((float)c_mono.lap[di][bl]);
            mag = fmaxf(mag, __shfl_xor_sync(kFull, mag, 16));
            // stop when every constraint row holds to 1e-13 of its terms
            // (FP64: 1e-15; both near the rounding level of the sums)
            const float rtol = W64 ? 1e-15f : 1e-13f;
            const bool done = __all_sync(kFull, bl >= l || fabsf(c_b) <= rtol * mag);
            if (done) break;
            // z = D Ginv D c (lanes 0..l-1)
            const float dc = bl < l ? c_b * dsc[bl] : 0.0f;
            float zb = 0.0f;
            for (int a = 0; a < l; ++a) zb = fmaf(G[bl < l ? bl : 0][a], __shfl_sync(kFull, dc, a), zb);
            if (lane < l) zz[lane] = zb * dsc[lane];
            __syncwarp();
            if (lane < n) {
                if (W64) {
                    double corr = 0.0;
                    for (int b = 0; b < l; ++b) corr = fma(Qd[lane][b], (double)zz[b], corr);
                    wd[lane] += corr;
                } else if (pass == 0) {
                    // the first correction is large: its product with Q is compensated
                    FFAcc acc(wf[lane]);
                    for (int b = 0; b < l; ++b) acc.sub(Qf[lane][b], make_float2(-zz[b], 0.0f));
                    wf[lane] = ff_fast_sum(acc.hi, __fadd_rn(acc.lo, __fadd_rn(acc.la, acc.lb)));
                } else {
                    // later ones are small: their FP32 rounding is far below the tolerance
                    float corr = 0.0f;
                    for (int b = 0; b < l; ++b) corr = fmaf(Qf[lane][b].x, zz[b], corr);
                    const float2 t = ff_two_sum(wf[lane].x, corr);
                    wf[lane] = ff_fast_sum(t.x, __fadd_rn(t.y, wf[lane].y));
                }
            }
            __syncwarp();
        }
        // residual check (FP32): r = l_phi - A w, lambda = (Q^T Q)^-1 Q^T r, e = r - Q lambda.
        // Short dependency chains: w in FP32 staged once, two accumulators per
        // sum, the multipliers broadcast from shared memory.
        if (lane < n) rr[lane] = w32(lane);
        __syncwarp();
        float lphi = 0.0f, r_own = 0.0f;
        if (lane < n) {
            float r2 = 0.0f;
#pragma unroll
            for (int a = 0; a < DIM; ++a) r2 = fmaf(x32(lane, a), x32(lane, a), r2);
            float rk2 = r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f;
            for (int i = 3; i < k; i += 2) rk2 *= r2;
            lphi = (float)(k * (k + DIM - 2)) * rk2;
            // (A w)_lane with A = phi(||xi_lane - xi_j||) evaluated on the fly
            float xo[DIM];
#pragma unroll
            for (int a = 0; a < DIM; ++a) xo[a] = x32(lane, a);
            float a0 = 0.0f, a1 = 0.0f;
            int j = 0;
            auto phi_w = [&](int jj) {
                float d2 = 0.0f;
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    const float t = xo[a] - x32(jj, a);
                    d2 = fmaf(t, t, d2);
                }
                return phs32(d2, k) * rr[jj];
            };
            for (; j + 1 < n; j += 2) {
                a0 += phi_w(j);
                a1 += phi_w(j + 1);
            }
            if (j < n) a0 += phi_w(j);
            r_own = lphi - (a0 + a1);
        }
        __syncwarp();
        if (lane < n) rr[lane] = r_own;
        __syncwarp();
        float q0 = 0.0f, q1 = 0.0f;
        if (bl < l) {
            int j = j0;
            for (; j + 1 < j1; j += 2) {
                q0 = fmaf(q32(j, bl), rr[j], q0);
                q1 = fmaf(q32(j + 1, bl), rr[j + 1], q1);
            }
            if (j < j1) q0 = fmaf(q32(j, bl), rr[j], q0);
        }
        float qr = q0 + q1;
        qr += __shfl_xor_sync(kFull, qr, 16);
        if (bl < l && hl == 0) u[bl] = qr * dsc[bl];
        __syncwarp();
        if (lane < l) {
            float l0 = 0.0f, l1 = 0.0f, l2 = 0.0f;
            int a = 0;
            for (; a + 2 < l; a += 3) {
                l0 = fmaf(G[lane][a], u[a], l0);
                l1 = fmaf(G[lane][a + 1], u[a + 1], l1);
                l2 = fmaf(G[lane][a + 2], u[a + 2], l2);
            }
            for (; a < l; ++a) l0 = fmaf(G[lane][a], u[a], l0);
            zz[lane] = (l0 + l1 + l2) * dsc[lane];
        }
        __syncwarp();
        float e = 0.0f;
        if (lane < n) {
            float e0 = 0.0f, e1 = 0.0f;
            int b = 0;
            for (; b + 1 < l; b += 2) {
                e0 = fmaf(q32(lane, b), zz[b], e0);
                e1 = fmaf(q32(lane, b + 1), zz[b + 1], e1);
            }
            if (b < l) e0 = fmaf(q32(lane, b), zz[b], e0);
            e = fabsf(r_own - (e0 + e1));
        }
        float emax = e, lmax = fabsf(lphi);
        for (int o = 16; o; o >>= 1) {
            emax = fmaxf(emax, __shfl_xor_sync(kFull, emax, o));
            lmax = fmaxf(lmax, __shfl_xor_sync(kFull, lmax, o));
        }
        const float rho = emax / fmaxf(lmax, 1e-30f);
        const bool accept = __all_sync(kFull, ok) && rho <= J.tau && !isnan(rho);
        if (J.rho_out && lane == 0) J.rho_out[row - P.row_begin] = rho;
        if (accept) {
            const double inv2 = 1.0 / (s * s);
            if (lane < n) P.vals[0][rb + lane] = (W64 ? wd[lane] : WideFF::to_d(wf[lane])) * inv2;
            if (P.status && lane == 0) P.status[row] = MM_ST_ACCEPTED;
        } else if (lane == 0) {
            const int slot = atomicAdd(J.fb_count, 1);
            J.fb_list[slot] = (int)row;
            if (P.status) P.status[row] = MM_ST_NONCONVERGED;
        }
        __syncwarp();
    }
}

// the FP32 + FP64-refinement solver for stencils the residual check rejected;
// its own stragglers go on to the FP64 solver through a second queue
template <int DIM, int RPL>
__global__ void __launch_bounds__(128) k_surrogate_fallback_mixed(WParams P, int *list2, int *count2) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const MixedLayout Ly = mixed_layout(P.n_max, P.l, 1, DIM);
    char *base = (char *)smem + (size_t)wib * Ly.bytes;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t count = *P.list_count;
    for (int64_t t = gw; t < count; t += nw) {
        const int64_t row = (int64_t)P.list[t];
        if (mixed_row<DIM, RPL, 1>(P, row, base) && lane == 0) {
            const int slot = atomicAdd(count2, 1);
            list2[slot] = (int)row;
        }
        __syncwarp();
    }
}

// the FP64 solver for stencils the residual check rejected
template <int DIM>
__global__ void __launch_bounds__(128) k_surrogate_fallback(WParams P) {
    extern __shared__ double smem[];
    const int wib = threadIdx.x >> 5;
    double *base = smem + (size_t)wib * fp64_warp_doubles(P.M_max, P.pitch64, P.n_max, DIM);
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t count = *P.list_count;
    for (int64_t t = gw; t < count; t += nw) fp64_row<DIM>(P, (int64_t)P.list[t], base, true);
}

// padded parameter layout <-> the plain layout W1 [H x n_in], b1, W2, b2, W3,
// b3, W4 [n_out x H], b4 (row-major [out][in])
void plain_to_padded(const mm_mlp *net, const float *plain, std::vector<float> &pad) {
    pad.assign((size_t)net->np_pad, 0.f);
    const float *q = plain;
    const int ins[4] = {net->n_in, kH, kH, kH}, outs[4] = {kH, kH, kH, net->n_out};
    const int pins[4] = {kKIN, kH, kH, kH};
    for (int l = 0; l < 4; ++l) {
        for (int o = 0; o < outs[l]; ++o)
            for (int i = 0; i < ins[l]; ++i) pad[net->oW[l] + (int64_t)o * pins[l] + i] = *q++;
        for (int o = 0; o < outs[l]; ++o) pad[net->ob[l] + o] = *q++;
    }
}

void padded_to_plain(const mm_mlp *net, const float *pad, float *plain) {
    float *q = plain;
    const int ins[4] = {net->n_in, kH, kH, kH}, outs[4] = {kH, kH, kH, net->n_out};
    const int pins[4] = {kKIN, kH, kH, kH};
    for (int l = 0; l < 4; ++l) {
        for (int o = 0; o < outs[l]; ++o)
            for (int i = 0; i < ins[l]; ++i) *q++ = pad[net->oW[l] + (int64_t)o * pins[l] + i];
        for (int o = 0; o < outs[l]; ++o) *q++ = pad[net->ob[l] + o];
    }
}

int64_t plain_count(int n_in, int n_out) {
    return (int64_t)kH * n_in + kH + 2 * ((int64_t)kH * kH + kH) + (int64_t)n_out * kH + n_out;
}

}  // namespace

int mlp_init_device(mm_ctx *ctx) {
    MonoTable t;
    mono_table_host(t);
    MM_CUDA_CHECK(ctx, cudaMemcpyToSymbol(c_mono, &t, sizeof(t)));
    return MM_OK;
}

extern "C" {

int mm_mlp_create(mm_ctx *ctx, mm_mlp **out, int n_in, int hidden, int n_layers, int n_out,
                  uint64_t seed) {
    if (!ctx || !out) return MM_EBADARG;
    ctx->err.clear();
    *out = nullptr;
    if (hidden != kH || n_layers != 3 || n_in < 1 || n_in > kKIN || n_out < 1 || n_out > kKOUT)
        return mm_fail(ctx, MM_EUNSUPPORTED, "this build supports 3 hidden layers of 256, n_in <= 64, n_out <= 32");
    DeviceGuard g(ctx);
    mm_mlp *net = new mm_mlp();
    net->device = ctx->device;
    net->n_in = n_in;
    net->n_out = n_out;
    net->bmax = 65536;
    int64_t off = 0;
    const int64_t wsz[4] = {(int64_t)kH * kKIN, (int64_t)kH * kH, (int64_t)kH * kH, (int64_t)kKOUT * kH};
    const int64_t bsz[4] = {kH, kH, kH, kKOUT};
    for (int l = 0; l < 4; ++l) {
        net->oW[l] = off;
        off += wsz[l];
        net->ob[l] = off;
        off += bsz[l];
    }
    net->np_pad = off;
    const int64_t B = net->bmax;
    const size_t npart = (size_t)64 * kH * kH;
    size_t bytes_f = sizeof(float) * (size_t)(4 * off + 3 * B * kH + B * kKOUT + 1 + 2 * kKOUT + npart);
    const int64_t wt_elems = 2 * (int64_t)kH * kH + (int64_t)kH * kKOUT;
    size_t bytes_h = sizeof(bf16) * (size_t)(wsz[0] + wsz[1] + wsz[2] + wsz[3] + 3 * B * kH + B * kKIN +
                                             B * kKOUT + 2 * B * kH + wt_elems + 3 * B * kH + B * kKIN +
                                             B * kKOUT + 2 * B * kH + kMlpTcImageElems) + 256;
    char *fb = nullptr, *hb = nullptr;
    if (cudaMalloc(&fb, bytes_f) != cudaSuccess || cudaMalloc(&hb, bytes_h) != cudaSuccess) {
        cudaGetLastError();
        if (fb) cudaFree(fb);
        delete net;
        return mm_fail(ctx, MM_ENOMEM, "MLP buffers");
    }
    float *f = (float *)fb;
    net->p = f; f += off;
    net->g = f; f += off;
    net->am = f; f += off;
    net->av = f; f += off;
    net->Z = f; f += 3 * B * kH;
    net->Y = f; f += B * kKOUT;
    net->loss = f; f += 1;
    net->ymean = f; f += kKOUT;
    net->ystd = f; f += kKOUT;
    net->part = f;
    bf16 *h = (bf16 *)hb;
    net->wb = h; h += wsz[0] + wsz[1] + wsz[2] + wsz[3];
    net->Hb = h; h += 3 * B * kH;
    net->Xb = h; h += B * kKIN;
    net->dY = h; h += B * kKOUT;
    net->dZa = h; h += B * kH;
    net->dZb = h; h += B * kH;
    net->WT = h; h += wt_elems;
    net->HT = h; h += 3 * B * kH;
    net->XT = h; h += B * kKIN;
    net->dYT = h; h += B * kKOUT;
    net->dZTa = h; h += B * kH;
    net->dZTb = h; h += B * kH;
    net->img = h; h += kMlpTcImageElems;     // offsets so far are multiples of 256 elements
    net->tc_err = (int *)h;
    // initial weights: U(-1/sqrt(fan_in), 1/sqrt(fan_in)), zero biases (plain layout)
    std::mt19937_64 rng(seed);
    std::vector<float> plain((size_t)plain_count(n_in, n_out));
    {
        float *q = plain.data();
        const int ins[4] = {n_in, kH, kH, kH}, outs[4] = {kH, kH, kH, n_out};
        for (int l = 0; l < 4; ++l) {
            std::uniform_real_distribution<float> U(-1.f / std::sqrt((float)ins[l]), 1.f / std::sqrt((float)ins[l]));
            for (int64_t i = 0; i < (int64_t)outs[l] * ins[l]; ++i) *q++ = U(rng);
            for (int o = 0; o < outs[l]; ++o) *q++ = 0.f;
        }
    }
    std::vector<float> pad;
    plain_to_padded(net, plain.data(), pad);
    net->h_mean.assign(kKOUT, 0.f);
    net->h_std.assign(kKOUT, 1.f);
    cudaError_t e = cudaMemcpy(net->p, pad.data(), sizeof(float) * off, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(net->am, 0, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMemset(net->av, 0, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMemset(net->tc_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(net->ymean, net->h_mean.data(), sizeof(float) * kKOUT, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(net->ystd, net->h_std.data(), sizeof(float) * kKOUT, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(fb);
        cudaFree(hb);
        delete net;
        return mm_fail(ctx, MM_ECUDA, "MLP init: %s", cudaGetErrorString(e));
    }
    int rc = refresh_bf16(ctx, net);
    if (rc == MM_OK) rc = cudaStreamSynchronize(ctx->stream) == cudaSuccess ? MM_OK : MM_ECUDA;
    if (rc != MM_OK) {
        cudaFree(fb);
        cudaFree(hb);
        delete net;
        return rc;
    }
    *out = net;
    return MM_OK;
}

void mm_mlp_destroy(mm_mlp *net) {
    if (!net) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(net->device);
    cudaDeviceSynchronize();
    cudaFree(net->p);
    cudaFree(net->wb);
    if (prev >= 0) cudaSetDevice(prev);
    delete net;
}

int64_t mm_mlp_num_params(const mm_mlp *net) { return net ? plain_count(net->n_in, net->n_out) : -1; }

int mm_mlp_set_params(mm_ctx *ctx, mm_mlp *net, const float *h_params) {
    if (!ctx || !net || !h_params) return MM_EBADARG;
    DeviceGuard g(ctx);
    std::vector<float> pad;
    plain_to_padded(net, h_params, pad);
    MM_CUDA_CHECK(ctx, cudaMemcpyAsync(net->p, pad.data(), sizeof(float) * pad.size(), cudaMemcpyHostToDevice, ctx->stream));
    int rc = refresh_bf16(ctx, net);
    if (rc != MM_OK) return rc;
    MM_CUDA_CHECK(ctx, cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}

int mm_mlp_get_params(mm_ctx *ctx, const mm_mlp *net, float *h_params) {
    if (!ctx || !net || !h_params) return MM_EBADARG;
    DeviceGuard g(ctx);
    std::vector<float> pad((size_t)net->np_pad);
    MM_CUDA_CHECK(ctx, cudaStreamSynchronize(ctx->stream));
    MM_CUDA_CHECK(ctx, cudaMemcpy(pad.data(), net->p, sizeof(float) * pad.size(), cudaMemcpyDeviceToHost));
    padded_to_plain(net, pad.data(), h_params);
    return MM_OK;
}

int mm_mlp_set_output_scaling(mm_ctx *ctx, mm_mlp *net, const float *h_mean, const float *h_std) {
    if (!ctx || !net || !h_mean || !h_std) return MM_EBADARG;
    DeviceGuard g(ctx);
    for (int c = 0; c < net->n_out; ++c) {
        if (!(h_std[c] > 0)) return mm_fail(ctx, MM_EBADARG, "output scale must be > 0");
        net->h_mean[c] = h_mean[c];
        net->h_std[c] = h_std[c];
    }
    MM_CUDA_CHECK(ctx, cudaMemcpy(net->ymean, net->h_mean.data(), sizeof(float) * kKOUT, cudaMemcpyHostToDevice));
    MM_CUDA_CHECK(ctx, cudaMemcpy(net->ystd, net->h_std.data(), sizeof(float) * kKOUT, cudaMemcpyHostToDevice));
    return MM_OK;
}

}  // extern "C"

namespace {

// Column mean and standard deviation (n - 1 in the denominator, floored at
// 1e-6) of t [B x ncol]: one block per column, two passes, block sums in a
// fixed order.
__global__ void __launch_bounds__(256) k_column_stats(const float *t, int64_t B, int ncol, float *mean,
                                                      float *std) {
    __shared__ double sh[256];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < B; r += blockDim.x) s += (double)t[r * ncol + c];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double mu = sh[0] / (double)B;
    __syncthreads();
    double v = 0.0;
    for (int64_t r = threadIdx.x; r < B; r += blockDim.x) {
        const double d = (double)t[r * ncol + c] - mu;
        v += d * d;
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mean[c] = (float)mu;
        std[c] = fmaxf((float)sqrt(sh[0] / (double)(B > 1 ? B - 1 : 1)), 1e-6f);
    }
}

// Weights of rows [r0, r1) (n entries each) in scaled units, w s^q, as FP32
__global__ void k_scaled_targets(const int64_t *rp, const double *vals, const double *scale, int64_t r0,
                                 int64_t r1, int n, int q, float *out) {
    const int64_t total = (r1 - r0) * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n;
        const int j = (int)(e - i * n);
        const double s = scale[i];
        double f = 1.0;
        for (int t = 0; t < q; ++t) f *= s;
        out[e] = (float)(vals[rp[r0 + i] + j] * f);
    }
}

}  // namespace

extern "C" {

int mm_mlp_fit_output_scaling(mm_ctx *ctx, mm_mlp *net, int64_t B, const float *d_t) {
    if (!ctx || !net || B < 1 || !d_t) return MM_EBADARG;
    ctx->err.clear();
    DeviceGuard g(ctx);
    k_column_stats<<<net->n_out, 256, 0, ctx->stream>>>(d_t, B, net->n_out, net->ymean, net->ystd);
    MM_LAUNCH_CHECK(ctx);
    // host copies (checkpoints carry them)
    MM_CUDA_CHECK(ctx, cudaMemcpyAsync(net->h_mean.data(), net->ymean, sizeof(float) * net->n_out,
                                       cudaMemcpyDeviceToHost, ctx->stream));
    MM_CUDA_CHECK(ctx, cudaMemcpyAsync(net->h_std.data(), net->ystd, sizeof(float) * net->n_out,
                                       cudaMemcpyDeviceToHost, ctx->stream));
    MM_CUDA_CHECK(ctx, cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}

int mm_surrogate_targets(mm_ctx *ctx, const mm_csr_pattern *stencils, int64_t row_begin, int64_t row_end, int n,
                         const double *d_vals, const double *d_scale, int q, float *d_out) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if (!stencils || !stencils->d_row_ptr || row_begin < 0 || row_end < row_begin || row_end > stencils->nrows ||
        n < 1 || q < 0 || q > 4 || !d_vals || !d_scale || !d_out)
        return mm_fail(ctx, MM_EBADARG, "bad arguments to mm_surrogate_targets");
    if (row_end == row_begin) return MM_OK;
    DeviceGuard g(ctx);
    const int64_t total = (row_end - row_begin) * n;
    k_scaled_targets<<<grid1(ctx, total), 256, 0, ctx->stream>>>(stencils->d_row_ptr, d_vals, d_scale, row_begin,
                                                                 row_end, n, q, d_out);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

int mm_mlp_forward(mm_ctx *ctx, mm_mlp *net, int64_t B, const float *d_x, float *d_y) {
    if (!ctx || !net || B < 0 || (B > 0 && (!d_x || !d_y))) return MM_EBADARG;
    ctx->err.clear();
    DeviceGuard g(ctx);
    if (!ctx->mlp_layered) {
        // fused inference on the tensor cores, all rows in one launch
        MlpTcArgs a{};
        a.x = d_x;
        a.n_in = net->n_in;
        a.B = B;
        a.img = net->img;
        a.b1 = net->p + net->ob[0];
        a.b2 = net->p + net->ob[1];
        a.b3 = net->p + net->ob[2];
        a.b4 = net->p + net->ob[3];
        a.ymean = net->ymean;
        a.ystd = net->ystd;
        a.n_out = net->n_out;
        a.y = d_y;
        a.err = net->tc_err;
        return mlp_tc_forward(ctx, a);
    }
    for (int64_t b0 = 0; b0 < B; b0 += net->bmax) {
        const int64_t bs = std::min(net->bmax, B - b0);
        k_pack_x<<<grid1(ctx, bs * kKIN), 256, 0, ctx->stream>>>(d_x + b0 * net->n_in, bs, net->n_in, net->Xb,
                                                                  nullptr, 0);
        MM_LAUNCH_CHECK(ctx);
        int rc = forward(ctx, net, bs);
        if (rc != MM_OK) return rc;
        k_denorm<<<grid1(ctx, bs * net->n_out), 256, 0, ctx->stream>>>(net->Y, bs, net->n_out, net->ymean,
                                                                        net->ystd, d_y + b0 * net->n_out);
        MM_LAUNCH_CHECK(ctx);
    }
    return MM_OK;
}

int mm_mlp_grad(mm_ctx *ctx, mm_mlp *net, int64_t B, const float *d_x, const float *d_t,
                float *h_grads, float *h_loss) {
    if (!ctx || !net || B < 1 || B > net->bmax || !d_x || !d_t) return MM_EBADARG;
    ctx->err.clear();
    DeviceGuard g(ctx);
    MM_CUDA_CHECK(ctx, cudaMemsetAsync(net->loss, 0, sizeof(float), ctx->stream));
    k_pack_x<<<grid1(ctx, B * kKIN), 256, 0, ctx->stream>>>(d_x, B, net->n_in, net->Xb, net->XT, net->bmax);
    MM_LAUNCH_CHECK(ctx);
    int rc = forward(ctx, net, B);
    if (rc == MM_OK) rc = backward(ctx, net, B, d_t);
    if (rc != MM_OK) return rc;
    MM_CUDA_CHECK(ctx, cudaStreamSynchronize(ctx->stream));
    if (h_grads) {
        std::vector<float> pad((size_t)net->np_pad);
        MM_CUDA_CHECK(ctx, cudaMemcpy(pad.data(), net->g, sizeof(float) * pad.size(), cudaMemcpyDeviceToHost));
        padded_to_plain(net, pad.data(), h_grads);
    }
    if (h_loss) MM_CUDA_CHECK(ctx, cudaMemcpy(h_loss, net->loss, sizeof(float), cudaMemcpyDeviceToHost));
    return MM_OK;
}

int mm_mlp_train_step(mm_ctx *ctx, mm_mlp *net, int64_t B, const float *d_x, const float *d_t,
                      float lr, float *d_loss) {
    if (!ctx || !net || B < 1 || B > net->bmax || !d_x || !d_t || !(lr > 0)) return MM_EBADARG;
    ctx->err.clear();
    DeviceGuard g(ctx);
    cudaStream_t st = ctx->stream;
    MM_CUDA_CHECK(ctx, cudaMemsetAsync(net->loss, 0, sizeof(float), st));
    k_pack_x<<<grid1(ctx, B * kKIN), 256, 0, st>>>(d_x, B, net->n_in, net->Xb, net->XT, net->bmax);
    MM_LAUNCH_CHECK(ctx);
    int rc = forward(ctx, net, B);
    if (rc == MM_OK) rc = backward(ctx, net, B, d_t);
    if (rc != MM_OK) return rc;
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)net->step), c2 = 1.f - powf(b2, (float)net->step);
    k_adam<<<grid1(ctx, net->np_pad), 256, 0, st>>>(net->p, net->g, net->am, net->av, net->np_pad, lr, b1, b2,
                                                     1e-8f, c1, c2);
    MM_LAUNCH_CHECK(ctx);
    rc = refresh_bf16(ctx, net);
    if (rc != MM_OK) return rc;
    if (d_loss) MM_CUDA_CHECK(ctx, cudaMemcpyAsync(d_loss, net->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
    return MM_OK;
}

int mm_mlp_save(mm_ctx *ctx, const mm_mlp *net, const char *path) {
    if (!ctx || !net || !path) return MM_EBADARG;
    DeviceGuard g(ctx);
    MM_CUDA_CHECK(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<float> buf((size_t)(3 * net->np_pad));
    MM_CUDA_CHECK(ctx, cudaMemcpy(buf.data(), net->p, sizeof(float) * net->np_pad, cudaMemcpyDeviceToHost));
    MM_CUDA_CHECK(ctx, cudaMemcpy(buf.data() + net->np_pad, net->am, sizeof(float) * net->np_pad, cudaMemcpyDeviceToHost));
    MM_CUDA_CHECK(ctx, cudaMemcpy(buf.data() + 2 * net->np_pad, net->av, sizeof(float) * net->np_pad, cudaMemcpyDeviceToHost));
    FILE *f = fopen(path, "wb");
    if (!f) return mm_fail(ctx, MM_EBADARG, "cannot write %s", path);
    const int hdr[6] = {0x4d4c5031 /* 'MLP1' */, net->n_in, net->H, net->L, net->n_out, net->step};
    fwrite(hdr, sizeof hdr, 1, f);
    fwrite(net->h_mean.data(), sizeof(float), kKOUT, f);
    fwrite(net->h_std.data(), sizeof(float), kKOUT, f);
    fwrite(buf.data(), sizeof(float), buf.size(), f);
    fclose(f);
    return MM_OK;
}

int mm_mlp_load(mm_ctx *ctx, mm_mlp *net, const char *path) {
    if (!ctx || !net || !path) return MM_EBADARG;
    DeviceGuard g(ctx);
    FILE *f = fopen(path, "rb");
    if (!f) return mm_fail(ctx, MM_EBADARG, "cannot read %s", path);
    int hdr[6];
    std::vector<float> mean(kKOUT), sd(kKOUT), buf((size_t)(3 * net->np_pad));
    bool okr = fread(hdr, sizeof hdr, 1, f) == 1 && hdr[0] == 0x4d4c5031 && hdr[1] == net->n_in &&
               hdr[2] == net->H && hdr[3] == net->L && hdr[4] == net->n_out &&
               fread(mean.data(), sizeof(float), kKOUT, f) == (size_t)kKOUT &&
               fread(sd.data(), sizeof(float), kKOUT, f) == (size_t)kKOUT &&
               fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    fclose(f);
    if (!okr) return mm_fail(ctx, MM_EBADARG, "%s is not a checkpoint of this network", path);
    net->step = hdr[5];
    net->h_mean = mean;
    net->h_std = sd;
    MM_CUDA_CHECK(ctx, cudaMemcpy(net->p, buf.data(), sizeof(float) * net->np_pad, cudaMemcpyHostToDevice));
    MM_CUDA_CHECK(ctx, cudaMemcpy(net->am, buf.data() + net->np_pad, sizeof(float) * net->np_pad, cudaMemcpyHostToDevice));
    MM_CUDA_CHECK(ctx, cudaMemcpy(net->av, buf.data() + 2 * net->np_pad, sizeof(float) * net->np_pad, cudaMemcpyHostToDevice));
    MM_CUDA_CHECK(ctx, cudaMemcpy(net->ymean, mean.data(), sizeof(float) * kKOUT, cudaMemcpyHostToDevice));
    MM_CUDA_CHECK(ctx, cudaMemcpy(net->ystd, sd.data(), sizeof(float) * kKOUT, cudaMemcpyHostToDevice));
    int rc = refresh_bf16(ctx, net);
    if (rc == MM_OK) MM_CUDA_CHECK(ctx, cudaStreamSynchronize(ctx->stream));
    return rc;
}

int mm_stencil_features(mm_ctx *ctx, int dim, int64_t N, const double *d_pts,
                        const mm_csr_pattern *stencils, int64_t row_begin, int64_t row_end, int n,
                        int orient, float *d_x, double *d_scale) {
    if (!ctx) return MM_EBADARG;
    ctx->err.clear();
    if ((dim != 2 && dim != 3) || N < 1 || !d_pts || !stencils || !stencils->d_row_ptr ||
        !stencils->d_col || row_begin < 0 || row_end < row_begin || row_end > stencils->nrows ||
        n < 1 || n > 32 || !d_x)
        return mm_fail(ctx, MM_EBADARG, "bad arguments");
    DeviceGuard g(ctx);
    const int64_t rows = row_end - row_begin;
    if (rows == 0) return MM_OK;
    const int blocks = (int)std::min<int64_t>((rows + 3) / 4, (int64_t)ctx->num_sms * 32);
    if (dim == 2) k_features<2><<<blocks, 128, 0, ctx->stream>>>(d_pts, stencils->d_row_ptr, stencils->d_col, row_begin, row_end, n, orient, d_x, d_scale);
    else k_features<3><<<blocks, 128, 0, ctx->stream>>>(d_pts, stencils->d_row_ptr, stencils->d_col, row_begin, row_end, n, orient, d_x, d_scale);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

int mm_rbffd_weights_surrogate(mm_ctx *ctx, mm_mlp *net, int k, int m, int dim, int64_t N,
                               const double *d_pts, const mm_csr_pattern *stencils,
                               int64_t row_begin, int64_t row_end, int n, double tau,
                               int fallback_precision, double *d_lap_vals, int32_t *d_status,
                               float *d_rho) {
    if (!ctx || !net) return MM_EBADARG;
    ctx->err.clear();
    if (dim != 2 || n * dim != net->n_in || n != net->n_out)
        return mm_fail(ctx, MM_EBADARG, "the network expects 2D stencils of %d nodes", net->n_out);
    if (!(tau > 0)) return mm_fail(ctx, MM_EBADARG, "tau must be > 0");
    if (fallback_precision != MM_FP64 && fallback_precision != MM_FP32_IR)
        return mm_fail(ctx, MM_EBADARG, "fallback precision must be MM_FP64 or MM_FP32_IR");
    double *vals[1] = {d_lap_vals};
    WeightsJob job{};
    int rc = weights_job_from_args(ctx, MM_LAP, k, m, dim, N, d_pts, nullptr, stencils, row_begin,
                                   row_end, n, vals, d_status, &job);
    if (rc != MM_OK) return rc;
    DeviceGuard g(ctx);
    const int64_t rows = row_end - row_begin;
    if (rows == 0) return MM_OK;
    WParams P = wparams_from_job(ctx, job);
    if (P.l > 16) return mm_fail(ctx, MM_EUNSUPPORTED, "surrogate projection handles l <= 16");
    const int64_t chunk = net->bmax;
    WsCarve wc;
    const size_t o_x = wc.take<float>((size_t)std::min(rows, chunk) * n * dim);
    const size_t o_y = wc.take<float>((size_t)std::min(rows, chunk) * n);
    const size_t o_cnt = wc.take<int>(2);
    const size_t o_list = wc.take<int>((size_t)rows);
    const size_t o_list2 = wc.take<int>((size_t)rows);
    char *ws = mm_workspace(ctx, wc.off);
    if (!ws) return mm_fail(ctx, MM_ENOMEM, "surrogate workspace of %zu bytes", wc.off);
    float *x = (float *)(ws + o_x), *y = (float *)(ws + o_y);
    int *cnt = (int *)(ws + o_cnt), *list = (int *)(ws + o_list), *list2 = (int *)(ws + o_list2);
    cudaStream_t st = ctx->stream;
    MM_CUDA_CHECK(ctx, cudaMemsetAsync(cnt, 0, 2 * sizeof(int), st));
    for (int64_t r0 = row_begin; r0 < row_end; r0 += chunk) {
        const int64_t r1 = std::min(row_end, r0 + chunk);
        rc = mm_stencil_features(ctx, dim, N, d_pts, stencils, r0, r1, n, 1, x, nullptr);
        if (rc != MM_OK) return rc;
        rc = mm_mlp_forward(ctx, net, r1 - r0, x, y);
        if (rc != MM_OK) return rc;
        ProjParams J{};
        J.P = P;
        J.P.row_begin = r0;
        J.P.row_end = r1;
        J.wt = y;
        J.tau = (float)tau;
        J.fb_list = list;
        J.fb_count = cnt;
        J.rho_out = d_rho ? d_rho + (r0 - row_begin) : nullptr;
        const int blocks = (int)std::min<int64_t>((r1 - r0 + 3) / 4, (int64_t)ctx->num_sms * 32);
        if (ctx->wide64) k_project<2, true><<<blocks, 128, 0, st>>>(J);
        else k_project<2, false><<<blocks, 128, 0, st>>>(J);
        MM_LAUNCH_CHECK(ctx);
    }
    // rejected stencils: FP32 + FP64 refinement first if asked, then FP64
    WParams F = P;
    F.list = list;
    F.list_count = cnt;
    if (fallback_precision == MM_FP32_IR) {
        const MixedLayout Ly = mixed_layout(P.n_max, P.l, 1, dim);
        const int rpl0 = (P.M_max + 31) / 32;
        const void *mk0 = rpl0 <= 1 ? (const void *)k_surrogate_fallback_mixed<2, 1>
                                    : (rpl0 == 2 ? (const void *)k_surrogate_fallback_mixed<2, 2>
                                                 : (const void *)k_surrogate_fallback_mixed<2, 3>);
        const int mw = mm_warps_per_block(ctx, mk0, Ly.bytes, 4);
        const size_t msm = Ly.bytes * mw;
        const int rpl = (P.M_max + 31) / 32;
        const void *mk = rpl <= 1 ? (const void *)k_surrogate_fallback_mixed<2, 1>
                                  : (rpl == 2 ? (const void *)k_surrogate_fallback_mixed<2, 2>
                                              : (const void *)k_surrogate_fallback_mixed<2, 3>);
        MM_CUDA_CHECK(ctx, mm_set_smem(ctx, mk, msm));
        const int mblocks = (int)std::min<int64_t>((rows + mw - 1) / mw, (int64_t)ctx->num_sms * 32);
        if (rpl <= 1) k_surrogate_fallback_mixed<2, 1><<<mblocks, mw * 32, msm, st>>>(F, list2, cnt + 1);
        else if (rpl == 2) k_surrogate_fallback_mixed<2, 2><<<mblocks, mw * 32, msm, st>>>(F, list2, cnt + 1);
        else k_surrogate_fallback_mixed<2, 3><<<mblocks, mw * 32, msm, st>>>(F, list2, cnt + 1);
        MM_LAUNCH_CHECK(ctx);
        F.list = list2;
        F.list_count = cnt + 1;
    }
    const size_t w64 = fp64_warp_doubles(F.M_max, F.pitch64, F.n_max, dim) * sizeof(double);
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(4, (96 * 1024) / w64));
    const size_t sm = w64 * wpb;
    MM_CUDA_CHECK(ctx, mm_set_smem(ctx, (const void *)k_surrogate_fallback<2>, sm));
    const int blocks = (int)std::min<int64_t>((rows + wpb - 1) / wpb, (int64_t)ctx->num_sms * 32);
    k_surrogate_fallback<2><<<blocks, wpb * 32, sm, st>>>(F);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

}  // extern "C"
