/*
 * mm.h -- C ABI of libmm, a GB300 (sm_103a) implementation of the RBF-FD
 * stencil-weight pipeline of strong-form mesh-free methods (Slak & Kosec,
 * "Medusa: a C++ library for solving PDEs using strong form mesh-free
 * methods", arXiv 1912.13282):
 *
 *   nodes -> stencils (mm_knn_stencils, Section 2.1)
 *         -> weights  (mm_rbffd_weights, Section 2.2.2, eq. rbf-system-aug)
 *         -> operator (CSR, one value array per operator, Section 3.3)
 *         -> application to fields (mm_apply_operator, mm_diffuse, Section 2.3.1)
 *
 * Conventions shared by every call:
 *  - Device pointers are named d_*; everything else lives on the host.
 *  - The caller allocates and owns every device buffer it passes.  The
 *    library owns only the workspace inside an mm_ctx.
 *  - Every call is enqueued on the context's CUDA stream and returns without
 *    waiting for the GPU, except where a comment says it synchronises.
 *    Argument checks that need only host data happen before anything is
 *    enqueued.
 *  - Return value: MM_OK (0) or a negative MM_E* code; mm_last_error() then
 *    holds a message.  No C++ exception crosses this boundary.
 *  - Per-node outcomes go to an optional int32 status array (MM_ST_*).
 *  - Indices are 0-based; stencil row i lists node i first (the paper's
 *    I(i)_1 = i becomes col[row_ptr[i]] == i).
 *  - Points are float64, array-of-structures [N x dim], dim in {2, 3}.
 */
#ifndef MM_H
#define MM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ return codes */
#define MM_OK 0
#define MM_EBADARG -1     /* invalid argument (see mm_last_error)              */
#define MM_ENOMEM -2      /* workspace allocation failed                       */
#define MM_ECUDA -3       /* a CUDA runtime call failed                        */
#define MM_EUNSUPPORTED -4 /* a size or option outside what this build handles */
#define MM_ENOCONV -5     /* an iterative solve stopped without converging     */
#define MM_ESINGULAR -6   /* a zero pivot in a factorisation                   */

/* ------------------------------------------------------- per-node statuses */
#define MM_ST_OK 0
#define MM_ST_SINGULAR 1      /* pivot <= M*u*max|K|: weights set to 0         */
#define MM_ST_NONCONVERGED 2  /* refinement did not converge (then fallback)   */
#define MM_ST_FALLBACK 3      /* mixed/surrogate path: solved by the FP64 path */
#define MM_ST_BADARG 4        /* bad stencil row (size, centre, index)         */
#define MM_ST_DUPLICATE 5     /* kNN: another node coincides with this one     */
#define MM_ST_ACCEPTED 6      /* surrogate: projected prediction accepted      */

/* ------------------------------------------------------------ operator bits */
#define MM_LAP 1u   /* Laplacian                                   */
#define MM_DX 2u    /* d/dx                                        */
#define MM_DY 4u    /* d/dy                                        */
#define MM_DZ 8u    /* d/dz (dim 3)                                */
#define MM_DN 16u   /* d/dn = sum_a n_a d/dx_a with the node normal */
/* second derivatives d2/dx_a dx_b (z ones need dim 3); the batched call
 * (mm_rbffd_weights_batched) takes at most 5 operator bits per class */
#define MM_DXX 32u
#define MM_DXY 64u
#define MM_DYY 128u
#define MM_DXZ 256u
#define MM_DYZ 512u
#define MM_DZZ 1024u

/* ------------------------------------------------------------ precisions */
#define MM_FP64 0     /* plain FP64 solve                                      */
#define MM_FP32_IR 1  /* FP32 Gauss-Jordan inverse + FP64-residual iterative
                         refinement (at least two steps); condition-number /
                         non-convergence fallback to FP64                      */

/* ------------------------------------------------------------ kNN methods */
#define MM_KNN_AUTO 0
#define MM_KNN_BRUTE 1  /* exhaustive scan of all nodes                     */
#define MM_KNN_GRID 2   /* uniform-grid binning + ring search (exact)       */

/* ------------------------------------------------------------ ctx options */
#define MM_OPT_IR_TOL 1        /* IR stop: estimated rel. forward error (1e-9) */
#define MM_OPT_IR_MAX_STEPS 2  /* IR residual evaluations at most (4); below 2
                                  every stencil goes to the FP64 solve        */
#define MM_OPT_KAPPA_MAX 3     /* fallback if kappa1 * u32 exceeds (0.1);
                                  kappa1 = ||K||_1 ||K^-1||_1, the second norm
                                  taken exactly from the FP32 inverse         */
#define MM_OPT_WIDE 4          /* arithmetic of the refinement residuals and of
                                  the surrogate's consistency projection:      */
#define MM_WIDE_FF 0           /*   double-FP32 pairs (~48-bit significand,
                                    compensated sums on the FP32 pipe; default) */
#define MM_WIDE_FP64 1         /*   native FP64                                */
#define MM_OPT_MLP_INFER 5     /* MLP inference (mm_mlp_forward, surrogate):    */
#define MM_MLP_FUSED 0         /*   one fused tensor-core kernel (default)     */
#define MM_MLP_LAYERED 1       /*   layer-by-layer GEMMs (the training path)   */
#define MM_OPT_GJ 6            /* storage of the FP32 Gauss-Jordan inverse:     */
#define MM_GJ_AUTO 0           /*   rows in registers for systems of 33..48    */
                               /*   unknowns (M_max rounded up to 40 or 48),   */
                               /*   shared memory otherwise (default)          */
#define MM_GJ_SHARED 1         /*   shared memory for every size (same result) */

typedef struct mm_ctx mm_ctx;

/*
 * Create a context on CUDA device `device`, enqueuing on `cuda_stream` (a
 * cudaStream_t, NULL = legacy default stream).  *out receives the context.
 * Errors: MM_EBADARG (out NULL), MM_ECUDA (device not usable).
 */
int mm_ctx_create(mm_ctx **out, int device, void *cuda_stream);

/* Free the context and its workspace (synchronises its stream).  NULL is a no-op. */
void mm_ctx_destroy(mm_ctx *ctx);

/* Switch the stream later calls enqueue on. */
int mm_ctx_set_stream(mm_ctx *ctx, void *cuda_stream);

/* Set a tuning option (MM_OPT_*).  Errors: MM_EBADARG for unknown keys or
 * out-of-range values. */
int mm_ctx_set_option(mm_ctx *ctx, int key, double value);

/* Message of the last failed call on this context ("" if none).  The string
 * is owned by the context and valid until its next call. */
const char *mm_last_error(const mm_ctx *ctx);

/* Bytes of device workspace the context holds now, over its buffers (0
 * until a call needed one; they only grow, and are freed by mm_ctx_destroy);
 * -1 for NULL. */
int64_t mm_ctx_workspace_bytes(const mm_ctx *ctx);

/* -------------------------------------------------------------- stencils */
/*
 * One block of query nodes for mm_knn_stencils: nodes q_begin..q_end-1 get
 * stencils of n nodes, written row-major to d_idx[(q - q_begin) * n + j].
 */
typedef struct {
    int64_t q_begin, q_end;
    int32_t n;
    int32_t *d_idx;
} mm_knn_range;

/*
 * Stencils of the n closest nodes (Section 2.1, "some number of closest
 * neighbours"; each node in its own stencil, first).  Candidates are all N
 * nodes of d_pts [N x dim].  Row q lists q, then the n-1 other nodes in
 * ascending (squared distance computed in FP64 as sum_a (x_a - c_a)^2 without
 * fused multiply-add, node index).  This ranking is exact, so results are
 * bit-identical to any other exact implementation of it.
 *   method   MM_KNN_GRID (binned ring search), MM_KNN_BRUTE, or MM_KNN_AUTO.
 *   d_status optional [N] int32: MM_ST_DUPLICATE where another node
 *            coincides with the query, else MM_ST_OK (entries of nodes in
 *            no range untouched).
 * Requirements: 1 <= n <= 64, n <= N, N < 2^31, finite coordinates.
 * Errors: MM_EBADARG, MM_EUNSUPPORTED (n > 64), MM_ENOMEM, MM_ECUDA.
 */
int mm_knn_stencils(mm_ctx *ctx, int dim, int64_t N, const double *d_pts, int nranges,
                    const mm_knn_range *ranges, int method, int32_t *d_status);

/*
 * Balanced stencils (Section 3.1: FindBalancedSupport "also ensures that
 * stencils are balanced around the central node"; the paper gives no rule,
 * this is the library's reading).  For every query node c of a range: the K
 * closest nodes (the ranking of mm_knn_stencils, c first) are the candidates;
 * a candidate j lies in the orthant o(j) = sum_a 2^a [x_j,a - x_c,a < 0]
 * (2^dim orthants); each orthant contributes its first (n - 1) / 2^dim
 * candidates (integer division) in ranking order; the remaining slots go to
 * the closest candidates not taken.  Row q lists c, then the n - 1 taken
 * candidates in ranking order.  With K = n the result is mm_knn_stencils'.
 *   ranges   as mm_knn_stencils (n per range), 1 <= n <= K.
 *   K        candidates per query, n <= K <= 64, K <= N.
 *   d_status optional: as mm_knn_stencils.
 * Uses a second context buffer of (query rows) x K int32 for the candidates.
 * Errors: MM_EBADARG, MM_EUNSUPPORTED (K > 64), MM_ENOMEM, MM_ECUDA.
 */
int mm_balanced_stencils(mm_ctx *ctx, int dim, int64_t N, const double *d_pts, int nranges,
                         const mm_knn_range *ranges, int K, int method, int32_t *d_status);

/* ------------------------------------------------------------ CSR pattern */
/* Device CSR stencil pattern: row i spans col[row_ptr[i] .. row_ptr[i+1]-1]. */
typedef struct {
    int64_t nrows;
    int64_t nnz;
    const int64_t *d_row_ptr;  /* [nrows + 1] */
    const int32_t *d_col;      /* [nnz]       */
} mm_csr_pattern;

/* ---------------------------------------------------------------- weights */
/*
 * RBF-FD weights with polyharmonic splines phi(r) = r^k and monomials of
 * total degree <= m (Section 2.2.2, eq. rbf-system-aug): for every row i in
 * [row_begin, row_end) of the stencil pattern, with x_c the centre,
 * s = max_j ||x_j - x_c|| and xi_j = (x_j - x_c)/s,
 *     [A Q; Q^T 0] [w; lambda] = [l_phi; l_q],
 *     A_ij = ||xi_i - xi_j||^k, Q_ib = q_b(xi_i),
 * l_phi, l_q = the operator applied to each basis function at xi = 0; the
 * stored weights are w / s^q (q = 2 for MM_LAP and second derivatives, 1 for
 * first derivatives).
 *
 *   ops        bitmask of MM_LAP | MM_DX | MM_DY | MM_DZ | MM_DN and the
 *              second derivatives MM_DXX .. MM_DZZ (these need m >= 2); more
 *              than 5 bits are computed in launches of at most 5 columns.
 *   k, m       odd k in {3, 5, 7}; 0 <= m <= 6; l = C(m + dim, dim).
 *   d_pts      [N x dim] nodes; d_normals [N x dim] unit normals (needed
 *              only with MM_DN; may be NULL otherwise).
 *   stencils   rows are nodes; rows in range must have 1 <= n_i <= n_max,
 *              col[row_ptr[i]] == i and indices in [0, N).
 *   n_max      largest stencil size in the range; n_max + l <= 96.
 *   precision  MM_FP64 or MM_FP32_IR.
 *   d_vals     HOST array of device pointers, one per set bit of ops in bit
 *              order; d_vals[r][row_ptr[i] + j] receives the weight of node j
 *              of row i.  Several entries may alias the same array when
 *              different row ranges write different operators into it.
 *   d_status   optional [nrows] int32 (MM_ST_OK, MM_ST_SINGULAR, MM_ST_FALLBACK,
 *              MM_ST_BADARG).  Singular or bad rows get zero weights.
 * Errors: MM_EBADARG, MM_EUNSUPPORTED, MM_ENOMEM, MM_ECUDA.
 */
int mm_rbffd_weights(mm_ctx *ctx, unsigned ops, int k, int m, int dim, int64_t N,
                     const double *d_pts, const double *d_normals,
                     const mm_csr_pattern *stencils, int64_t row_begin, int64_t row_end,
                     int n_max, int precision, double *const *d_vals, int32_t *d_status);

/* ------------------------------------------------------- GWLS weights */
#define MM_SCALE_FARTHEST 0   /* s = largest distance from the centre in the stencil */
#define MM_SCALE_NEAREST 1    /* s = distance to the closest other node            */

/*
 * Generalized weighted least squares weights (Section 2.2.1): for every row i
 * in [row_begin, row_end), with x_c the centre, xi_j = (x_j - x_c)/s, the
 * monomials b of total degree <= m (graded order), B_jb = b(xi_j) and
 * W = diag(omega(xi_j)), omega(x) = exp(-|x|^2 / sigma^2), the weights are
 *     w^T = (L b)(0)^T (W B)^+ W,
 * i.e. w = W y with y the minimum-norm solution of (W B)^T y = (L b)(0);
 * stored as w / s^q like mm_rbffd_weights.  Computed in FP64 by a Householder
 * QR of W B (one warp per stencil).
 *   ops, m, dim, N, d_pts, d_normals, stencils, row range, d_vals, d_status:
 *              as mm_rbffd_weights (no k; n_max <= 64).
 *   sigma      Gaussian width, finite and > 0 (in scaled units).
 *   scale      MM_SCALE_FARTHEST or MM_SCALE_NEAREST (the paper's example
 *              setup scales to the closest node).
 * Rows with fewer nodes than monomials, or with W B of numerically deficient
 * rank, get MM_ST_SINGULAR and zero weights; bad rows (index out of range,
 * centre not first, n_i outside [1, n_max], a single node with
 * MM_SCALE_NEAREST) get MM_ST_BADARG and zero weights.
 * Errors: MM_EBADARG, MM_EUNSUPPORTED (n_max > 64), MM_ECUDA.
 */
int mm_wls_weights(mm_ctx *ctx, unsigned ops, int m, double sigma, int scale, int dim, int64_t N,
                   const double *d_pts, const double *d_normals, const mm_csr_pattern *stencils,
                   int64_t row_begin, int64_t row_end, int n_max, double *const *d_vals,
                   int32_t *d_status);

/* ----------------------------------------------- batched (mixed) classes */
/*
 * One stencil class for mm_rbffd_weights_batched: the arguments of one
 * mm_rbffd_weights call.  Classes may differ in dimension, node set, stencil
 * size, degree, PHS exponent and operators.
 */
typedef struct {
    unsigned ops;                 /* MM_LAP | MM_DX | ...                            */
    int k, m, dim;
    int64_t N;                    /* nodes of d_pts                                  */
    const double *d_pts;          /* [N x dim]                                       */
    const double *d_normals;      /* [N x dim] or NULL without MM_DN                 */
    mm_csr_pattern stencils;      /* device CSR pattern (by value)                   */
    int64_t row_begin, row_end;   /* rows of this class                              */
    int n_max;                    /* largest stencil size in the rows                */
    double *d_vals[5];            /* one array per set bit of ops, in bit order      */
    int32_t *d_status;            /* [stencils.nrows] or NULL                        */
} mm_weights_class;

/* Launch shape of the persistent batched kernel. */
typedef struct {
    int warps_per_block;   /* stencils in flight per CTA (1..8)                      */
    int blocks_per_sm;     /* resident CTAs per SM; grid = blocks_per_sm * SM count  */
    int chunk_rows;        /* rows per work item taken from the queue                */
} mm_launch_config;

/*
 * Weights of several stencil classes in ONE persistent launch (plus one
 * FP64 launch for stencils the FP32 solver hands over).  The paper computes
 * the weights of all nodes in one OpenMP loop (Section 5); here every warp
 * repeatedly takes a chunk of rows of some class from an atomic work queue,
 * so classes of very different cost share the GPU without a tail per class.
 * Per class the results equal those of mm_rbffd_weights with the same
 * arguments and precision (bit for bit; classes with 2 or 3 operators run on
 * the 4-column solver whose spare column has a zero right-hand side).
 *   nclasses   1..96 classes per call.
 *   precision  MM_FP64 or MM_FP32_IR.  With MM_FP32_IR, classes with all
 *              five operators are processed by separate launches in this call.
 *   config     launch shape, or NULL: the context's tuned shape for this batch
 *              signature (mm_autotune_batched), else a default.
 * Graph capture: the call enqueues only kernels and memsets; class
 * descriptors travel as a kernel parameter.  Make one call with the same
 * classes before capturing it, so the context workspace is already large
 * enough (growing it would allocate).
 * Errors: as mm_rbffd_weights; MM_EBADARG for nclasses out of range.
 */
int mm_rbffd_weights_batched(mm_ctx *ctx, int nclasses, const mm_weights_class *classes,
                             int precision, const mm_launch_config *config);

/*
 * Autotuner for mm_rbffd_weights_batched: times candidate launch shapes
 * (warps per CTA, CTAs per SM, rows per work item) on the first
 * `sample_rows` rows of every class (0 = 16384) and stores the fastest in the
 * context under the batch signature (dims, stencil sizes, degrees, operator
 * counts, precision); later calls with config == NULL use it.  Writes weights
 * of the sampled rows as a side effect.  Synchronises; not for use inside a
 * stream capture.  *best and *best_ms (either may be NULL) receive the winner.
 */
int mm_autotune_batched(mm_ctx *ctx, int nclasses, const mm_weights_class *classes, int precision,
                        int64_t sample_rows, mm_launch_config *best, double *best_ms);

/* Save / load the context's tuned launch shapes as a text table (one line per
 * batch signature).  Loading merges into the context's table. */
int mm_tile_table_save(const mm_ctx *ctx, const char *path);
int mm_tile_table_load(mm_ctx *ctx, const char *path);

/*
 * Allocation-free variant of mm_rbffd_weights with precision MM_FP32_IR.
 * The paper has no counterpart: this exists for callers that cannot allocate
 * device memory when they call in -- e.g. a process whose memory pool has
 * already reserved the GPU's memory (a cudaMalloc there fails or fragments
 * it), or a latency-critical loop where a cudaFree would synchronise the
 * whole device.  The regular call may grow the context workspace to hold the
 * queue of stencils handed from the FP32 solve to the FP64 solve; this one
 * keeps that queue in a fixed array of 1 + 2^20 int32 (4 MiB) inside the
 * library image, present on every GPU that loads the library until exit.
 *   Same arguments and results as mm_rbffd_weights(..., MM_FP32_IR, ...).
 *   At most 2^20 rows per call (row_end - row_begin); larger ranges fail
 *   with MM_EUNSUPPORTED before anything is enqueued.
 *   Calls no cudaMalloc, cudaFree or allocating library routine, and never
 *   touches the context workspace (mm_ctx_workspace_bytes stays as it was).
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) and caches it; make that first call before any
 *   stream capture.  Only a successful lookup is cached (a failed one is
 *   retried by the next call).  The cached address is that of the device's
 *   primary context: after cudaDeviceReset it is stale, so do not call this
 *   entry point again in a process that reset the device.
 *   Every call shares the array, which keeps the last call's contents; the
 *   call clears the queue length on its stream first.  Calls whose GPU work
 *   overlaps (different streams, or different contexts on one device) race on
 *   the queue: serialise them.
 * Errors: as mm_rbffd_weights; MM_ECUDA if the address lookup fails.
 */
int mm_rbffd_weights_ir_noalloc(mm_ctx *ctx, unsigned ops, int k, int m, int dim, int64_t N,
                                const double *d_pts, const double *d_normals,
                                const mm_csr_pattern *stencils, int64_t row_begin,
                                int64_t row_end, int n_max, double *const *d_vals,
                                int32_t *d_status);

/* ------------------------------------------------------ operator application */
/*
 * y = alpha * L u + beta * y with L the CSR operator (stencils, d_vals):
 * (L u)_i = sum_j vals[row_ptr[i] + j] * u[col[row_ptr[i] + j]], the explicit
 * evaluation w^T u_I(i) of Section 2.3.1.  d_u [ncols], d_y [nrows]; d_y must
 * not alias d_u.  beta == 0 ignores the old contents of d_y.
 * Errors: MM_EBADARG, MM_ECUDA.
 */
int mm_apply_operator(mm_ctx *ctx, const mm_csr_pattern *stencils, const double *d_vals,
                      const double *d_u, double alpha, double beta, double *d_y);

/*
 * `steps` explicit Euler steps u <- u + dt * L u (eq. exp-start .. exp-end)
 * on rows with d_fixed[i] == 0; rows with d_fixed[i] != 0 keep their value
 * (Dirichlet nodes).  The operator must be square (nrows == length of d_u).
 * d_work [nrows] float64 is caller-owned scratch.  The final field is in d_u.
 * Errors: MM_EBADARG, MM_ECUDA.
 */
int mm_diffuse(mm_ctx *ctx, const mm_csr_pattern *stencils, const double *d_vals,
               const uint8_t *d_fixed, double dt, int steps, double *d_u, double *d_work);

/* Row kinds of mm_diffuse_bc */
#define MM_ROW_INTERNAL 0
#define MM_ROW_DIRICHLET 1
#define MM_ROW_NEUMANN 2

/*
 * mm_diffuse with Neumann nodes (eq. exp-end of Section 2.3.1).  Every step
 * uses the previous step's field:
 *   d_kind[i] == MM_ROW_INTERNAL:  u_i <- u_i + dt (L u)_i
 *   d_kind[i] == MM_ROW_NEUMANN:   row i of the operator holds the node's
 *       d/dn weights, centre first (as mm_rbffd_weights writes them), and
 *       u_i <- (g_i - sum_{j >= 2} w_ij u_{I(i,j)}) / w_i1
 *   any other kind (MM_ROW_DIRICHLET): u_i kept.
 * d_g [nrows] Neumann data g_n (NULL: 0), constant in time; it must not alias
 * d_u or d_work.  A centre weight of 0 gives a non-finite value.  The update
 * divides by the centre d/dn weight, so with one-sided stencils whose centre
 * weight is small against the others, coupled Neumann nodes amplify errors
 * from step to step.  A sufficient condition for them not to: over the
 * Neumann rows i, max_i sum_{j >= 2, node j Neumann} |w_ij| / |w_i1| < 1 (the
 * Neumann values' update is then a contraction in the max norm); on the
 * one-sided stencils around holes of a disk this ratio can exceed 10^2, and
 * the scheme is then unstable whatever dt.  Errors: as mm_diffuse.
 */
int mm_diffuse_bc(mm_ctx *ctx, const mm_csr_pattern *stencils, const double *d_vals,
                  const uint8_t *d_kind, const double *d_g, double dt, int steps, double *d_u,
                  double *d_work);

/*
 * General second-order operator from derivative weights (eq. gen-op,
 * Section 3.3): for the rows i in [row_begin, row_end),
 *     d_out[e] = sum_t a_t(i) * d_terms[t][e]   for each entry e of row i,
 * a_t(i) = d_coef[t][i] (per-node coefficient, [nrows]) or 1 where d_coef (a
 * HOST array of nterms device pointers, or NULL for all 1) has NULL.  The
 * terms are value arrays of the same CSR pattern, e.g. the weights of d/dx_a
 * and d2/dx_a dx_b; d_out may be one of them.  Entries outside the rows are
 * not written.  Requirements: 1 <= nterms <= 10.  Errors: MM_EBADARG, MM_ECUDA.
 */
int mm_combine_operators(mm_ctx *ctx, const mm_csr_pattern *stencils, int64_t row_begin, int64_t row_end,
                         int nterms, const double *const *d_terms, const double *const *d_coef,
                         double *d_out);

/* ----------------------------------------------------------- implicit solve */
/*
 * The implicit discretisation of Section 2.3.2: every node's equation becomes
 * one sparse row -- interior nodes the weights of the PDE's operator (e.g.
 * the Laplacian of the Poisson problem of Section 5), Dirichlet nodes the
 * identity, Neumann nodes their d/dn weights -- and M u = r is solved with
 * BiCGSTAB preconditioned by an incomplete LU factorisation (the paper's
 * benchmark uses ILUT; this library uses ILU(0), the incomplete LU on the
 * pattern of M, no dropping and no fill-in).
 *
 * Matrices of these calls are square CSR (nrows == number of unknowns, at
 * most 64 entries per row, column indices in [0, nrows)) on the device.
 */

/*
 * Assembles the implicit matrix from stencil rows: row i's entries sorted by
 * column into d_col_out / d_vals_out (same row pointers as `stencils`, which
 * must list node i in row i); rows with d_kind[i] == MM_ROW_DIRICHLET become
 * the identity row on the same pattern (1 on the diagonal, explicit zeros
 * elsewhere), every other row keeps the values of d_vals (interior: the
 * operator's weights, MM_ROW_NEUMANN: the d/dn weights).  d_kind NULL: no
 * Dirichlet rows.  The right-hand side is the caller's (f, the Dirichlet
 * values, g_n).  Synchronises (to report bad rows).
 * Errors: MM_EBADARG (a row without its own index, a repeated or out-of-range
 * column), MM_EUNSUPPORTED (a row of more than 64 entries), MM_ECUDA.
 */
int mm_implicit_assemble(mm_ctx *ctx, const mm_csr_pattern *stencils, const double *d_vals,
                         const uint8_t *d_kind, int32_t *d_col_out, double *d_vals_out);

/*
 * ILU(0) factors of the sorted matrix A (rows with increasing columns and a
 * diagonal entry): d_factors [nnz] receives L (unit diagonal implied, strictly
 * lower entries) and U (the rest) on A's pattern, so that (L U)_ij = A_ij for
 * every (i, j) of the pattern; d_diag [nrows] the position of each diagonal
 * entry.  Rows are eliminated in the plain row-by-row order with IEEE
 * roundings and no fused multiply-add, so the factors equal those of the
 * sequential algorithm bit for bit.  d_factors may equal d_vals (in place).
 * Synchronises.  Errors: MM_EBADARG (unsorted row, missing diagonal),
 * MM_ESINGULAR (a zero pivot), MM_EUNSUPPORTED (a row longer than 64),
 * MM_ECUDA (including a dependency wait that timed out).
 */
int mm_ilu0(mm_ctx *ctx, const mm_csr_pattern *A, const double *d_vals, double *d_factors,
            int64_t *d_diag);

/*
 * x = (L U)^-1 b with the factors of mm_ilu0 on the same pattern: forward
 * then back substitution, each row waiting only for the unknowns it needs
 * (no level sets).  d_b and d_x are [nrows], distinct.  Synchronises.
 * Errors: MM_EBADARG, MM_ECUDA.
 */
int mm_ilu0_solve(mm_ctx *ctx, const mm_csr_pattern *A, const double *d_factors,
                  const int64_t *d_diag, const double *d_b, double *d_x);

/*
 * BiCGSTAB (van der Vorst's algorithm) for A x = b, preconditioned by the
 * ILU(0) factors d_factors / d_diag of A (NULL: no preconditioner), starting
 * from the d_x given; stops when the recursively updated residual satisfies
 * ||r||_2 <= tol ||b||_2, on a breakdown (rho or omega or r^.v equal to 0) or
 * after maxit iterations.  All scalars stay on the GPU; the host looks at
 * them every 16 iterations (later iterations of that batch do nothing).
 * *iters and *relres (either may be NULL) receive the iterations taken and
 * the final relative residual.  Synchronises.
 * Errors: MM_ENOCONV (breakdown or iteration limit; d_x holds the last
 * iterate), MM_EBADARG, MM_ENOMEM, MM_ECUDA.
 */
int mm_bicgstab(mm_ctx *ctx, const mm_csr_pattern *A, const double *d_vals,
                const double *d_factors, const int64_t *d_diag, const double *d_b, double *d_x,
                double tol, int maxit, int *iters, double *relres);

/* ------------------------------------------------- learned surrogate (MLP) */
/*
 * A GELU multilayer perceptron n_in -> 256 -> 256 -> 256 -> n_out that maps
 * the scaled offsets of a 2D stencil (features, see mm_stencil_features) to
 * its scaled Laplacian weights.  No counterpart in the paper: it is trained
 * on weights this library computes.  BF16 weights and activations, FP32
 * accumulation on the tensor cores, FP32 master parameters updated by Adam.
 * Parameters in the plain layout W1 [256 x n_in], b1, W2 [256 x 256], b2,
 * W3, b3, W4 [n_out x 256], b4 (row-major [out][in]) as FP32 host arrays.
 * The network predicts (y - mean)/std per output (mm_mlp_set_output_scaling).
 */
typedef struct mm_mlp mm_mlp;

/* Create with U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from `seed`, zero
 * biases.  Supported: hidden == 256, n_layers == 3, n_in <= 64, n_out <= 32.
 * The network owns its device buffers (params, Adam state, activations for
 * 65536 rows).  Errors: MM_EUNSUPPORTED, MM_ENOMEM, MM_ECUDA. */
int mm_mlp_create(mm_ctx *ctx, mm_mlp **out, int n_in, int hidden, int n_layers, int n_out,
                  uint64_t seed);
void mm_mlp_destroy(mm_mlp *net);
int64_t mm_mlp_num_params(const mm_mlp *net);
/* Host parameter arrays in the plain layout (mm_mlp_num_params floats); both synchronise. */
int mm_mlp_set_params(mm_ctx *ctx, mm_mlp *net, const float *h_params);
int mm_mlp_get_params(mm_ctx *ctx, const mm_mlp *net, float *h_params);
/* Output scaling: targets are learned as (y - mean[c]) / std[c]; host arrays [n_out]. */
int mm_mlp_set_output_scaling(mm_ctx *ctx, mm_mlp *net, const float *h_mean, const float *h_std);
/* The same from training targets d_t [B x n_out] (device): per column the mean
 * and the standard deviation (B - 1 in the denominator, at least 1e-6), two
 * passes in a fixed order.  Synchronises. */
int mm_mlp_fit_output_scaling(mm_ctx *ctx, mm_mlp *net, int64_t B, const float *d_t);
/* Training targets of the surrogate: the weights of rows [row_begin,
 * row_end) (n entries each) in scaled units, d_out[(i - row_begin) n + j] =
 * d_vals[row_ptr[i] + j] * d_scale[i - row_begin]^q as FP32 (q = 2 for the
 * Laplacian; d_scale from mm_stencil_features).  Errors: MM_EBADARG. */
int mm_surrogate_targets(mm_ctx *ctx, const mm_csr_pattern *stencils, int64_t row_begin, int64_t row_end, int n,
                         const double *d_vals, const double *d_scale, int q, float *d_out);
/* d_y [B x n_out] = network(d_x [B x n_in]) (FP32 in and out, scaling undone).
 * By default one fused tensor-core kernel (tcgen05, activations kept on chip);
 * MM_OPT_MLP_INFER = MM_MLP_LAYERED runs the layer-by-layer training path.  A
 * fused launch whose internal waits time out writes NaN for the affected rows
 * (never observed; it guards against a hang). */
int mm_mlp_forward(mm_ctx *ctx, mm_mlp *net, int64_t B, const float *d_x, float *d_y);
/* One Adam step (lr; beta 0.9/0.999, eps 1e-8) on the mean squared error over
 * B <= 65536 rows of targets d_t [B x n_out]; d_loss (device, optional)
 * receives the loss before the step. */
int mm_mlp_train_step(mm_ctx *ctx, mm_mlp *net, int64_t B, const float *d_x, const float *d_t,
                      float lr, float *d_loss);
/* Gradient of the same loss w.r.t. the parameters, plain layout, into host
 * h_grads (no update); h_loss optional.  Synchronises. */
int mm_mlp_grad(mm_ctx *ctx, mm_mlp *net, int64_t B, const float *d_x, const float *d_t,
                float *h_grads, float *h_loss);
/* Checkpoint: FP32 parameters, Adam state, step count and output scaling. */
int mm_mlp_save(mm_ctx *ctx, const mm_mlp *net, const char *path);
int mm_mlp_load(mm_ctx *ctx, mm_mlp *net, const char *path);

/*
 * Features of stencils: for rows [row_begin, row_end) of n nodes each,
 * d_x[(i - row_begin) * n * dim + j * dim + a] = (x_j - x_c)_a / s with
 * s = max_j ||x_j - x_c|| (FP32), d_scale[i - row_begin] = s (optional).
 * orient != 0 (2D): offsets in the stencil's canonical frame -- rotated so
 * node 1 lies on +x, mirrored so node 2 has y >= 0 (Laplacian weights are
 * invariant under both).  The surrogate path uses orient = 1.  n <= 32.
 */
int mm_stencil_features(mm_ctx *ctx, int dim, int64_t N, const double *d_pts,
                        const mm_csr_pattern *stencils, int64_t row_begin, int64_t row_end, int n,
                        int orient, float *d_x, double *d_scale);

/*
 * Laplacian weights through the surrogate: features -> network -> scaled
 * weights w~; exact FP64 least-norm projection onto the monomial rows of
 * eq. rbf-system-aug, (Q^T Q) z = l_q - Q^T w~, w = w~ + Q z (FP32 Cholesky of
 * the Jacobi-scaled Gram matrix, FP64 constraint residuals until they hold to
 * 1e-15 relative); checked against the other rows: rho = ||r - Q lambda||_inf /
 * ||l_phi||_inf with r = l_phi - A w and lambda the least-squares multipliers
 * (FP32).  rho <= tau: weights w / s^2 stored, status MM_ST_ACCEPTED;
 * otherwise the stencil is solved by the method itself: with
 * fallback_precision MM_FP64 by the FP64 solve (status MM_ST_FALLBACK), with
 * MM_FP32_IR by the FP32 + FP64-refinement solve (status MM_ST_OK), which
 * hands its own stragglers to the FP64 solve.  The network input is the
 * canonical-frame features (mm_stencil_features, orient = 1).  2D only,
 * n == n_out of the network, l <= 16.  d_rho (optional, [rows]) receives rho.
 */
int mm_rbffd_weights_surrogate(mm_ctx *ctx, mm_mlp *net, int k, int m, int dim, int64_t N,
                               const double *d_pts, const mm_csr_pattern *stencils,
                               int64_t row_begin, int64_t row_end, int n, double tau,
                               int fallback_precision, double *d_lap_vals, int32_t *d_status,
                               float *d_rho);

/* ------------------------------------------------------- range partition */
/*
 * Splitting one node set over several GPUs.  The weights of every node come
 * from its own stencil (Section 2.2), so the node set splits into contiguous
 * ranges of a space-filling order, one per GPU; each GPU also holds the halo
 * of its range (the nodes of other ranges within a radius of its own), forms
 * its nodes' stencils and operator rows from range + halo, and an explicit
 * step (Section 2.3.1) needs only the halo's new values from the other GPUs.
 * The paper names distributed execution as future work (Section 6).  Both
 * calls are host-only (no context, no GPU) and take host arrays.
 */

/*
 * Morton (Z-order) permutation of the N nodes h_pts [N x dim] (coordinates
 * quantised to a common grid over the bounding box, 31 bits per axis in 2D,
 * 21 in 3D; equal codes in index order): h_perm [N] receives the original
 * index of the k-th node in that order, h_starts [nparts + 1] the balanced
 * range boundaries (h_starts[p] = floor(N p / nparts)); range p is
 * h_perm[h_starts[p] .. h_starts[p+1]-1].
 * Errors: MM_EBADARG (dim not 2/3, non-finite points, nparts outside [1, N]).
 */
int mm_partition_morton(int dim, int64_t N, const double *h_pts, int nparts, int64_t *h_perm,
                        int64_t *h_starts);

/*
 * Halo of the range h_perm[begin .. end-1]: every node outside it whose
 * distance to some node of the range is <= radius, in increasing index order,
 * into h_halo [capacity]; *nhalo receives the count (also when it exceeds
 * capacity, which returns MM_EUNSUPPORTED with the first `capacity` written).
 * With range + halo as the candidates, a range node's n-node stencil is
 * exactly its stencil in the whole set (mm_knn_stencils' ranking) whenever
 * its n-th closest candidate lies within `radius` of it: every node closer
 * than that is within the radius, hence among the candidates.
 * Errors: MM_EBADARG (bad points, range, radius, or h_perm not a permutation
 * on the range), MM_EUNSUPPORTED (capacity too small).
 */
int mm_partition_halo(int dim, int64_t N, const double *h_pts, const int64_t *h_perm, int64_t begin,
                      int64_t end, double radius, int64_t *h_halo, int64_t capacity, int64_t *nhalo);

/* ------------------------------------------------------------- measurement */
/*
 * Measured arithmetic peak of this GPU for the pipe `which` (0 = FP64 FMA,
 * 1 = FP32 FMA), in FLOP/s (an FMA counts 2), from a dependent-chain-free
 * FMA loop over every SM.  Synchronises.  Errors: MM_EBADARG, MM_ECUDA.
 */
int mm_measure_fma_peak(mm_ctx *ctx, int which, double *flops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* MM_H */
