/*
 * oracle.c -- plain, slow CPU oracle for RBF-FD stencil weights (arXiv
 * 1912.13282, "Medusa: a C++ library for solving PDEs using strong form
 * mesh-free methods", Slak & Kosec).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path; the two meet only through the
 * seeded node generators in nodesets/.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC (no FMA
 * contraction, round-to-nearest-even, so its results do not depend on the
 * compiler's choice of fused operations).
 *
 * What it computes, each with the passage it follows:
 *   orc_knn_brute           Section 2.1 (stencils of the n closest nodes, the
 *                           node itself first); exhaustive search, ranked by
 *                           (squared distance in FP64, node index).
 *   orc_balanced_brute      Section 3.1 (FindBalancedSupport, stencils balanced
 *                           around the node): a quota per orthant among the K
 *                           nearest candidates, then the nearest of the rest.
 *   orc_rbffd_weights       Section 2.2.2, eq. rbf-system-aug and the RHS
 *                           definitions around it; Section 3.3 (weights for
 *                           all nodes and operators stored per operator).
 *   orc_rbffd_weights_f128  the same in _Float128 (higher-precision check).
 *   orc_lu_solve            the partial-pivot LU used by the above, exposed
 *                           for pinning against a library solver.
 *   orc_kkt / orc_kkt_cond1 the assembled augmented matrix and its 1-norm
 *                           condition number from an explicit inverse.
 *   orc_spmv, orc_diffuse   Section 2.3.1 (explicit evaluation w^T u_I(i) and
 *                           explicit Euler, eq. exp-start..exp-end, interior
 *                           update with Dirichlet nodes held).
 *   orc_diffuse_bc          the same with Neumann nodes: eq. exp-end, the
 *                           discrete d/dn of the node set equal to g_n and
 *                           solved for the node's own value.
 *   orc_ilu0, orc_ilu0_solve, orc_bicgstab
 *                           the implicit solve of Section 2.3.2: BiCGSTAB
 *                           (van der Vorst) with an incomplete-LU
 *                           preconditioner of the ILUT family, here ILU(0)
 *                           (the pattern of A, no dropping).
 *   orc_project_lap         least-norm correction of given scaled Laplacian
 *                           weights onto the monomial rows Q^T w = l_q of
 *                           eq. rbf-system-aug.
 *   orc_phi_residual_lap    relative residual of the remaining rows,
 *                           min_lambda ||A w + Q lambda - l_phi||_inf / ||l_phi||_inf
 *                           (lambda the least-squares minimiser).
 *   orc_mlp_*               FP64 forward/backward of a plain GELU MLP and an
 *                           Adam step (no counterpart in the paper).
 *
 * Parity status: every function above is pinned by the CPU tests except the
 * threaded batch drivers' speed, which nothing needs to pin.
 */
#include <math.h>
#include <float.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_SINGULAR 1
#define ORC_BADARG 4
#define ORC_DUPLICATE 5
#define ORC_NOMEM 6

#define ORC_OP_LAP 0
#define ORC_OP_DX 1
#define ORC_OP_DY 2
#define ORC_OP_DZ 3
#define ORC_OP_DN 4
/* second derivatives d^2/dx_a dx_b, bits 5..10: xx, xy, yy, xz, yz, zz */
#define ORC_OP_DXX 5
#define ORC_NOPS 11

#define ORC_MAXDIM 3
#define ORC_MAXDEG 6

/* ---------------------------------------------------------------- monomials */
/* Exponent tables for total degree <= m, graded lexicographic order:
 * degree ascending, inside a degree the exponent of x_0 descending, then x_1... */
static int g_mono[ORC_MAXDIM + 1][ORC_MAXDEG + 1][128 * ORC_MAXDIM];
static int g_mono_l[ORC_MAXDIM + 1][ORC_MAXDEG + 1];
static pthread_once_t g_mono_once = PTHREAD_ONCE_INIT;

static void mono_rec(int dim, int pos, int remaining, int *cur, int *tab, int *count)
{
    if (pos == dim - 1) {
        cur[pos] = remaining;
        for (int a = 0; a < ORC_MAXDIM; ++a) tab[*count * ORC_MAXDIM + a] = a < dim ? cur[a] : 0;
        ++*count;
        return;
    }
    for (int e = remaining; e >= 0; --e) {
        cur[pos] = e;
        mono_rec(dim, pos + 1, remaining - e, cur, tab, count);
    }
}

static void mono_init(void)
{
    for (int dim = 1; dim <= ORC_MAXDIM; ++dim)
        for (int m = 0; m <= ORC_MAXDEG; ++m) {
            int count = 0, cur[ORC_MAXDIM] = {0, 0, 0};
            for (int deg = 0; deg <= m; ++deg) mono_rec(dim, 0, deg, cur, g_mono[dim][m], &count);
            g_mono_l[dim][m] = count;
        }
}

static int orc_monomials(int dim, int m, const int **E)
{
    pthread_once(&g_mono_once, mono_init);
    *E = g_mono[dim][m];
    return g_mono_l[dim][m];
}

static int orc_popcount(unsigned v)
{
    int c = 0;
    for (; v; v >>= 1) c += (int)(v & 1u);
    return c;
}

/* Exported for the tests: number of monomials and their exponents. */
int orc_monomial_table(int dim, int m, int *exps_out /* [l*dim] or NULL */)
{
    if (dim < 1 || dim > ORC_MAXDIM || m < 0 || m > ORC_MAXDEG) return -1;
    const int *E;
    int l = orc_monomials(dim, m, &E);
    if (exps_out)
        for (int b = 0; b < l; ++b)
            for (int a = 0; a < dim; ++a) exps_out[b * dim + a] = E[b * ORC_MAXDIM + a];
    return l;
}

/* ------------------------------------------------- two instantiations of the
 * per-node weights: double and _Float128                                     */
static double sqrt_d(double x) { return sqrt(x); }

/* Square root in _Float128 by Newton's (Heron's) iteration y <- (y + x/y)/2
 * from the double square root; two steps take 53 correct bits past 113. */
static _Float128 sqrt_q(_Float128 x)
{
    if (!(x > 0)) return (_Float128)0;
    _Float128 y = (_Float128)sqrt((double)x);
    for (int i = 0; i < 3; ++i) y = (y + x / y) / 2;
    return y;
}

#define REAL double
#define FN(x) x##_d
#define RSQRT_(x) sqrt_d(x)
#include "rbffd_node.inc"
#undef REAL
#undef FN
#undef RSQRT_

#define REAL _Float128
#define FN(x) x##_q
#define RSQRT_(x) sqrt_q(x)
#include "rbffd_node.inc"
#undef REAL
#undef FN
#undef RSQRT_

static const double U64 = DBL_EPSILON / 2;
/* unit roundoff of binary128: 2^-113 */
#define U128 ((_Float128)1.0 / ((_Float128)(1ULL << 56) * (_Float128)(1ULL << 57)))

/* ------------------------------------------------------------ thread helper */
typedef struct {
    void (*body)(void *ctx, int64_t begin, int64_t end);
    void *ctx;
    int64_t begin, end;
} orc_chunk;

static void *orc_chunk_run(void *p)
{
    orc_chunk *c = (orc_chunk *)p;
    c->body(c->ctx, c->begin, c->end);
    return NULL;
}

/* Split [begin, end) into nthreads contiguous chunks and run body on each. */
static void orc_parallel_for(int nthreads, int64_t begin, int64_t end,
                             void (*body)(void *, int64_t, int64_t), void *ctx)
{
    int64_t total = end - begin;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (total < nthreads * 4 || nthreads == 1) { body(ctx, begin, end); return; }
    pthread_t th[256];
    orc_chunk ch[256];
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        ch[t].body = body;
        ch[t].ctx = ctx;
        ch[t].begin = begin + total * t / nthreads;
        ch[t].end = begin + total * (t + 1) / nthreads;
        if (t == 0) continue;
        if (pthread_create(&th[t], NULL, orc_chunk_run, &ch[t]) == 0) ++started;
        else { ch[t].body(ch[t].ctx, ch[t].begin, ch[t].end); th[t] = 0; }
    }
    body(ctx, ch[0].begin, ch[0].end);
    for (int t = 1; t < nthreads; ++t)
        if (th[t]) pthread_join(th[t], NULL);
    (void)started;
}

/* ---------------------------------------------------------------- kNN brute */
typedef struct {
    int dim;
    int64_t N;
    const double *pts;
    const int64_t *queries;
    int n;
    int32_t *idx;
    int32_t *status;
} knn_job;

/* (d2, j) < (e2, i) in the ranking order: squared distance, then node index */
static int key_less(double d2, int64_t j, double e2, int64_t i)
{
    return d2 < e2 || (d2 == e2 && j < i);
}

static void knn_body(void *p, int64_t qb, int64_t qe)
{
    knn_job *J = (knn_job *)p;
    int n = J->n, dim = J->dim;
    double *bd = (double *)malloc(sizeof(double) * (size_t)(n > 1 ? n : 1));
    int64_t *bi = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 1 ? n : 1));
    for (int64_t q = qb; q < qe; ++q) {
        int64_t c = J->queries[q];
        const double *xc = J->pts + c * dim;
        int have = 0, dup = 0;
        int cap = n - 1; /* the centre takes slot 0 */
        for (int64_t j = 0; j < J->N; ++j) {
            if (j == c) continue;
            const double *xj = J->pts + j * dim;
            double d2 = 0.0;
            for (int a = 0; a < dim; ++a) {
                double d = xj[a] - xc[a];
                d2 = d2 + d * d;
            }
            if (d2 == 0.0) dup = 1;
            if (cap == 0) continue;
            if (have == cap && !key_less(d2, j, bd[have - 1], bi[have - 1])) continue;
            int pos = have < cap ? have : cap - 1;
            if (have < cap) ++have;
            while (pos > 0 && key_less(d2, j, bd[pos - 1], bi[pos - 1])) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bd[pos] = d2;
            bi[pos] = j;
        }
        int32_t *out = J->idx + q * n;
        out[0] = (int32_t)c;
        for (int t = 0; t < cap; ++t) out[t + 1] = t < have ? (int32_t)bi[t] : -1;
        if (J->status) J->status[q] = dup ? ORC_DUPLICATE : (have < cap ? ORC_BADARG : ORC_OK);
    }
    free(bd);
    free(bi);
}

/*
 * Stencils of the n nearest nodes (Section 2.1: each node in its own stencil,
 * first).  For every query node c = queries[q] the row idx[q*n .. q*n+n-1]
 * holds c, then the n-1 other nodes with the smallest (squared distance,
 * index), ascending.  status[q] (optional) is ORC_DUPLICATE if another node
 * coincides with c, ORC_BADARG if N < n.
 */
int orc_knn_brute(int dim, int64_t N, const double *pts, int64_t nq, const int64_t *queries,
                  int n, int32_t *idx, int32_t *status, int nthreads)
{
    if (dim < 1 || dim > ORC_MAXDIM || n < 1 || N < 1) return ORC_BADARG;
    knn_job J = {dim, N, pts, queries, n, idx, status};
    orc_parallel_for(nthreads, 0, nq, knn_body, &J);
    return ORC_OK;
}

/*
 * Balanced stencils (Section 3.1 names FindBalancedSupport: stencils "balanced
 * around the central node"; the paper states no rule, this is the reading the
 * library implements).  For query c: the K nearest nodes (orc_knn_brute's
 * ranking, c first) are the candidates; every other candidate j lies in the
 * orthant o(j) = sum_a 2^a [x_j,a - x_c,a < 0]; with quota = (n - 1) / 2^dim
 * (integer division) the candidates are scanned in ranking order and j is
 * taken if fewer than `quota` earlier candidates of o(j) were taken; then,
 * while fewer than n - 1 are taken, the not-yet-taken candidates are added in
 * ranking order.  The row is c followed by the taken candidates in ranking
 * order.  status as orc_knn_brute (ORC_BADARG also when K < n or N < K).
 */
int orc_balanced_brute(int dim, int64_t N, const double *pts, int64_t nq, const int64_t *queries,
                       int n, int K, int32_t *idx, int32_t *status, int nthreads)
{
    if (dim < 1 || dim > ORC_MAXDIM || n < 1 || K < n || K > 64 || N < 1) return ORC_BADARG;
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nq > 0 ? nq : 1) * (size_t)K);
    if (!cand) return ORC_NOMEM;
    int rc = orc_knn_brute(dim, N, pts, nq, queries, K, cand, status, nthreads);
    const int quota = (n - 1) / (1 << dim);
    for (int64_t q = 0; rc == ORC_OK && q < nq; ++q) {
        const int32_t *cq = cand + q * K;
        int32_t *out = idx + q * n;
        const int64_t c = cq[0];
        int taken[64 + 1] = {0};
        int per[8] = {0};
        int count = 0;
        for (int t = 1; t < K && count < n - 1; ++t) {
            if (cq[t] < 0) break;
            int o = 0;
            for (int a = 0; a < dim; ++a)
                if (pts[(int64_t)cq[t] * dim + a] - pts[c * dim + a] < 0.0) o |= 1 << a;
            if (per[o] < quota) {
                per[o] += 1;
                taken[t] = 1;
                ++count;
            }
        }
        for (int t = 1; t < K && count < n - 1; ++t)
            if (cq[t] >= 0 && !taken[t]) {
                taken[t] = 1;
                ++count;
            }
        out[0] = (int32_t)c;
        int w = 1;
        for (int t = 1; t < K && w < n; ++t)
            if (taken[t]) out[w++] = cq[t];
        for (; w < n; ++w) out[w] = -1;
        if (status && status[q] == ORC_OK && count < n - 1) status[q] = ORC_BADARG;
    }
    free(cand);
    return rc;
}

/* ------------------------------------------------------------ batch weights */
typedef struct {
    int dim;
    const double *pts, *normals;
    const int64_t *row_ptr;
    const int32_t *col;
    int k, m;
    unsigned ops;
    double *const *vals;     /* one [nnz] array per set bit of ops */
    double *const *svals;    /* optional scaled weights, same layout */
    double *scale;           /* optional [nrows] */
    int32_t *status;
    int quad;                /* 1: compute in _Float128 */
} w_job;

static void weights_body(void *p, int64_t rb, int64_t re)
{
    w_job *J = (w_job *)p;
    const int *E;
    int l = orc_monomials(J->dim, J->m, &E);
    int R = orc_popcount(J->ops);
    int nmax = 0;
    for (int64_t i = rb; i < re; ++i) {
        int n = (int)(J->row_ptr[i + 1] - J->row_ptr[i]);
        if (n > nmax) nmax = n;
    }
    int M = nmax + l;
    size_t wsz = (size_t)M * M + (size_t)M * R + (size_t)nmax * J->dim + 16;
    double *work = NULL, *w = NULL, *ws = NULL;
    _Float128 *workq = NULL, *wq = NULL, *wsq = NULL;
    if (J->quad) {
        workq = (_Float128 *)malloc(sizeof(_Float128) * wsz);
        wq = (_Float128 *)malloc(sizeof(_Float128) * (size_t)(R * nmax + 1));
        wsq = (_Float128 *)malloc(sizeof(_Float128) * (size_t)(R * nmax + 1));
    } else {
        work = (double *)malloc(sizeof(double) * wsz);
        w = (double *)malloc(sizeof(double) * (size_t)(R * nmax + 1));
        ws = (double *)malloc(sizeof(double) * (size_t)(R * nmax + 1));
    }
    for (int64_t i = rb; i < re; ++i) {
        int64_t b = J->row_ptr[i];
        int n = (int)(J->row_ptr[i + 1] - b);
        const int32_t *st = J->col + b;
        int rc;
        if (n < 1 || st[0] != (int32_t)i) {
            rc = ORC_BADARG;
            for (int r = 0; r < R; ++r)
                for (int j = 0; j < n; ++j) {
                    J->vals[r][b + j] = 0.0;
                    if (J->svals) J->svals[r][b + j] = 0.0;
                }
        } else if (J->quad) {
            _Float128 s = 0;
            rc = stencil_weights_q(J->dim, J->pts, J->normals, n, st, J->k, J->m, J->ops,
                                   wq, wsq, &s, workq, U128);
            for (int r = 0; r < R; ++r)
                for (int j = 0; j < n; ++j) {
                    J->vals[r][b + j] = (double)wq[r * n + j];
                    if (J->svals) J->svals[r][b + j] = (double)wsq[r * n + j];
                }
            if (J->scale) J->scale[i] = (double)s;
        } else {
            double s = 0;
            rc = stencil_weights_d(J->dim, J->pts, J->normals, n, st, J->k, J->m, J->ops,
                                   w, ws, &s, work, U64);
            for (int r = 0; r < R; ++r)
                for (int j = 0; j < n; ++j) {
                    J->vals[r][b + j] = w[r * n + j];
                    if (J->svals) J->svals[r][b + j] = ws[r * n + j];
                }
            if (J->scale) J->scale[i] = s;
        }
        if (J->status) J->status[i] = rc;
    }
    free(work); free(w); free(ws);
    free(workq); free(wq); free(wsq);
}

/*
 * RBF-FD weights for rows [row_begin, row_end) of a CSR stencil pattern
 * (rows are nodes; col[row_ptr[i]] must be i).  vals[r][row_ptr[i] + j] is
 * the weight of stencil node j for the r-th set bit of ops (bit 0 Laplacian,
 * 1..3 d/dx, d/dy, d/dz, 4 d/dn using normals[i*dim..]).  svals (optional)
 * gets the same weights in scaled units, scale (optional) the scale s.
 * status[i] is ORC_OK, ORC_SINGULAR (weights zeroed) or ORC_BADARG.
 */
static int weights_common(int dim, const double *pts, const double *normals,
                          const int64_t *row_ptr, const int32_t *col, int64_t row_begin,
                          int64_t row_end, int k, int m, unsigned ops, double *const *vals,
                          double *const *svals, double *scale, int32_t *status, int nthreads,
                          int quad)
{
    if (dim < 2 || dim > ORC_MAXDIM || m < 0 || m > ORC_MAXDEG || k < 3 || (k % 2) == 0 ||
        ops == 0 || ops >= (1u << ORC_NOPS))
        return ORC_BADARG;
    w_job J = {dim, pts, normals, row_ptr, col, k, m, ops, vals, svals, scale, status, quad};
    orc_parallel_for(nthreads, row_begin, row_end, weights_body, &J);
    return ORC_OK;
}

int orc_rbffd_weights(int dim, const double *pts, const double *normals, const int64_t *row_ptr,
                      const int32_t *col, int64_t row_begin, int64_t row_end, int k, int m,
                      unsigned ops, double *const *vals, double *const *svals, double *scale,
                      int32_t *status, int nthreads)
{
    return weights_common(dim, pts, normals, row_ptr, col, row_begin, row_end, k, m, ops, vals,
                          svals, scale, status, nthreads, 0);
}

/* Same in _Float128, results rounded to double. */
int orc_rbffd_weights_f128(int dim, const double *pts, const double *normals,
                           const int64_t *row_ptr, const int32_t *col, int64_t row_begin,
                           int64_t row_end, int k, int m, unsigned ops, double *const *vals,
                           double *const *svals, double *scale, int32_t *status, int nthreads)
{
    return weights_common(dim, pts, normals, row_ptr, col, row_begin, row_end, k, m, ops, vals,
                          svals, scale, status, nthreads, 1);
}

/* ------------------------------------------------- exposed building blocks */
/* Solve K x = B (M x M, R columns, both row-major, overwritten). */
int orc_lu_solve(int M, double *K, int R, double *B)
{
    return lu_solve_d(M, K, R, B, U64);
}

/*
 * The assembled scaled system of one stencil: K_out (M x M), B_out (M x R),
 * xi_out (n x dim scaled offsets), s_out.  M = n + l.
 */
int orc_kkt(int dim, const double *pts, const double *normals, int n, const int32_t *st, int k,
            int m, unsigned ops, double *K_out, double *B_out, double *xi_out, double *s_out)
{
    int qpow[ORC_NOPS];
    return assemble_d(dim, pts, normals, n, st, k, m, ops, K_out, B_out, qpow, s_out, xi_out);
}

/* kappa_1(K) = ||K||_1 ||K^-1||_1 of the assembled system of one stencil,
 * inverse by the LU above applied to the identity.  Returns +inf if singular. */
double orc_kkt_cond1(int dim, const double *pts, int n, const int32_t *st, int k, int m)
{
    const int *E;
    int l = orc_monomials(dim, m, &E);
    int M = n + l;
    double *K = (double *)malloc(sizeof(double) * (size_t)M * M);
    double *K2 = (double *)malloc(sizeof(double) * (size_t)M * M);
    double *B = (double *)malloc(sizeof(double) * (size_t)M * (M > 5 ? M : 5));
    double *xi = (double *)malloc(sizeof(double) * (size_t)n * dim);
    double s, res;
    int qpow[ORC_NOPS];
    int rc = assemble_d(dim, pts, NULL, n, st, k, m, 1u << ORC_OP_LAP, K, B, qpow, &s, xi);
    if (rc != ORC_OK) { res = INFINITY; goto out; }
    double n1 = 0;
    for (int j = 0; j < M; ++j) {
        double c = 0;
        for (int i = 0; i < M; ++i) c += fabs(K[i * M + j]);
        if (c > n1) n1 = c;
    }
    memcpy(K2, K, sizeof(double) * (size_t)M * M);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) B[i * M + j] = (i == j) ? 1.0 : 0.0;
    if (lu_solve_d(M, K2, M, B, U64) != ORC_OK) { res = INFINITY; goto out; }
    double ni = 0;
    for (int j = 0; j < M; ++j) {
        double c = 0;
        for (int i = 0; i < M; ++i) c += fabs(B[i * M + j]);
        if (c > ni) ni = c;
    }
    res = n1 * ni;
out:
    free(K); free(K2); free(B); free(xi);
    return res;
}

/* ----------------------------------------------------- operator application */
/* y_i = alpha * sum_j vals[j] u[col[j]] + beta * y_i over the CSR rows
 * (explicit evaluation w^T u_I(i), Section 2.3.1). */
void orc_spmv(int64_t nrows, const int64_t *row_ptr, const int32_t *col, const double *vals,
              const double *u, double alpha, double beta, double *y)
{
    for (int64_t i = 0; i < nrows; ++i) {
        double acc = 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) acc = acc + vals[p] * u[col[p]];
        y[i] = beta == 0.0 ? alpha * acc : alpha * acc + beta * y[i];
    }
}

/* Explicit steps with boundary kinds, eq. exp-start..exp-end, every update
 * from the previous step's values: kind 0 (internal) u_i <- u_i + dt (L u)_i;
 * kind 1 (Dirichlet) keeps u_i; kind 2 (Neumann) takes the node's row as its
 * d/dn weights (centre first) and sets
 *     u_i <- (g_i - sum_{j >= 2} w_ij u_j) / w_i1,
 * g = NULL meaning g_i = 0. */
int orc_diffuse_bc(int64_t nrows, const int64_t *row_ptr, const int32_t *col, const double *vals,
                   const uint8_t *kind, const double *g, double dt, int steps, double *u)
{
    double *nu = (double *)malloc(sizeof(double) * (size_t)(nrows > 0 ? nrows : 1));
    if (!nu) return ORC_NOMEM;
    for (int t = 0; t < steps; ++t) {
        for (int64_t i = 0; i < nrows; ++i) {
            if (kind[i] == 1) {
                nu[i] = u[i];
            } else if (kind[i] == 2) {
                double s = 0.0;
                for (int64_t p = row_ptr[i] + 1; p < row_ptr[i + 1]; ++p) s = s + vals[p] * u[col[p]];
                nu[i] = ((g ? g[i] : 0.0) - s) / vals[row_ptr[i]];
            } else {
                double acc = 0.0;
                for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) acc = acc + vals[p] * u[col[p]];
                nu[i] = u[i] + dt * acc;
            }
        }
        memcpy(u, nu, sizeof(double) * (size_t)nrows);
    }
    free(nu);
    return ORC_OK;
}

/* ILU(0) in place on a CSR matrix whose rows have sorted columns and a
 * diagonal entry: afterwards the strictly lower part holds L (unit diagonal
 * implied) and the rest U, with (L U)_ij = A_ij for every (i, j) of the
 * pattern (row-by-row elimination, updates outside the pattern dropped).
 * diag[i] receives the position of (i, i).  ORC_BADARG: a diagonal entry is
 * missing; ORC_SINGULAR: a zero pivot. */
int orc_ilu0(int64_t n, const int64_t *rp, const int32_t *col, double *val, int64_t *diag)
{
    int64_t *where = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!where) return ORC_NOMEM;
    for (int64_t i = 0; i < n; ++i) where[i] = -1;
    int rc = ORC_OK;
    for (int64_t i = 0; i < n && rc == ORC_OK; ++i) {
        diag[i] = -1;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            where[col[p]] = p;
            if (col[p] == i) diag[i] = p;
        }
        if (diag[i] < 0) rc = ORC_BADARG;
        for (int64_t p = rp[i]; rc == ORC_OK && p < rp[i + 1] && col[p] < i; ++p) {
            const int64_t k = col[p];
            if (val[diag[k]] == 0.0) { rc = ORC_SINGULAR; break; }
            const double lik = val[p] / val[diag[k]];
            val[p] = lik;
            for (int64_t q = diag[k] + 1; q < rp[k + 1]; ++q) {
                const int64_t w = where[col[q]];
                if (w >= 0) val[w] = val[w] - lik * val[q];
            }
        }
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) where[col[p]] = -1;
        if (rc == ORC_OK && val[diag[i]] == 0.0) rc = ORC_SINGULAR;
    }
    free(where);
    return rc;
}

/* x = (L U)^-1 b with the factors of orc_ilu0 (forward, then back substitution). */
void orc_ilu0_solve(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                    const int64_t *diag, const double *b, double *x)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = b[i];
        for (int64_t p = rp[i]; p < diag[i]; ++p) s = s - val[p] * x[col[p]];
        x[i] = s;
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int64_t p = diag[i] + 1; p < rp[i + 1]; ++p) s = s - val[p] * x[col[p]];
        x[i] = s / val[diag[i]];
    }
}

static void orc_csr_mv(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                       const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s = s + val[p] * x[col[p]];
        y[i] = s;
    }
}

static double orc_dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = s + a[i] * b[i];
    return s;
}

/* BiCGSTAB (van der Vorst 1992) for A x = b, preconditioned by the ILU(0)
 * factors fval/diag of the same pattern (M = L U; NULL: none), x holding the
 * initial guess on entry.  Stops when ||b - A x||_2 <= tol ||b||_2 (the
 * recursively updated residual), or after maxit iterations.  *iters and
 * *relres receive the iterations taken and the final relative residual.
 * Returns ORC_OK when converged, ORC_SINGULAR on a breakdown or no
 * convergence. */
int orc_bicgstab(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                 const double *fval, const int64_t *diag, const double *b, double *x,
                 double tol, int maxit, int *iters, double *relres)
{
    double *w = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * 8);
    if (!w) return ORC_NOMEM;
    double *r = w, *rh = w + n, *p = w + 2 * n, *v = w + 3 * n, *ph = w + 4 * n, *s = w + 5 * n,
           *sh = w + 6 * n, *t = w + 7 * n;
    orc_csr_mv(n, rp, col, val, x, t);
    for (int64_t i = 0; i < n; ++i) {
        r[i] = b[i] - t[i];
        rh[i] = r[i];
        p[i] = v[i] = 0.0;
    }
    const double nb = sqrt(orc_dot(n, b, b));
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    double res = sqrt(orc_dot(n, r, r)) / (nb > 0 ? nb : 1.0);
    int it = 0, rc = ORC_SINGULAR;
    if (res <= tol) rc = ORC_OK;
    while (rc != ORC_OK && it < maxit) {
        ++it;
        const double rho1 = orc_dot(n, rh, r);
        if (rho1 == 0.0 || omega == 0.0) break;
        const double beta = (rho1 / rho) * (alpha / omega);
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        if (fval) orc_ilu0_solve(n, rp, col, fval, diag, p, ph);
        else memcpy(ph, p, sizeof(double) * (size_t)n);
        orc_csr_mv(n, rp, col, val, ph, v);
        const double rv = orc_dot(n, rh, v);
        if (rv == 0.0) break;
        alpha = rho1 / rv;
        for (int64_t i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
        if (fval) orc_ilu0_solve(n, rp, col, fval, diag, s, sh);
        else memcpy(sh, s, sizeof(double) * (size_t)n);
        orc_csr_mv(n, rp, col, val, sh, t);
        const double tt = orc_dot(n, t, t);
        omega = tt > 0.0 ? orc_dot(n, t, s) / tt : 0.0;
        for (int64_t i = 0; i < n; ++i) {
            x[i] = x[i] + alpha * ph[i] + omega * sh[i];
            r[i] = s[i] - omega * t[i];
        }
        rho = rho1;
        res = sqrt(orc_dot(n, r, r)) / (nb > 0 ? nb : 1.0);
        if (res <= tol) rc = ORC_OK;
    }
    *iters = it;
    *relres = res;
    free(w);
    return rc;
}

/* Explicit Euler steps u <- u + dt * L u on rows with fixed[i] == 0; rows with
 * fixed[i] != 0 keep their value (Dirichlet nodes), eq. exp-start..exp-end. */
int orc_diffuse(int64_t nrows, const int64_t *row_ptr, const int32_t *col, const double *vals,
                const uint8_t *fixed, double dt, int steps, double *u)
{
    double *nu = (double *)malloc(sizeof(double) * (size_t)(nrows > 0 ? nrows : 1));
    if (!nu) return ORC_NOMEM;
    for (int t = 0; t < steps; ++t) {
        for (int64_t i = 0; i < nrows; ++i) {
            if (fixed[i]) { nu[i] = u[i]; continue; }
            double acc = 0.0;
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) acc = acc + vals[p] * u[col[p]];
            nu[i] = u[i] + dt * acc;
        }
        memcpy(u, nu, sizeof(double) * (size_t)nrows);
    }
    free(nu);
    return ORC_OK;
}

/* ------------------------------------------ projection and residual check */
/*
 * Least-norm correction of scaled Laplacian weights wt (n entries) of one
 * stencil onto the monomial rows of eq. rbf-system-aug:
 *   (Q^T Q) z = l_q - Q^T wt,   w = wt + Q z.
 */
int orc_project_lap(int dim, const double *pts, int n, const int32_t *st, int k, int m,
                    const double *wt, double *w_out)
{
    const int *E;
    int l = orc_monomials(dim, m, &E);
    int M = n + l;
    double *K = (double *)malloc(sizeof(double) * (size_t)M * M);
    double *B = (double *)malloc(sizeof(double) * (size_t)M);
    double *xi = (double *)malloc(sizeof(double) * (size_t)n * dim);
    double *G = (double *)malloc(sizeof(double) * (size_t)l * l);
    double *z = (double *)malloc(sizeof(double) * (size_t)l);
    double s;
    int qpow[ORC_NOPS];
    int rc = assemble_d(dim, pts, NULL, n, st, k, m, 1u << ORC_OP_LAP, K, B, qpow, &s, xi);
    if (rc == ORC_OK) {
        /* Q_ib = K[i][n+b], l_q = B[n+b] */
        for (int a = 0; a < l; ++a) {
            for (int b = 0; b < l; ++b) {
                double g = 0;
                for (int i = 0; i < n; ++i) g = g + K[i * M + n + a] * K[i * M + n + b];
                G[a * l + b] = g;
            }
            double qw = 0;
            for (int i = 0; i < n; ++i) qw = qw + K[i * M + n + a] * wt[i];
            z[a] = B[n + a] - qw;
        }
        rc = lu_solve_d(l, G, 1, z, U64);
        if (rc == ORC_OK)
            for (int i = 0; i < n; ++i) {
                double c = 0;
                for (int b = 0; b < l; ++b) c = c + K[i * M + n + b] * z[b];
                w_out[i] = wt[i] + c;
            }
    }
    free(K); free(B); free(xi); free(G); free(z);
    return rc;
}

/*
 * rho = ||A w + Q lambda - l_phi||_inf / ||l_phi||_inf for scaled Laplacian
 * weights w of one stencil, lambda = argmin ||A w + Q lambda - l_phi||_2
 * (normal equations Q^T Q lambda = Q^T (l_phi - A w)).  Returns -1 on error.
 */
double orc_phi_residual_lap(int dim, const double *pts, int n, const int32_t *st, int k, int m,
                            const double *w)
{
    const int *E;
    int l = orc_monomials(dim, m, &E);
    int M = n + l;
    double *K = (double *)malloc(sizeof(double) * (size_t)M * M);
    double *B = (double *)malloc(sizeof(double) * (size_t)M);
    double *xi = (double *)malloc(sizeof(double) * (size_t)n * dim);
    double *G = (double *)malloc(sizeof(double) * (size_t)l * l);
    double *lam = (double *)malloc(sizeof(double) * (size_t)l);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double s, res = -1;
    int qpow[ORC_NOPS];
    if (assemble_d(dim, pts, NULL, n, st, k, m, 1u << ORC_OP_LAP, K, B, qpow, &s, xi) == ORC_OK) {
        for (int i = 0; i < n; ++i) {
            double aw = 0;
            for (int j = 0; j < n; ++j) aw = aw + K[i * M + j] * w[j];
            r[i] = B[i] - aw; /* l_phi - A w */
        }
        for (int a = 0; a < l; ++a) {
            for (int b = 0; b < l; ++b) {
                double g = 0;
                for (int i = 0; i < n; ++i) g = g + K[i * M + n + a] * K[i * M + n + b];
                G[a * l + b] = g;
            }
            double t = 0;
            for (int i = 0; i < n; ++i) t = t + K[i * M + n + a] * r[i];
            lam[a] = t;
        }
        if (lu_solve_d(l, G, 1, lam, U64) == ORC_OK) {
            double num = 0, den = 0;
            for (int i = 0; i < n; ++i) {
                double ql = 0;
                for (int b = 0; b < l; ++b) ql = ql + K[i * M + n + b] * lam[b];
                double e = fabs(ql - r[i]);
                if (e > num) num = e;
                if (fabs(B[i]) > den) den = fabs(B[i]);
            }
            res = den > 0 ? num / den : num;
        }
    }
    free(K); free(B); free(xi); free(G); free(lam); free(r);
    return res;
}

/* ---------------------------------------------------------------------- MLP */
/*
 * A plain multilayer perceptron in FP64:
 *   h_0 = x,  h_t = gelu(W_t h_{t-1} + b_t) for t = 1..L,  y = W_{L+1} h_L + b_{L+1},
 * gelu(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) (Hendrycks & Gimpel's
 * tanh form).  Parameters are packed as W_1 [H x n_in], b_1 [H], W_2 [H x H],
 * b_2, ..., W_{L+1} [n_out x H], b_{L+1}; W row-major [out][in].
 * Loss = mean over the B x n_out entries of (y - t)^2.
 */
static double gelu_d(double z)
{
    const double c = 0.7978845608028654; /* sqrt(2/pi) */
    return 0.5 * z * (1.0 + tanh(c * (z + 0.044715 * z * z * z)));
}

static double gelu_grad_d(double z)
{
    const double c = 0.7978845608028654;
    double t = tanh(c * (z + 0.044715 * z * z * z));
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * c * (1.0 + 3.0 * 0.044715 * z * z);
}

int64_t orc_mlp_nparams(int n_in, int H, int L, int n_out)
{
    return (int64_t)H * n_in + H + (int64_t)(L - 1) * ((int64_t)H * H + H) + (int64_t)n_out * H + n_out;
}

/* Forward pass; returns the loss if targets != NULL, writes y [B x n_out]. */
double orc_mlp_forward(int n_in, int H, int L, int n_out, const double *params, int64_t B,
                       const double *x, const double *targets, double *y)
{
    double *a = (double *)malloc(sizeof(double) * (size_t)(H > n_in ? H : n_in));
    double *h = (double *)malloc(sizeof(double) * (size_t)(H > n_in ? H : n_in));
    double loss = 0;
    for (int64_t bi = 0; bi < B; ++bi) {
        const double *p = params;
        int width = n_in;
        for (int i = 0; i < n_in; ++i) h[i] = x[bi * n_in + i];
        for (int t = 0; t < L; ++t) {
            const double *W = p, *bb = p + (int64_t)H * width;
            for (int o = 0; o < H; ++o) {
                double z = bb[o];
                for (int i = 0; i < width; ++i) z = z + W[(int64_t)o * width + i] * h[i];
                a[o] = gelu_d(z);
            }
            p = bb + H;
            memcpy(h, a, sizeof(double) * (size_t)H);
            width = H;
        }
        const double *W = p, *bb = p + (int64_t)n_out * H;
        for (int o = 0; o < n_out; ++o) {
            double z = bb[o];
            for (int i = 0; i < H; ++i) z = z + W[(int64_t)o * H + i] * h[i];
            y[bi * n_out + o] = z;
            if (targets) {
                double e = z - targets[bi * n_out + o];
                loss = loss + e * e;
            }
        }
    }
    free(a); free(h);
    return targets ? loss / (double)(B * n_out) : 0.0;
}

/* Forward + backward: grads (same packing as params) of the mean squared
 * error; returns the loss. */
double orc_mlp_grad(int n_in, int H, int L, int n_out, const double *params, int64_t B,
                    const double *x, const double *targets, double *grads)
{
    int64_t np = orc_mlp_nparams(n_in, H, L, n_out);
    memset(grads, 0, sizeof(double) * (size_t)np);
    int wmax = H > n_in ? H : n_in;
    double *hs = (double *)malloc(sizeof(double) * (size_t)(L + 1) * wmax); /* h_0..h_L */
    double *zs = (double *)malloc(sizeof(double) * (size_t)(L + 1) * wmax); /* z_1..z_L */
    double *gy = (double *)malloc(sizeof(double) * (size_t)(n_out > wmax ? n_out : wmax));
    double *gh = (double *)malloc(sizeof(double) * (size_t)wmax);
    double *gz = (double *)malloc(sizeof(double) * (size_t)wmax);
    const double **Wp = (const double **)malloc(sizeof(double *) * (size_t)(L + 1));
    double **Gp = (double **)malloc(sizeof(double *) * (size_t)(L + 1));
    int *win = (int *)malloc(sizeof(int) * (size_t)(L + 1));
    {
        const double *p = params;
        double *g = grads;
        int width = n_in;
        for (int t = 0; t <= L; ++t) {
            int out = t < L ? H : n_out;
            Wp[t] = p; Gp[t] = g; win[t] = width;
            p += (int64_t)out * width + out;
            g += (int64_t)out * width + out;
            width = H;
        }
    }
    double loss = 0;
    double scale = 2.0 / (double)(B * n_out);
    for (int64_t bi = 0; bi < B; ++bi) {
        for (int i = 0; i < n_in; ++i) hs[i] = x[bi * n_in + i];
        for (int t = 0; t < L; ++t) {
            int width = win[t];
            const double *W = Wp[t], *bb = W + (int64_t)H * width;
            for (int o = 0; o < H; ++o) {
                double z = bb[o];
                for (int i = 0; i < width; ++i) z = z + W[(int64_t)o * width + i] * hs[t * wmax + i];
                zs[(t + 1) * wmax + o] = z;
                hs[(t + 1) * wmax + o] = gelu_d(z);
            }
        }
        {
            const double *W = Wp[L], *bb = W + (int64_t)n_out * H;
            for (int o = 0; o < n_out; ++o) {
                double z = bb[o];
                for (int i = 0; i < H; ++i) z = z + W[(int64_t)o * H + i] * hs[L * wmax + i];
                double e = z - targets[bi * n_out + o];
                loss = loss + e * e;
                gy[o] = scale * e;
            }
            double *GW = Gp[L], *Gb = GW + (int64_t)n_out * H;
            for (int i = 0; i < H; ++i) gh[i] = 0;
            for (int o = 0; o < n_out; ++o) {
                Gb[o] = Gb[o] + gy[o];
                for (int i = 0; i < H; ++i) {
                    GW[(int64_t)o * H + i] = GW[(int64_t)o * H + i] + gy[o] * hs[L * wmax + i];
                    gh[i] = gh[i] + W[(int64_t)o * H + i] * gy[o];
                }
            }
        }
        for (int t = L - 1; t >= 0; --t) {
            int width = win[t];
            const double *W = Wp[t];
            double *GW = Gp[t], *Gb = GW + (int64_t)H * width;
            for (int o = 0; o < H; ++o) gz[o] = gh[o] * gelu_grad_d(zs[(t + 1) * wmax + o]);
            for (int i = 0; i < width; ++i) gh[i] = 0;
            for (int o = 0; o < H; ++o) {
                Gb[o] = Gb[o] + gz[o];
                for (int i = 0; i < width; ++i) {
                    GW[(int64_t)o * width + i] = GW[(int64_t)o * width + i] + gz[o] * hs[t * wmax + i];
                    gh[i] = gh[i] + W[(int64_t)o * width + i] * gz[o];
                }
            }
        }
    }
    free(hs); free(zs); free(gy); free(gh); free(gz); free(Wp); free(Gp); free(win);
    return loss / (double)(B * n_out);
}

/* One Adam step (Kingma & Ba, 2015) at step count t >= 1:
 * m <- b1 m + (1-b1) g,  v <- b2 v + (1-b2) g^2,
 * p <- p - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
void orc_adam(int64_t np, double *params, const double *grads, double *m, double *v, int t,
              double lr, double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < np; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * grads[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grads[i] * grads[i];
        params[i] = params[i] - lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
