"""ctypes front-end of the plain FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module; the product path never
does.  It builds ``liboracle.so`` next to this file with gcc (no FMA
contraction, no fast-math) on first use.

Every function takes and returns numpy arrays; see oracle.c for the passage of
the paper each one follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "rbffd_node.inc")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, SINGULAR, BADARG, DUPLICATE = 0, 1, 4, 5
OP_LAP, OP_DX, OP_DY, OP_DZ, OP_DN = 1, 2, 4, 8, 16

_p = np.ctypeslib.ndpointer
_dptr = C.POINTER(C.c_double)


def build(force: bool = False) -> str:
    """Compile liboracle.so if it is missing or older than its sources."""
    with _lock:
        stale = force or not os.path.exists(_LIB_PATH) or any(
            os.path.getmtime(s) > os.path.getmtime(_LIB_PATH) for s in _SRC)
        if stale:
            tmp = _LIB_PATH + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11",
                   "-shared", "-fPIC", "-o", tmp, _SRC[0], "-lm", "-lpthread"]
            subprocess.run(cmd, check=True, cwd=_HERE)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB_PATH)
    i64, i32, u32, dbl = C.c_int64, C.c_int32, C.c_uint32, C.c_double
    lib.orc_monomial_table.argtypes = [C.c_int, C.c_int, C.c_void_p]
    lib.orc_monomial_table.restype = C.c_int
    lib.orc_knn_brute.argtypes = [C.c_int, i64, C.c_void_p, i64, C.c_void_p, C.c_int,
                                  C.c_void_p, C.c_void_p, C.c_int]
    lib.orc_balanced_brute.argtypes = [C.c_int, i64, C.c_void_p, i64, C.c_void_p, C.c_int, C.c_int,
                                       C.c_void_p, C.c_void_p, C.c_int]
    lib.orc_balanced_brute.restype = C.c_int
    lib.orc_knn_brute.restype = C.c_int
    wargs = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, i64, i64, C.c_int,
             C.c_int, u32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    lib.orc_rbffd_weights.argtypes = wargs
    lib.orc_rbffd_weights.restype = C.c_int
    lib.orc_rbffd_weights_f128.argtypes = wargs
    lib.orc_rbffd_weights_f128.restype = C.c_int
    lib.orc_lu_solve.argtypes = [C.c_int, C.c_void_p, C.c_int, C.c_void_p]
    lib.orc_lu_solve.restype = C.c_int
    lib.orc_kkt.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                            C.c_int, u32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_kkt.restype = C.c_int
    lib.orc_kkt_cond1.argtypes = [C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int]
    lib.orc_kkt_cond1.restype = dbl
    lib.orc_spmv.argtypes = [i64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, dbl, dbl,
                             C.c_void_p]
    lib.orc_spmv.restype = None
    lib.orc_diffuse.argtypes = [i64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, dbl,
                                C.c_int, C.c_void_p]
    lib.orc_diffuse.restype = C.c_int
    lib.orc_diffuse_bc.argtypes = [i64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   dbl, C.c_int, C.c_void_p]
    lib.orc_diffuse_bc.restype = C.c_int
    lib.orc_ilu0.argtypes = [i64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_ilu0.restype = C.c_int
    lib.orc_ilu0_solve.argtypes = [i64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p]
    lib.orc_ilu0_solve.restype = None
    lib.orc_bicgstab.argtypes = [i64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, dbl, C.c_int, C.POINTER(C.c_int),
                                 C.POINTER(dbl)]
    lib.orc_bicgstab.restype = C.c_int
    lib.orc_project_lap.argtypes = [C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int,
                                    C.c_void_p, C.c_void_p]
    lib.orc_project_lap.restype = C.c_int
    lib.orc_phi_residual_lap.argtypes = [C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                         C.c_int, C.c_void_p]
    lib.orc_phi_residual_lap.restype = dbl
    lib.orc_mlp_nparams.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
    lib.orc_mlp_nparams.restype = i64
    lib.orc_mlp_forward.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, i64,
                                    C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_mlp_forward.restype = dbl
    lib.orc_mlp_grad.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, i64,
                                 C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_mlp_grad.restype = dbl
    lib.orc_adam.argtypes = [i64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, dbl,
                             dbl, dbl, dbl]
    lib.orc_adam.restype = None
    _lib = lib
    return lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def nthreads_default() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


# ----------------------------------------------------------------- stencils
def monomials(dim: int, m: int) -> np.ndarray:
    """Exponent table [l, dim] of the degree <= m monomials, graded lex order."""
    lib = _load()
    l = lib.orc_monomial_table(dim, m, None)
    out = np.zeros((l, dim), dtype=np.int32)
    lib.orc_monomial_table(dim, m, _ptr(out))
    return out


def knn(pts: np.ndarray, n: int, queries=None, nthreads: int = 1):
    """Brute-force stencils: (idx [nq, n] int32, status [nq] int32)."""
    lib = _load()
    pts = _c(pts, np.float64)
    N, dim = pts.shape
    q = np.arange(N, dtype=np.int64) if queries is None else _c(queries, np.int64)
    idx = np.empty((len(q), n), dtype=np.int32)
    st = np.empty(len(q), dtype=np.int32)
    rc = lib.orc_knn_brute(dim, N, _ptr(pts), len(q), _ptr(q), n, _ptr(idx), _ptr(st), nthreads)
    if rc != OK:
        raise ValueError(f"orc_knn_brute rc={rc}")
    return idx, st


def balanced(pts: np.ndarray, n: int, K: int, queries=None, nthreads: int = 1):
    """Balanced stencils of n nodes among the K nearest candidates
    (orc_balanced_brute): (idx [nq, n] int32, status [nq] int32)."""
    lib = _load()
    pts = _c(pts, np.float64)
    N, dim = pts.shape
    q = np.arange(N, dtype=np.int64) if queries is None else _c(queries, np.int64)
    idx = np.empty((len(q), n), dtype=np.int32)
    st = np.empty(len(q), dtype=np.int32)
    rc = lib.orc_balanced_brute(dim, N, _ptr(pts), len(q), _ptr(q), n, K, _ptr(idx), _ptr(st), nthreads)
    if rc != OK:
        raise ValueError(f"orc_balanced_brute rc={rc}")
    return idx, st


def op_list(ops: int):
    return [b for b in range(11) if ops & (1 << b)]


def weights(pts, row_ptr, col, k, m, ops, normals=None, rows=None, nthreads: int = 1,
            quad: bool = False, scaled: bool = False):
    """RBF-FD weights for CSR rows.  Returns (vals [R, nnz], status [nrows],
    scale [nrows]) and, if ``scaled``, the scaled weights as a 4th item.
    Rows outside ``rows`` (a (begin, end) pair) are left as zeros."""
    lib = _load()
    pts = _c(pts, np.float64)
    N, dim = pts.shape
    row_ptr = _c(row_ptr, np.int64)
    col = _c(col, np.int32)
    nrows = len(row_ptr) - 1
    nnz = int(row_ptr[-1])
    rb, re = (0, nrows) if rows is None else rows
    R = len(op_list(ops))
    vals = np.zeros((R, nnz), dtype=np.float64)
    svals = np.zeros((R, nnz), dtype=np.float64) if scaled else None
    scale = np.zeros(nrows, dtype=np.float64)
    status = np.zeros(nrows, dtype=np.int32)
    nrm = None if normals is None else _c(normals, np.float64)
    vp = (C.c_void_p * R)(*[vals[r].ctypes.data for r in range(R)])
    sp = None if svals is None else (C.c_void_p * R)(*[svals[r].ctypes.data for r in range(R)])
    fn = lib.orc_rbffd_weights_f128 if quad else lib.orc_rbffd_weights
    rc = fn(dim, _ptr(pts), _ptr(nrm), _ptr(row_ptr), _ptr(col), rb, re, k, m, ops,
            C.cast(vp, C.c_void_p), None if sp is None else C.cast(sp, C.c_void_p),
            _ptr(scale), _ptr(status), nthreads)
    if rc != OK:
        raise ValueError(f"orc_rbffd_weights rc={rc}")
    if scaled:
        return vals, status, scale, svals
    return vals, status, scale


def lu_solve(K, B):
    """Solve K X = B with the oracle's partial-pivot LU; returns (X, rc)."""
    lib = _load()
    K = np.array(K, dtype=np.float64, order="C")
    B = np.array(B, dtype=np.float64, order="C")
    squeeze = B.ndim == 1
    if squeeze:
        B = B[:, None].copy()
    rc = lib.orc_lu_solve(K.shape[0], _ptr(K), B.shape[1], _ptr(B))
    return (B[:, 0] if squeeze else B), rc


def kkt(pts, stencil, k, m, ops, normals=None):
    """Assembled system of one stencil: (K [M,M], B [M,R], xi [n,dim], s)."""
    lib = _load()
    pts = _c(pts, np.float64)
    dim = pts.shape[1]
    st = _c(stencil, np.int32)
    n = len(st)
    l = len(monomials(dim, m))
    M = n + l
    R = len(op_list(ops))
    K = np.zeros((M, M))
    B = np.zeros((M, R))
    xi = np.zeros((n, dim))
    s = np.zeros(1)
    nrm = None if normals is None else _c(normals, np.float64)
    rc = lib.orc_kkt(dim, _ptr(pts), _ptr(nrm), n, _ptr(st), k, m, ops, _ptr(K), _ptr(B),
                     _ptr(xi), _ptr(s))
    if rc != OK:
        raise ValueError(f"orc_kkt rc={rc}")
    return K, B, xi, float(s[0])


def kkt_cond1(pts, stencil, k, m) -> float:
    lib = _load()
    pts = _c(pts, np.float64)
    st = _c(stencil, np.int32)
    return lib.orc_kkt_cond1(pts.shape[1], _ptr(pts), len(st), _ptr(st), k, m)


# ------------------------------------------------------- operator application
def spmv(row_ptr, col, vals, u, alpha=1.0, beta=0.0, y=None):
    lib = _load()
    row_ptr = _c(row_ptr, np.int64)
    col = _c(col, np.int32)
    vals = _c(vals, np.float64)
    u = _c(u, np.float64)
    nrows = len(row_ptr) - 1
    y = np.zeros(nrows) if y is None else np.array(y, dtype=np.float64)
    lib.orc_spmv(nrows, _ptr(row_ptr), _ptr(col), _ptr(vals), _ptr(u), alpha, beta, _ptr(y))
    return y


def diffuse(row_ptr, col, vals, fixed, dt, steps, u):
    lib = _load()
    row_ptr = _c(row_ptr, np.int64)
    col = _c(col, np.int32)
    vals = _c(vals, np.float64)
    fixed = _c(fixed, np.uint8)
    u = np.array(u, dtype=np.float64)
    rc = lib.orc_diffuse(len(row_ptr) - 1, _ptr(row_ptr), _ptr(col), _ptr(vals), _ptr(fixed),
                         dt, steps, _ptr(u))
    if rc != OK:
        raise MemoryError("orc_diffuse")
    return u


def diffuse_bc(row_ptr, col, vals, kind, g, dt, steps, u):
    """Explicit steps with internal (0), Dirichlet (1) and Neumann (2) rows,
    eq. exp-start..exp-end (see orc_diffuse_bc); g [nrows] or None."""
    lib = _load()
    row_ptr = _c(row_ptr, np.int64)
    col = _c(col, np.int32)
    vals = _c(vals, np.float64)
    kind = _c(kind, np.uint8)
    gg = None if g is None else _c(g, np.float64)
    u = np.array(u, dtype=np.float64)
    rc = lib.orc_diffuse_bc(len(row_ptr) - 1, _ptr(row_ptr), _ptr(col), _ptr(vals), _ptr(kind),
                            _ptr(gg), dt, steps, _ptr(u))
    if rc != OK:
        raise MemoryError("orc_diffuse_bc")
    return u


def sort_rows(row_ptr, col, vals):
    """The same CSR matrix with the columns of every row in ascending order."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    row_of = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    order = np.lexsort((col, row_of))
    return row_ptr.copy(), col[order].astype(np.int32), np.asarray(vals, dtype=np.float64)[order]


def ilu0(row_ptr, col, vals):
    """ILU(0) factors of a CSR matrix with sorted rows and a diagonal in every
    row: (factor values in the same pattern, diagonal positions)."""
    lib = _load()
    row_ptr = _c(row_ptr, np.int64)
    col = _c(col, np.int32)
    f = np.array(vals, dtype=np.float64)
    n = len(row_ptr) - 1
    diag = np.zeros(n, dtype=np.int64)
    rc = lib.orc_ilu0(n, _ptr(row_ptr), _ptr(col), _ptr(f), _ptr(diag))
    if rc != OK:
        raise ValueError(f"orc_ilu0 rc={rc}")
    return f, diag


def ilu0_solve(row_ptr, col, fvals, diag, b):
    lib = _load()
    row_ptr = _c(row_ptr, np.int64)
    col = _c(col, np.int32)
    fvals = _c(fvals, np.float64)
    diag = _c(diag, np.int64)
    b = _c(b, np.float64)
    x = np.zeros(len(b))
    lib.orc_ilu0_solve(len(b), _ptr(row_ptr), _ptr(col), _ptr(fvals), _ptr(diag), _ptr(b), _ptr(x))
    return x


def bicgstab(row_ptr, col, vals, b, x0=None, precondition=True, tol=1e-12, maxit=5000):
    """BiCGSTAB with ILU(0) (or no) preconditioning on a CSR matrix with
    sorted rows: (x, converged, iterations, relative residual)."""
    lib = _load()
    row_ptr = _c(row_ptr, np.int64)
    col = _c(col, np.int32)
    vals = _c(vals, np.float64)
    b = _c(b, np.float64)
    x = np.zeros(len(b)) if x0 is None else np.array(x0, dtype=np.float64)
    f, diag = ilu0(row_ptr, col, vals) if precondition else (None, None)
    it, res = C.c_int(0), C.c_double(0.0)
    rc = lib.orc_bicgstab(len(b), _ptr(row_ptr), _ptr(col), _ptr(vals), _ptr(f), _ptr(diag), _ptr(b),
                          _ptr(x), tol, maxit, C.byref(it), C.byref(res))
    return x, rc == OK, it.value, res.value


def combine_operators(row_ptr, terms, coefs, rows=None):
    """General second-order operator from derivative weights (eq. gen-op):
    w_L[e] = sum_t a_t(i) w_t[e] for every entry e of row i; coefs[t] is a
    per-node array [nrows] or None (coefficient 1).  Rows outside ``rows``
    (a (begin, end) pair) are zero."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    nrows = len(row_ptr) - 1
    rb, re = (0, nrows) if rows is None else rows
    row_of = np.repeat(np.arange(nrows), np.diff(row_ptr))
    out = np.zeros(int(row_ptr[-1]))
    sel = (row_of >= rb) & (row_of < re)
    for w, a in zip(terms, coefs):
        c = np.ones(nrows) if a is None else np.asarray(a, dtype=np.float64)
        out[sel] += c[row_of[sel]] * np.asarray(w)[sel]
    return out


# ------------------------------------------------- projection / residual check
def project_lap(pts, stencil, k, m, w_tilde):
    lib = _load()
    pts = _c(pts, np.float64)
    st = _c(stencil, np.int32)
    wt = _c(w_tilde, np.float64)
    out = np.zeros(len(st))
    rc = lib.orc_project_lap(pts.shape[1], _ptr(pts), len(st), _ptr(st), k, m, _ptr(wt), _ptr(out))
    if rc != OK:
        raise ValueError(f"orc_project_lap rc={rc}")
    return out


def phi_residual_lap(pts, stencil, k, m, w) -> float:
    lib = _load()
    pts = _c(pts, np.float64)
    st = _c(stencil, np.int32)
    w = _c(w, np.float64)
    return lib.orc_phi_residual_lap(pts.shape[1], _ptr(pts), len(st), _ptr(st), k, m, _ptr(w))


# ------------------------------------------------------------------------ MLP
def mlp_nparams(n_in, H, L, n_out) -> int:
    return int(_load().orc_mlp_nparams(n_in, H, L, n_out))


def mlp_forward(n_in, H, L, n_out, params, x, targets=None):
    lib = _load()
    params = _c(params, np.float64)
    x = _c(x, np.float64)
    B = x.shape[0]
    y = np.zeros((B, n_out))
    t = None if targets is None else _c(targets, np.float64)
    loss = lib.orc_mlp_forward(n_in, H, L, n_out, _ptr(params), B, _ptr(x), _ptr(t), _ptr(y))
    return y, loss


def mlp_grad(n_in, H, L, n_out, params, x, targets):
    lib = _load()
    params = _c(params, np.float64)
    x = _c(x, np.float64)
    t = _c(targets, np.float64)
    g = np.zeros_like(params)
    loss = lib.orc_mlp_grad(n_in, H, L, n_out, _ptr(params), x.shape[0], _ptr(x), _ptr(t), _ptr(g))
    return loss, g


def adam(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step on copies; returns (params, m, v)."""
    lib = _load()
    p = np.array(params, dtype=np.float64)
    m = np.array(m, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    g = _c(grads, np.float64)
    lib.orc_adam(len(p), _ptr(p), _ptr(g), _ptr(m), _ptr(v), t, lr, b1, b2, eps)
    return p, m, v
