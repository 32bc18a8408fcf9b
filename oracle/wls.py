"""Weighted least squares (GWLS) stencil weights, plain numpy in FP64.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this module; the product path never does.

Section 2.2.1 ("Generalized weighted least squares"): around the centre p* the
approximant is u_hat(p) = b((p - p*)/s)^T alpha with basis b = the monomials of
total degree <= m (graded lexicographic order), and alpha minimises
||W (B alpha - u)||_2 with B_ij = b_j((p_i - p*)/s) and W = diag(omega_i),
omega_i = omega((p_i - p*)/s).  The weight function is the Gaussian
omega(x) = exp(-||x||^2 / sigma^2).  Then alpha = (W B)^+ W u and the weights of
an operator L are

    w^T = (L b)(0)^T (W B)^+ W,

the right-hand side taken in the scaled variable, so the stored weights are
w / s^q (q = 1 for first, 2 for second derivatives).  This module evaluates
that formula literally, with the pseudoinverse from numpy's SVD (the paper's
example setup also uses an SVD).  The scale s is the distance to the farthest
node of the stencil ("farthest") or to the closest other node ("nearest", the
paper's example).  Rank-deficient W B (including n < number of basis
functions) gives status SINGULAR and zero weights.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _orc

OK, SINGULAR, BADARG = 0, 1, 4
SCALE_FARTHEST, SCALE_NEAREST = 0, 1

# operator bits: 0 Laplacian, 1..3 d/dx, d/dy, d/dz, 4 d/dn, 5..10 the second
# derivatives xx, xy, yy, xz, yz, zz
_SECOND = {5: (0, 0), 6: (0, 1), 7: (1, 1), 8: (0, 2), 9: (1, 2), 10: (2, 2)}


def op_order(bit: int) -> int:
    return 2 if bit == 0 or bit >= 5 else 1


def rhs(dim: int, m: int, ops: int, normal=None) -> np.ndarray:
    """(L b)(0) for every requested operator (bit order) and monomial b:
    [R, l].  A monomial prod_a x_a^e_a has, at 0, first derivative 1 along a
    exactly when e = unit_a, second derivative 2 along (a, a) when e =
    2 unit_a, and 1 along (a, b), a != b, when e = unit_a + unit_b."""
    E = _orc.monomials(dim, m)
    out = np.zeros((len(_orc.op_list(ops)), len(E)))
    for r, bit in enumerate(_orc.op_list(ops)):
        for j, e in enumerate(E):
            e = tuple(int(v) for v in e)
            unit = [tuple(int(a == c) for c in range(dim)) for a in range(dim)]
            if bit == 0:
                out[r, j] = sum(2.0 for a in range(dim) if e == tuple(2 * v for v in unit[a]))
            elif 1 <= bit <= 3:
                out[r, j] = 1.0 if e == unit[bit - 1] else 0.0
            elif bit == 4:
                out[r, j] = sum(float(normal[a]) for a in range(dim) if e == unit[a])
            else:
                a, b = _SECOND[bit]
                target = tuple(unit[a][c] + unit[b][c] for c in range(dim))
                if e == target:
                    out[r, j] = 2.0 if a == b else 1.0
    return out


def basis_matrix(xi: np.ndarray, m: int) -> np.ndarray:
    """B [n, l]: the monomials of degree <= m at the scaled offsets xi [n, dim]."""
    E = _orc.monomials(xi.shape[1], m)
    return np.prod(xi[:, None, :] ** E[None, :, :], axis=2)


def stencil_weights(x: np.ndarray, m: int, ops: int, sigma: float, scale: int, normal=None):
    """Weights of one stencil, x [n, dim] with the centre first.  Returns
    (w [R, n], status, s, scaled weights [R, n])."""
    n, dim = x.shape
    R = len(_orc.op_list(ops))
    zero = np.zeros((R, n))
    d = x - x[0]
    dist = np.sqrt((d * d).sum(1))
    if n < 1 or not np.all(np.isfinite(d)):
        return zero, BADARG, 0.0, zero
    if scale == SCALE_NEAREST:
        if n < 2 or not (dist[1:].min() > 0):
            return zero, BADARG, 0.0, zero
        s = float(dist[1:].min())
    else:
        if not (dist.max() > 0):
            return zero, BADARG, 0.0, zero
        s = float(dist.max())
    xi = d / s
    omega = np.exp(-(xi * xi).sum(1) / sigma ** 2)
    B = basis_matrix(xi, m)
    WB = omega[:, None] * B
    sv = np.linalg.svd(WB, compute_uv=False)
    l = B.shape[1]
    if n < l or sv[-1] <= max(n, l) * np.finfo(float).eps * sv[0]:
        return zero, SINGULAR, s, zero
    P = np.linalg.pinv(WB)                      # [l, n]
    Lb = rhs(dim, m, ops, normal)               # [R, l]
    ws = (Lb @ P) * omega[None, :]              # w^T = (L b)^T (W B)^+ W
    q = np.array([op_order(b) for b in _orc.op_list(ops)], dtype=float)
    return ws / s ** q[:, None], OK, s, ws


def weights(pts, row_ptr, col, m, ops, sigma, scale, normals=None, rows=None):
    """GWLS weights of CSR rows (rows = (begin, end) or None for all):
    (vals [R, nnz], status [nrows]); rows outside the range stay zero."""
    pts = np.asarray(pts, dtype=np.float64)
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    nrows = len(row_ptr) - 1
    rb, re = (0, nrows) if rows is None else rows
    R = len(_orc.op_list(ops))
    vals = np.zeros((R, int(row_ptr[-1])))
    status = np.zeros(nrows, dtype=np.int32)
    for i in range(rb, re):
        st = col[row_ptr[i]:row_ptr[i + 1]]
        if len(st) == 0 or st[0] != i or st.min() < 0 or st.max() >= len(pts):
            status[i] = BADARG
            continue
        nrm = None if normals is None else normals[i]
        w, status[i], _, _ = stencil_weights(pts[st], m, ops, sigma, scale, nrm)
        vals[:, row_ptr[i]:row_ptr[i + 1]] = w
    return vals, status
