"""Shared test helpers: error measures and monomial-reproduction residuals.

Error measure (per node and per operator):
    ||w_gpu - w_ref||_inf / ||w_ref||_inf
Monomial reproduction, in scaled units (xi = (x - x_c)/s, s = max distance),
    |sum_i w_s,i q_b(xi_i) - (L q_b)(0)| / max(1, sum_i |w_s,i q_b(xi_i)|).
"""
import itertools

import numpy as np

OPS = [("lap", 1), ("dx", 2), ("dy", 4), ("dz", 8), ("dn", 16), ("dxx", 32), ("dxy", 64), ("dyy", 128),
       ("dxz", 256), ("dyz", 512), ("dzz", 1024)]
SECOND = {"dxx": (0, 0), "dxy": (0, 1), "dyy": (1, 1), "dxz": (0, 2), "dyz": (1, 2), "dzz": (2, 2)}


def op_order(name):
    """Derivative order q of an operator (weights scale by s^-q)."""
    return 2 if name == "lap" or name in SECOND else 1


def op_names(ops):
    return [name for name, b in OPS if ops & b]


def exps_graded(dim, m):
    out = []
    for deg in range(m + 1):
        out.extend(e for e in itertools.product(range(deg, -1, -1), repeat=dim) if sum(e) == deg)
    return np.array(out, dtype=np.int64)


def lop(e, name, normal):
    e = np.asarray(e)
    if name == "lap":
        return 2.0 if (e.sum() == 2 and e.max() == 2) else 0.0
    if name == "dn":
        return float(sum(normal[a] for a in range(len(e)) if e.sum() == 1 and e[a] == 1))
    if name in SECOND:
        a, b = SECOND[name]
        if e.sum() != 2:
            return 0.0
        if a == b:
            return 2.0 if e[a] == 2 else 0.0
        return 1.0 if (e[a] == 1 and e[b] == 1) else 0.0
    a = {"dx": 0, "dy": 1, "dz": 2}[name]
    return 1.0 if (e.sum() == 1 and e[a] == 1) else 0.0


def rel_err_rows(w_gpu, w_ref, row_ptr, rows):
    """Per-row relative inf-norm error for the given rows."""
    out = np.empty(len(rows))
    for t, i in enumerate(rows):
        a, b = row_ptr[i], row_ptr[i + 1]
        den = np.abs(w_ref[a:b]).max()
        out[t] = np.abs(w_gpu[a:b] - w_ref[a:b]).max() / (den if den > 0 else 1.0)
    return out


def monomial_residual(pts, normals, row_ptr, col, w, name, m, rows):
    """Max scaled monomial-reproduction residual over the rows (unscaled
    weights w; operator order q rescales them by s^q)."""
    dim = pts.shape[1]
    E = exps_graded(dim, m)
    q = op_order(name)
    worst = 0.0
    for i in rows:
        a, b = row_ptr[i], row_ptr[i + 1]
        st = col[a:b]
        d = pts[st] - pts[st[0]]
        s = np.sqrt((d ** 2).sum(1)).max()
        xi = d / s
        ws = w[a:b] * s ** q
        Qm = np.stack([np.prod(xi ** e, axis=1) for e in E], axis=1)
        nrm = normals[i] if normals is not None else None
        lq = np.array([lop(e, name, nrm) for e in E])
        terms = ws[:, None] * Qm
        res = np.abs(terms.sum(0) - lq) / np.maximum(1.0, np.abs(terms).sum(0))
        worst = max(worst, res.max())
    return worst


def oracle_rows(oracle, pts, normals, rp, col, rows, k, m, ops, nthreads=8):
    """Oracle weights for arbitrary rows of a CSR stencil pattern (the rows'
    stencils renumbered locally, centres first): dict row -> [R, n] array."""
    rows = np.asarray(rows)
    st_list = [col[rp[i]:rp[i + 1]] for i in rows]
    others = np.setdiff1d(np.unique(np.concatenate(st_list)), rows)
    order = np.concatenate([rows, others])
    remap = np.full(pts.shape[0], -1, dtype=np.int64)
    remap[order] = np.arange(len(order))
    Nl = None if normals is None else normals[order]
    lcol = np.concatenate([remap[s] for s in st_list]).astype(np.int32)
    lrp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum([len(s) for s in st_list], out=lrp[1:])
    vals, status, _ = oracle.weights(pts[order], lrp, lcol, k, m, ops, normals=Nl,
                                     rows=(0, len(rows)), nthreads=nthreads)
    assert (status == 0).all()
    return {int(i): vals[:, lrp[t]:lrp[t + 1]] for t, i in enumerate(rows)}
