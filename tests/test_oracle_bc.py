"""Pins of the oracle's Neumann update (eq. exp-end) and of the general
second-order operator built from derivative weights (eq. gen-op); CPU only."""
import numpy as np
import pytest

import nodesets as NS


def test_diffuse_bc_without_neumann_rows_is_diffuse(oracle):
    rng = np.random.default_rng(0)
    n, N = 5, 60
    rp = np.arange(N + 1, dtype=np.int64) * n
    col = np.concatenate([[i] + list(rng.choice(np.delete(np.arange(N), i), n - 1, replace=False))
                          for i in range(N)]).astype(np.int32)
    vals = rng.normal(size=N * n)
    kind = (rng.random(N) < 0.2).astype(np.uint8)
    u = rng.normal(size=N)
    a = oracle.diffuse(rp, col, vals, kind, 0.01, 7, u)
    b = oracle.diffuse_bc(rp, col, vals, kind, None, 0.01, 7, u)
    assert np.array_equal(a, b)


def test_neumann_update_by_hand(oracle):
    """Four nodes: 0 and 3 internal, 1 Neumann (its row: centre weight 4,
    neighbours 0 and 3 with -1 and -3), 2 Dirichlet; two steps worked out by
    hand, each from the previous step's values."""
    rp = np.array([0, 3, 6, 7, 9])
    col = np.array([0, 1, 2, 1, 0, 3, 2, 3, 2], dtype=np.int32)
    vals = np.array([-2.0, 1.0, 1.0, 4.0, -1.0, -3.0, 1.0, -1.0, 1.0])
    kind = np.array([0, 2, 1, 0], dtype=np.uint8)
    g = np.array([0.0, 0.5, 0.0, 0.0])
    u0 = np.array([1.0, 2.0, 3.0, 4.0])
    one = oracle.diffuse_bc(rp, col, vals, kind, g, 0.1, 1, u0)
    assert np.allclose(one, [1.3, (0.5 + 1.0 + 12.0) / 4, 3.0, 3.9], rtol=0, atol=1e-15)
    two = oracle.diffuse_bc(rp, col, vals, kind, g, 0.1, 2, u0)
    assert np.allclose(two, [1.3 + 0.1 * (-2.6 + 3.375 + 3.0), (0.5 + 1.3 + 11.7) / 4, 3.0,
                             3.9 + 0.1 * (-3.9 + 3.0)], rtol=0, atol=1e-14)


def disk_operator(oracle, N=3000, seed=3):
    """Disk with holes: Laplacian rows inside, d/dn rows on the boundary
    (RBF-FD weights of the oracle), the kinds of the Poisson problem."""
    ns = NS.disk_holes(N, seed=seed)
    (ib, ie), (bb, be) = ns.classes["interior"], ns.classes["boundary"]
    sizes = np.zeros(ns.N, dtype=np.int64)
    sizes[ib:ie], sizes[bb:be] = 25, 30
    rp = np.zeros(ns.N + 1, dtype=np.int64)
    np.cumsum(sizes, out=rp[1:])
    col = np.zeros(rp[-1], dtype=np.int32)
    idx, _ = oracle.knn(ns.pts, 25, queries=np.arange(ib, ie), nthreads=8)
    col[rp[ib]:rp[ie]] = idx.ravel()
    idx, _ = oracle.knn(ns.pts, 30, queries=np.arange(bb, be), nthreads=8)
    col[rp[bb]:rp[be]] = idx.ravel()
    vals = np.zeros(rp[-1])
    v, st, _ = oracle.weights(ns.pts, rp, col, 5, 4, 1, normals=ns.normals, rows=(ib, ie), nthreads=8)
    vals[rp[ib]:rp[ie]] = v[0][rp[ib]:rp[ie]]
    v, st2, _ = oracle.weights(ns.pts, rp, col, 5, 4, 16, normals=ns.normals, rows=(bb, be), nthreads=8)
    vals[rp[bb]:rp[be]] = v[0][rp[bb]:rp[be]]
    kind = np.zeros(ns.N, dtype=np.uint8)
    kind[ns.dirichlet] = 1
    kind[ns.neumann] = 2
    return ns, rp, col, vals, kind


def test_linear_field_is_kept(oracle):
    """u = 1 + 2x - 3y: the Laplacian rows give 0 and the d/dn rows with
    g = grad u . n reproduce u, so a step leaves it unchanged (to the rows'
    residuals over the centre weight).  Only one step: the Neumann update
    divides by the centre d/dn weight, which on these one-sided stencils is
    as small as ~1e-2 against neighbours of ~1e2, so coupled Neumann nodes
    amplify rounding from step to step."""
    ns, rp, col, vals, kind = disk_operator(oracle)
    assert (kind == 2).any() and (kind == 1).any()
    u = 1 + 2 * ns.pts[:, 0] - 3 * ns.pts[:, 1]
    g = 2 * ns.normals[:, 0] - 3 * ns.normals[:, 1]
    out = oracle.diffuse_bc(rp, col, vals, kind, g, 1e-7, 1, u)
    assert np.abs(out - u).max() <= 1e-9 * np.abs(u).max()
    # a wrong Neumann datum moves the Neumann nodes
    bad = oracle.diffuse_bc(rp, col, vals, kind, g + 0.1, 1e-7, 1, u)
    assert np.abs(bad - u)[kind == 2].min() > 1e-6


def test_general_operator_is_exact_on_quadratics(oracle):
    """w_L = sum_t a_t(i) w_t with the RBF-FD weights of d/dx, d/dy, d2/dx2,
    d2/dxdy, d2/dy2 (degree-4 monomials reproduced) and random per-node
    coefficients: w_L^T p(x_I(i)) = sum_t a_t(i) (d_t p)(x_i) for a quadratic p."""
    ns = NS.disk_holes(3000, seed=5)
    b, e = ns.classes["interior"]
    rows = np.arange(b, b + 400)
    idx, _ = oracle.knn(ns.pts, 25, queries=rows, nthreads=8)
    rp = np.zeros(ns.N + 1, dtype=np.int64)
    rp[rows + 1] = 25
    rp = np.cumsum(rp)
    col = np.zeros(rp[-1], dtype=np.int32)
    col[:] = idx.ravel()
    ops = 2 | 4 | 32 | 64 | 128
    v, st, _ = oracle.weights(ns.pts, rp, col, 5, 4, ops, rows=(b, b + 400), nthreads=8)
    assert (st[b:b + 400] == 0).all()
    rng = np.random.default_rng(1)
    coefs = [rng.normal(size=ns.N) for _ in range(5)]
    coefs[2] = None                                   # coefficient 1
    wL = oracle.combine_operators(rp, list(v), coefs, rows=(b, b + 400))
    x, y = ns.pts[:, 0], ns.pts[:, 1]
    p = 1 + 2 * x - y + 3 * x * x - x * y + 0.5 * y * y
    dp = [2 + 6 * x - y, -1 - x + y, np.full(ns.N, 6.0), np.full(ns.N, -1.0), np.full(ns.N, 1.0)]
    for i in rows:
        lhs = float(np.dot(wL[rp[i]:rp[i + 1]], p[col[rp[i]:rp[i + 1]]]))
        ref = sum((1.0 if a is None else a[i]) * d[i] for a, d in zip(coefs, dp))
        scale = np.abs(wL[rp[i]:rp[i + 1]]).sum() * np.abs(p).max()
        assert abs(lhs - ref) <= 1e-11 * scale, (int(i), lhs, ref)
    assert not wL[:rp[b]].any() and not wL[rp[b + 400]:].any()
