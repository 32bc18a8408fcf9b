"""Pins of the CPU oracle against facts fixed by the paper and the mathematics.

Each test checks the oracle against something other than itself: brute force,
closed forms, invariants, a library solver, numerical differentiation of the
interpolant, convergence orders.  None of them needs a GPU.
"""
import itertools
import math
import os

import numpy as np
import pytest

import nodesets as NS

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers
def exps_graded(dim, m):
    """Exponents of the degree <= m monomials, enumerated independently of
    the oracle (itertools), in graded order with x_0's exponent descending."""
    out = []
    for deg in range(m + 1):
        tup = [e for e in itertools.product(range(deg, -1, -1), repeat=dim) if sum(e) == deg]
        out.extend(tup)
    return np.array(out, dtype=np.int64)


def lop_monomial(e, op, normal=None):
    """Operator applied to x^e at the origin (Laplacian, d/dx_a, d/dn,
    d2/dx_a dx_b): the derivative of x^e is nonzero at 0 only for the one
    monomial whose exponents match the derivative orders."""
    e = np.asarray(e)
    if op == "lap":
        return 2.0 if (e.sum() == 2 and e.max() == 2) else 0.0
    if op == "dn":
        return float(sum(normal[a] for a in range(len(e)) if e.sum() == 1 and e[a] == 1))
    if len(op) == 3:                                 # dxx, dxy, ... : d/dx_a d/dx_b
        a, b = "xyz".index(op[1]), "xyz".index(op[2])
        want = np.zeros(len(e), dtype=int)
        want[a] += 1
        want[b] += 1
        return float(math.factorial(want[a]) * (1 if a == b else math.factorial(want[b]))) \
            if np.array_equal(e, want) else 0.0
    a = {"dx": 0, "dy": 1, "dz": 2}[op]
    return 1.0 if (e.sum() == 1 and e[a] == 1) else 0.0


OPNAMES = [("lap", 1), ("dx", 2), ("dy", 4), ("dz", 8), ("dn", 16), ("dxx", 32), ("dxy", 64), ("dyy", 128),
           ("dxz", 256), ("dyz", 512), ("dzz", 1024)]


def random_stencils(ns, n, count, seed, oracle):
    rng = np.random.default_rng(seed)
    q = np.sort(rng.choice(ns.N, size=count, replace=False))
    idx, st = oracle.knn(ns.pts, n, queries=q, nthreads=4)
    assert (st == 0).all()
    return q, idx


def one_row_csr(stencil):
    return np.array([0, len(stencil)], dtype=np.int64)


def weights_for(oracle, pts, stencils, k, m, ops, normals=None, quad=False, scaled=False):
    """Oracle weights for a list of stencils (rows = their centres)."""
    # re-index: a local point set whose row i has centre i
    rows = len(stencils)
    n = stencils.shape[1]
    sub = np.unique(stencils.ravel())
    centres = stencils[:, 0]
    others = np.setdiff1d(sub, centres)
    order = np.concatenate([centres, others])
    remap = {int(g): i for i, g in enumerate(order)}
    P = pts[order]
    Nn = None if normals is None else normals[order]
    col = np.array([[remap[int(g)] for g in row] for row in stencils], dtype=np.int32).ravel()
    rp = np.arange(rows + 1, dtype=np.int64) * n
    res = oracle.weights(P, rp, col, k, m, ops, normals=Nn, rows=(0, rows), quad=quad,
                         scaled=scaled)
    return res, P, col.reshape(rows, n)


# ------------------------------------------------------------------ monomials
@pytest.mark.parametrize("dim", [2, 3])
def test_monomial_table(oracle, dim):
    for m in range(0, 7):
        E = oracle.monomials(dim, m)
        assert len(E) == math.comb(m + dim, dim)
        assert (E == exps_graded(dim, m)).all()


# ------------------------------------------------------------------------ kNN
@pytest.mark.parametrize("dim,n", [(2, 1), (2, 6), (2, 12), (2, 25), (3, 10), (3, 35)])
def test_knn_matches_sort(oracle, dim, n):
    rng = np.random.default_rng(dim * 100 + n)
    pts = rng.uniform(size=(400, dim))
    idx, st = oracle.knn(pts, n)
    assert (st == 0).all()
    for c in range(0, 400, 7):
        d2 = ((pts - pts[c]) ** 2).sum(axis=1)
        order = np.lexsort((np.arange(400), d2))
        order = order[order != c]
        assert idx[c, 0] == c
        assert (idx[c, 1:] == order[: n - 1]).all()


def test_knn_grid_ties(oracle):
    g = np.arange(10.0)
    X, Y = np.meshgrid(g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel()], 1)
    c = 5 * 10 + 5
    idx, _ = oracle.knn(pts, 9, queries=[c])
    # centre, 4 axis neighbours by index, then 4 diagonal neighbours by index
    assert idx[0].tolist() == [55, 45, 54, 56, 65, 44, 46, 64, 66]


def test_knn_duplicate_flagged(oracle):
    pts = np.array([[0, 0], [1, 0], [0, 1], [0, 0], [2, 2.0]])
    _, st = oracle.knn(pts, 3)
    assert st[0] == oracle.DUPLICATE and st[3] == oracle.DUPLICATE
    assert st[1] == 0


# ------------------------------------------------------------------------- LU
def test_lu_matches_library(oracle):
    rng = np.random.default_rng(1)
    for M in (5, 18, 40, 80):
        K = rng.normal(size=(M, M)) + M * np.eye(M) * 0.1
        B = rng.normal(size=(M, 3))
        X, rc = oracle.lu_solve(K, B)
        assert rc == 0
        ref = np.linalg.solve(K, B)
        assert np.abs(X - ref).max() <= 1e-11 * np.abs(ref).max()


def test_lu_needs_pivoting_and_flags_singular(oracle):
    K = np.array([[0.0, 1.0], [1.0, 0.0]])
    X, rc = oracle.lu_solve(K, np.array([2.0, 3.0]))
    assert rc == 0 and np.allclose(X, [3.0, 2.0])
    K = np.array([[1.0, 2.0], [2.0, 4.0]])
    _, rc = oracle.lu_solve(K, np.array([1.0, 1.0]))
    assert rc == oracle.SINGULAR


# ---------------------------------------------------------------- closed forms
def load_closed_forms():
    cases, cur = [], None
    with open(os.path.join(GOLDEN, "closed_form_stencils.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tag, rest = line.split(None, 1)
            if tag == "case":
                name, op, q = rest.split()
                cur = {"name": name, "op": op, "q": int(q)}
                cases.append(cur)
            elif tag == "nodes":
                cur["nodes"] = np.array([[float(v) for v in p.split()] for p in rest.split("|")])
            elif tag == "w":
                cur["w"] = np.array([float(v) for v in rest.split()])
    return cases


OPBIT = {"lap": 1, "dx": 2, "dy": 4, "dz": 8, "dxx": 32, "dxy": 64, "dyy": 128, "dxz": 256, "dyz": 512,
         "dzz": 1024}


@pytest.mark.parametrize("case", load_closed_forms(), ids=lambda c: c["name"] + "_" + c["op"])
@pytest.mark.parametrize("k", [3, 5, 7])
def test_closed_form_stencils(oracle, case, k):
    for h in (1.0, 0.01, 3e-4):
        for shift in (0.0, 0.37):
            pts = case["nodes"] * h + shift
            n = len(pts)
            vals, st, _ = oracle.weights(pts, one_row_csr(pts), np.arange(n, dtype=np.int32),
                                         k, 2, OPBIT[case["op"]], rows=(0, 1))
            assert st[0] == 0
            got = vals[0] * h ** case["q"]
            assert np.abs(got - case["w"]).max() <= 1e-12 * max(1.0, np.abs(case["w"]).max())


# ------------------------------------------------------- monomial reproduction
def scaled_offsets(pts, stencil):
    d = pts[stencil] - pts[stencil[0]]
    s = np.sqrt((d ** 2).sum(1)).max()
    return d / s, s


@pytest.mark.parametrize("cfg", [("square", 12, 3, 2), ("disk", 25, 5, 4), ("disk", 30, 5, 4),
                                 ("ball", 35, 3, 2), ("ball", 60, 3, 3), ("ball", 45, 3, 2)])
def test_monomial_reproduction(oracle, cfg):
    kind, n, k, m = cfg
    ns = {"square": lambda: NS.square(0.02), "disk": lambda: NS.disk_holes(15000, seed=3),
          "ball": lambda: NS.ball(20000, seed=4)}[kind]()
    dim = ns.dim
    ops = 1 | 2 | 4 | (8 if dim == 3 else 0) | 16 | 32 | 64 | 128 | ((256 | 512 | 1024) if dim == 3 else 0)
    rng = np.random.default_rng(5)
    normals = rng.normal(size=ns.pts.shape)
    normals /= np.linalg.norm(normals, axis=1, keepdims=True)
    _, stencils = random_stencils(ns, n, 40, 11, oracle)
    # local numbering: row r has centre r
    rows = len(stencils)
    sub_c = stencils[:, 0]
    others = np.setdiff1d(np.unique(stencils.ravel()), sub_c)
    order = np.concatenate([sub_c, others])
    remap = {int(g): i for i, g in enumerate(order)}
    P = ns.pts[order]
    Nl = normals[order]
    col = np.array([[remap[int(g)] for g in row] for row in stencils], dtype=np.int32)
    rp = np.arange(rows + 1, dtype=np.int64) * n
    vals, st, scale, svals = oracle.weights(P, rp, col.ravel(), k, m, ops, normals=Nl,
                                            rows=(0, rows), scaled=True)
    assert (st == 0).all()
    E = exps_graded(dim, m)
    names = [o for o, b in OPNAMES if ops & b]
    for r in range(rows):
        xi, s = scaled_offsets(P, col[r])
        assert abs(s - scale[r]) <= 1e-15 * s
        Qm = np.stack([np.prod(xi ** e, axis=1) for e in E], axis=1)   # [n, l]
        for oi, name in enumerate(names):
            ws = svals[oi, r * n:(r + 1) * n]
            lq = np.array([lop_monomial(e, name, Nl[r]) for e in E])
            terms = ws[:, None] * Qm
            resid = np.abs(terms.sum(0) - lq) / np.maximum(1.0, np.abs(terms).sum(0))
            assert resid.max() <= 1e-12, (name, resid.max())
            # unscaled weights = scaled / s^q
            q = 1 if name in ("dx", "dy", "dz", "dn") else 2
            assert np.allclose(vals[oi, r * n:(r + 1) * n] * s ** q, ws, rtol=1e-13, atol=0)
        # zero row sums of every derivative operator
        for oi in range(len(names)):
            w = svals[oi, r * n:(r + 1) * n]
            assert abs(w.sum()) <= 1e-12 * np.abs(w).sum()


# ------------------------------------- weights = operator of the interpolant
def phs_interpolant(xi, u, k, m):
    """Textbook PHS + polynomial interpolant of data u at nodes xi: returns a
    function s(x).  Built here with numpy, independently of the oracle."""
    n, dim = xi.shape
    E = exps_graded(dim, m)
    D = np.sqrt(((xi[:, None, :] - xi[None, :, :]) ** 2).sum(-1))
    Pm = np.stack([np.prod(xi ** e, axis=1) for e in E], axis=1)
    l = len(E)
    S = np.zeros((n + l, n + l))
    S[:n, :n] = D ** k
    S[:n, n:] = Pm
    S[n:, :n] = Pm.T
    coef = np.linalg.solve(S, np.concatenate([u, np.zeros(l)]))
    c, d = coef[:n], coef[n:]

    def s(x):
        x = np.atleast_2d(x)
        r = np.sqrt(((x[:, None, :] - xi[None, :, :]) ** 2).sum(-1))
        px = np.stack([np.prod(x ** e, axis=1) for e in E], axis=1)
        return (r ** k) @ c + px @ d
    return s


def fd_operator(s, dim, op, normal, delta):
    """Central finite differences of s at the origin, Richardson-extrapolated
    over steps delta, delta/2, delta/4 to cancel error terms in delta and
    delta^2 (the r^k kernel centred at the origin contributes an error linear
    in delta to the second difference, the smooth parts even powers)."""
    def once(dl):
        z = np.zeros(dim)
        if op == "lap":
            acc = 0.0
            for a in range(dim):
                e = np.zeros(dim); e[a] = dl
                acc += (s(z + e)[0] - 2 * s(z)[0] + s(z - e)[0]) / dl ** 2
            return acc
        if len(op) == 3:                             # d2/dx_a dx_b
            a, b = "xyz".index(op[1]), "xyz".index(op[2])
            ea = np.zeros(dim); ea[a] = dl
            eb = np.zeros(dim); eb[b] = dl
            if a == b:
                return (s(z + ea)[0] - 2 * s(z)[0] + s(z - ea)[0]) / dl ** 2
            return (s(z + ea + eb)[0] - s(z + ea - eb)[0] - s(z - ea + eb)[0] + s(z - ea - eb)[0]) / (4 * dl ** 2)
        direc = np.zeros(dim)
        if op == "dn":
            direc = np.asarray(normal, float)
        else:
            direc[{"dx": 0, "dy": 1, "dz": 2}[op]] = 1.0
        return (s(z + dl * direc)[0] - s(z - dl * direc)[0]) / (2 * dl)
    a, b, c = once(delta), once(delta / 2), once(delta / 4)
    l1, l2 = 2 * b - a, 2 * c - b
    return (4 * l2 - l1) / 3


@pytest.mark.parametrize("cfg", [(2, 12, 3, 2), (2, 25, 5, 4), (3, 20, 3, 2), (3, 30, 5, 3)])
def test_weights_differentiate_the_interpolant(oracle, cfg):
    """w^T u equals L applied to the local PHS + polynomial interpolant of u
    at the centre: this is what the augmented system of Section 2.2.2
    encodes, checked here through a separately built interpolant and
    numerical differentiation (pins A, Q, l_phi and l_q together)."""
    dim, n, k, m = cfg
    rng = np.random.default_rng(sum(cfg))
    pts = rng.uniform(-1, 1, size=(n, dim))
    pts[0] = 0.0
    pts = pts * 0.05 + 0.3
    normal = rng.normal(size=dim)
    normal /= np.linalg.norm(normal)
    nrm = np.tile(normal, (n, 1))
    ops = 1 | 2 | 4 | (8 if dim == 3 else 0) | 16 | 32 | 64 | 128 | ((256 | 512 | 1024) if dim == 3 else 0)
    names = [o for o, b in OPNAMES if ops & b]
    vals, st, scale, svals = oracle.weights(pts, one_row_csr(pts), np.arange(n, dtype=np.int32),
                                            k, m, ops, normals=nrm, rows=(0, 1), scaled=True)
    assert st[0] == 0
    xi, s = scaled_offsets(pts, np.arange(n))
    for trial in range(3):
        u = rng.normal(size=n)
        sfun = phs_interpolant(xi, u, k, m)
        for oi, name in enumerate(names):
            ref = fd_operator(sfun, dim, name, normal, 2e-3)
            got = svals[oi] @ u
            scale_ref = np.abs(svals[oi] * u).sum()
            assert abs(got - ref) <= 2e-6 * scale_ref, (name, got, ref)


# ---------------------------------------------------------------- invariances
def test_dilation_shift_rotation(oracle):
    ns = NS.disk_holes(8000, seed=7)
    _, stencils = random_stencils(ns, 25, 20, 3, oracle)
    (v0, st0, _), P, col = weights_for(oracle, ns.pts, stencils, 5, 4, 1 | 2 | 4)
    th = 0.7
    Rm = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    alpha = 3.7
    P2 = (P @ Rm.T) * alpha + np.array([10.0, -4.0])
    rows = len(stencils)
    rp = np.arange(rows + 1, dtype=np.int64) * 25
    v1, st1, _ = oracle.weights(P2, rp, col.ravel(), 5, 4, 1 | 2 | 4, rows=(0, rows))
    assert (st0 == 0).all() and (st1 == 0).all()
    for r in range(rows):
        sl = slice(r * 25, (r + 1) * 25)
        lap0, lap1 = v0[0, sl], v1[0, sl] * alpha ** 2
        assert np.abs(lap1 - lap0).max() <= 1e-9 * np.abs(lap0).max()
        # gradient weights rotate covariantly: w'_grad = R w_grad / alpha
        g0 = np.stack([v0[1, sl], v0[2, sl]])
        g1 = np.stack([v1[1, sl], v1[2, sl]]) * alpha
        assert np.abs(Rm @ g0 - g1).max() <= 1e-9 * np.abs(g0).max()


def test_grid_symmetry(oracle):
    h = 0.1
    g = np.array([(i, j) for i in (-1, 0, 1) for j in (-1, 0, 1)], float) * h
    order = [4, 3, 5, 1, 7, 0, 2, 6, 8]        # centre first
    pts = g[order]
    vals, st, _ = oracle.weights(pts, one_row_csr(pts), np.arange(9, dtype=np.int32), 3, 2,
                                 1 | 2 | 4, rows=(0, 1))
    lap, dx, dy = vals
    # nodes: 0 (0,0), 1 (0,-1), 2 (0,1), 3 (-1,0), 4 (1,0), 5 (-1,-1), 6 (-1,1), 7 (1,-1), 8 (1,1)
    tol = 1e-10 * abs(dx[4])
    assert np.ptp(lap[1:5]) <= 1e-10 * abs(lap[1]) and np.ptp(lap[5:]) <= 1e-10 * abs(lap[1])
    assert abs(lap.sum()) <= 1e-10 * abs(lap[0])
    assert abs(dx[3] + dx[4]) <= tol and abs(dx[1]) <= tol and abs(dx[2]) <= tol and abs(dx[0]) <= tol
    assert abs(dx[5] - dx[6]) <= tol and abs(dx[7] - dx[8]) <= tol and abs(dx[5] + dx[8]) <= tol
    assert abs(dy[1] + dy[2]) <= tol and abs(dy[3]) <= tol and abs(dy[4]) <= tol
    assert abs(dy[2] - dx[4]) <= tol and abs(dy[6] - dx[7]) <= tol


# ---------------------------------------------------------- higher precision
@pytest.mark.parametrize("cfg", [("disk", 25, 5, 4), ("ball", 35, 3, 2)])
def test_fp64_oracle_within_conditioning_of_f128(oracle, cfg):
    kind, n, k, m = cfg
    ns = NS.disk_holes(10000, seed=2) if kind == "disk" else NS.ball(15000, seed=2)
    _, stencils = random_stencils(ns, n, 25, 9, oracle)
    (v64, s64, _), P, col = weights_for(oracle, ns.pts, stencils, k, m, 1 | 2)
    (v128, s128, _), _, _ = weights_for(oracle, ns.pts, stencils, k, m, 1 | 2, quad=True)
    assert (s64 == 0).all() and (s128 == 0).all()
    for r in range(len(stencils)):
        kap = oracle.kkt_cond1(P, col[r], k, m)
        sl = slice(r * n, (r + 1) * n)
        for o in range(2):
            err = np.abs(v64[o, sl] - v128[o, sl]).max() / np.abs(v128[o, sl]).max()
            assert err <= max(1e-13, 20 * kap * 1.1e-16), (r, o, err, kap)


def test_cond1_matches_library(oracle):
    ns = NS.disk_holes(5000, seed=1)
    _, stencils = random_stencils(ns, 25, 6, 2, oracle)
    for st in stencils:
        K, _, _, _ = oracle.kkt(ns.pts, st, 5, 4, 1)
        assert abs(oracle.kkt_cond1(ns.pts, st, 5, 4) / np.linalg.cond(K, 1) - 1) < 1e-6
        assert np.allclose(K, K.T, rtol=0, atol=0)


# --------------------------------------------------------- pipeline (E1, E6)
def test_laplacian_error_falls_with_h(oracle):
    """Section 3.2 setup 5: r^5 + degree-2 monomials on 12 closest nodes of a
    regular grid, u = sin(pi x) sin(pi y); the max Laplacian error falls as
    h falls."""
    errs = []
    for h in (1 / 10, 1 / 20, 1 / 40):
        P = NS.regular_grid(h)
        idx, _ = oracle.knn(P, 12, nthreads=4)
        rp = NS.csr_uniform(len(P), 12)
        v, st, _ = oracle.weights(P, rp, idx.ravel(), 5, 2, 1, nthreads=4)
        assert (st == 0).all()
        lap = oracle.spmv(rp, idx.ravel(), v[0], NS.sin_product(P))
        errs.append(np.abs(lap - NS.sin_product_lap(P)).max())
    assert errs[0] > errs[1] > errs[2]


def poisson_error(oracle, h, n=12, k=3, m=2, seed=0):
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    ns = NS.square(h, seed=seed)
    idx, _ = oracle.knn(ns.pts, n, nthreads=8)
    rp = NS.csr_uniform(ns.N, n)
    v, st, _ = oracle.weights(ns.pts, rp, idx.ravel(), k, m, 1, nthreads=8)
    assert (st == 0).all()
    A = sp.csr_matrix((v[0], idx.ravel(), rp), shape=(ns.N, ns.N)).tolil()
    u = NS.sin_product(ns.pts)
    rhs = NS.sin_product_lap(ns.pts)
    b0, b1 = ns.classes["boundary"]
    for i in range(b0, b1):          # Dirichlet rows (Section 2.3.2): M_ii = 1, r_i = g_d
        A.rows[i] = [i]
        A.data[i] = [1.0]
        rhs[i] = u[i]
    sol = spla.spsolve(A.tocsr(), rhs)
    return np.abs(sol - u).max()


def test_poisson_convergence_order(oracle):
    """Manufactured Dirichlet Poisson problem on the jittered unit square
    (n = 12, r^3, m = 2): slope of the max error in h at least m - 1 = 1,
    observed close to 2."""
    hs = [0.04, 0.02, 0.01]
    errs = [poisson_error(oracle, h) for h in hs]
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert slope >= 1.0, (errs, slope)
    assert slope >= 1.6, (errs, slope)


# ------------------------------------------------------- operator application
def test_spmv_and_diffuse(oracle):
    import scipy.sparse as sp
    rng = np.random.default_rng(0)
    N, n = 500, 9
    rp = NS.csr_uniform(N, n)
    col = rng.integers(0, N, size=N * n).astype(np.int32)
    vals = rng.normal(size=N * n)
    u = rng.normal(size=N)
    y0 = rng.normal(size=N)
    A = sp.csr_matrix((vals, col, rp), shape=(N, N))
    y = oracle.spmv(rp, col, vals, u, alpha=0.5, beta=-2.0, y=y0)
    assert np.allclose(y, 0.5 * (A @ u) - 2.0 * y0, rtol=1e-13, atol=1e-13)
    fixed = (rng.uniform(size=N) < 0.2).astype(np.uint8)
    ref = u.copy()
    for _ in range(5):
        ref = np.where(fixed == 1, ref, ref + 0.01 * (A @ ref))
    got = oracle.diffuse(rp, col, vals, fixed, 0.01, 5, u)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- projection
def test_projection(oracle):
    ns = NS.disk_holes(8000, seed=5)
    _, stencils = random_stencils(ns, 25, 10, 4, oracle)
    rng = np.random.default_rng(3)
    for st in stencils:
        K, B, xi, s = oracle.kkt(ns.pts, st, 5, 4, 1)
        n = 25
        Q = K[:n, n:]
        lq = B[n:, 0]
        exact = np.linalg.solve(K, B)[:n, 0]
        wt = exact * (1 + 0.05 * rng.normal(size=n)) + 0.3 * rng.normal(size=n)
        w = oracle.project_lap(ns.pts, st, 5, 4, wt)
        # constraints hold, idempotent, equal to the orthogonal projection
        assert np.abs(Q.T @ w - lq).max() <= 1e-12 * max(1, np.abs(Q.T * np.abs(w)).sum(1).max())
        w2 = oracle.project_lap(ns.pts, st, 5, 4, w)
        assert np.abs(w2 - w).max() <= 1e-12 * np.abs(w).max()
        wmin = np.linalg.lstsq(Q.T, lq, rcond=None)[0]
        Pn = np.eye(n) - Q @ np.linalg.pinv(Q)
        ref = Pn @ wt + wmin
        assert np.abs(w - ref).max() <= 1e-9 * np.abs(ref).max()
        # exact weights are a fixed point; residual check is ~0 there, > 0 off it
        we = oracle.project_lap(ns.pts, st, 5, 4, exact)
        assert np.abs(we - exact).max() <= 1e-9 * np.abs(exact).max()
        assert oracle.phi_residual_lap(ns.pts, st, 5, 4, exact) <= 1e-9
        assert oracle.phi_residual_lap(ns.pts, st, 5, 4, w) > 1e-4


def test_phi_residual_hand_worked(oracle):
    """rho on a stencil worked out by hand.  Four nodes at the corners of a
    square of side h, centre first; k = 3, m = 1 (l = 3, so n = l + 1): the
    residual r = l_phi - A w minus its least-squares fit by Q is r's component
    along the single null vector v = (1, -1, -1, 1) of Q^T, so
    ||r - Q lambda||_inf = |v.r| / 4.  With s = sqrt(2) h and a = 1/sqrt(2):
    xi = (0,0), (a,0), (0,a), (a,a); l_phi,j = k (k + d - 2) r_j^(k-2) = 9 r_j
    = (0, 9a, 9a, 9), so ||l_phi||_inf = 9; column j of A holds
    ||xi_i - xi_j||^3 (here h = 0.1)."""
    pts = np.array([[0.3, 0.2], [0.4, 0.2], [0.3, 0.3], [0.4, 0.3]])
    st = np.arange(4, dtype=np.int32)
    a = 1 / math.sqrt(2)
    vl = 0 - 9 * a - 9 * a + 9                         # v . l_phi
    cases = {
        "zero": (np.zeros(4), vl),
        # A e_0 = (0, a^3, a^3, 1): v . A e_0 = 1 - 2 a^3
        "centre": (np.array([1.0, 0, 0, 0]), vl - (1 - 2 * a ** 3)),
        # A e_1 = (a^3, 0, 1, a^3): v . A e_1 = 2 a^3 - 1
        "node1": (np.array([0, 1.0, 0, 0]), vl - (2 * a ** 3 - 1)),
        # A e_3 = (1, a^3, a^3, 0): v . A (2 e_0 - e_3) = 2 (1 - 2 a^3) - (1 - 2 a^3)
        "mixed": (np.array([2.0, 0, 0, -1.0]), vl - 2 * (1 - 2 * a ** 3) + (1 - 2 * a ** 3)),
    }
    for name, (w, vr) in cases.items():
        ref = abs(vr) / 4 / 9
        got = oracle.phi_residual_lap(pts * 1.0, st, 3, 1, w)
        assert abs(got - ref) <= 1e-14, (name, got, ref)
    # the scale of the node set does not matter (w is in scaled units)
    got = oracle.phi_residual_lap(pts * 7.0 + 1.0, st, 3, 1, np.zeros(4))
    assert abs(got - (math.sqrt(2) - 1) / 4) <= 1e-14


def test_phi_residual_equals_orthogonal_complement(oracle):
    """On disk stencils (n = 25, k = 5, m = 4) rho equals the sup norm of the
    part of l_phi - A w orthogonal to range(Q), taken with an SVD projector
    (numpy), over ||l_phi||_inf; for exact weights it is ~0, and it grows
    linearly when w moves off them inside null(Q^T)."""
    ns = NS.disk_holes(8000, seed=5)
    _, stencils = random_stencils(ns, 25, 6, 4, oracle)
    rng = np.random.default_rng(11)
    n = 25
    for st in stencils:
        K, B, xi, s = oracle.kkt(ns.pts, st, 5, 4, 1)
        A, Q, lphi = K[:n, :n], K[:n, n:], B[:n, 0]
        U, sv, _ = np.linalg.svd(Q, full_matrices=True)
        Z = U[:, Q.shape[1]:]                           # basis of null(Q^T)
        exact = np.linalg.solve(K, B)[:n, 0]
        for t in (1e-3, 1e-2, 1e-1):
            d = Z @ rng.normal(size=Z.shape[1])
            w = exact + t * d / np.abs(d).max() * np.abs(exact).max()
            r = lphi - A @ w
            ref = np.abs(Z @ (Z.T @ r)).max() / np.abs(lphi).max()
            got = oracle.phi_residual_lap(ns.pts, st, 5, 4, w)
            assert abs(got - ref) <= 1e-9 * max(ref, 1e-6), (t, got, ref)


# ------------------------------------------------------------------------ MLP
def test_mlp_gradient_finite_differences(oracle):
    n_in, H, L, n_out, B = 5, 7, 3, 4, 6
    npar = oracle.mlp_nparams(n_in, H, L, n_out)
    assert npar == H * n_in + H + 2 * (H * H + H) + n_out * H + n_out
    rng = np.random.default_rng(0)
    p = rng.normal(size=npar) * 0.5
    x = rng.normal(size=(B, n_in))
    t = rng.normal(size=(B, n_out))
    loss, g = oracle.mlp_grad(n_in, H, L, n_out, p, x, t)
    y, loss2 = oracle.mlp_forward(n_in, H, L, n_out, p, x, t)
    assert abs(loss - loss2) <= 1e-14 * abs(loss)
    assert abs(loss - ((y - t) ** 2).mean()) <= 1e-14 * loss
    eps = 1e-6
    for i in rng.choice(npar, size=40, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (oracle.mlp_forward(n_in, H, L, n_out, pp, x, t)[1]
              - oracle.mlp_forward(n_in, H, L, n_out, pm, x, t)[1]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-3), (i, fd, g[i])


def test_mlp_gelu_reduces_to_known_values(oracle):
    # one hidden unit with identity-like weights: y = gelu(x) exactly
    n_in, H, L, n_out = 1, 1, 1, 1
    p = np.array([1.0, 0.0, 1.0, 0.0])            # W1, b1, W2, b2
    x = np.array([[0.0], [3.0], [-3.0], [1.0]])
    y, _ = oracle.mlp_forward(n_in, H, L, n_out, p, x)
    c = math.sqrt(2 / math.pi)
    ref = [0.5 * v * (1 + math.tanh(c * (v + 0.044715 * v ** 3))) for v in x[:, 0]]
    assert np.allclose(y[:, 0], ref, rtol=1e-15, atol=0)
    assert y[0, 0] == 0.0 and abs(y[1, 0] - 3.0) < 0.01 and abs(y[2, 0]) < 0.01


def test_adam_first_step_is_sign_step(oracle):
    g = np.array([0.5, -2.0, 1e-3])
    p, m, v = oracle.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.1, eps=0.0)
    assert np.allclose(p, -0.1 * np.sign(g), rtol=1e-14)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
