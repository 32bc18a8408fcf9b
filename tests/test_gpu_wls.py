"""GPU parity of the GWLS weights (mm_wls_weights, Section 2.2.1) against the
numpy oracle (oracle/wls.py, SVD pseudoinverse), through the C ABI.

Bar: per node and operator, ||w_gpu - w_ref||_inf / ||w_ref||_inf below
100 kappa(W B) u64 (two backward-stable FP64 solutions of the same least
squares problem differ by about kappa u), and the GPU weights reproduce the
basis to 1e-10 relative.  Statuses (singular, bad rows) match the oracle.
"""
import numpy as np
import pytest
import torch

import nodesets as NS
from _helpers import op_names, rel_err_rows

pytestmark = pytest.mark.gpu
U64 = np.finfo(float).eps / 2


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1912_13282_gb300 import _build
    _build.build()
    import paper_1912_13282_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def Wo(oracle):
    from oracle import wls
    return wls


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def knn_csr(oracle, ns, spec):
    """Oracle kNN stencils for the classes of a node set: (rp, col, classes)."""
    sizes = np.zeros(ns.N, dtype=np.int64)
    blocks = {}
    for cname, n, *_ in spec:
        b, e = (0, ns.N) if cname == "all" else ns.classes[cname]
        idx, _ = oracle.knn(ns.pts, n, queries=np.arange(b, e), nthreads=8)
        blocks[b] = idx
        sizes[b:e] = n
    rp = np.zeros(ns.N + 1, dtype=np.int64)
    np.cumsum(sizes, out=rp[1:])
    col = np.zeros(rp[-1], dtype=np.int32)
    for b, idx in blocks.items():
        col[rp[b]:rp[b] + idx.size] = idx.ravel()
    return rp, col


def run_gpu(ctx, ns, rp, col, b, e, n_max, m, ops, sigma, scale):
    vals = [torch.zeros(len(col), dtype=torch.float64, device="cuda") for _ in op_names(ops)]
    st = torch.full((ns.N,), -1, dtype=torch.int32, device="cuda")
    ctx.wls_weights(ops, m, sigma, scale, dev(ns.pts), dev(rp), dev(col), vals, row_begin=b, row_end=e,
                    n_max=n_max, normals=dev(ns.normals), status=st)
    torch.cuda.synchronize()
    return [v.cpu().numpy() for v in vals], st.cpu().numpy()


CASES = {
    # the paper's example setup: 9 closest nodes, degree 2, Gaussian sigma = 1, closest-node scale
    "square_paper": (lambda: NS.square(0.02), [("all", 9, 2, 1 | 2 | 4, 1.0, 1)]),
    "disk": (lambda: NS.disk_holes(20000, seed=5),
             [("interior", 25, 4, 1 | 2 | 4 | 32 | 64, 1.0, 1), ("boundary", 30, 2, 16, 0.7, 0)]),
    "disk_all6": (lambda: NS.disk_holes(8000, seed=6), [("interior", 16, 3, 1 | 2 | 4 | 32 | 64 | 128, 1.5, 1)]),
    # small systems, one stencil per thread
    "disk_n12": (lambda: NS.disk_holes(10000, seed=9),
                 [("interior", 12, 2, 1 | 2 | 4 | 32 | 64, 1.0, 1), ("boundary", 12, 2, 16, 1.2, 0)]),
    "ball_n10": (lambda: NS.ball(8000, seed=9), [("interior", 10, 1, 2 | 4 | 8, 1.0, 1)]),
    "ball": (lambda: NS.ball(15000, seed=6),
             [("interior", 35, 2, 1 | 2 | 4 | 8 | 1024, 0.8, 0), ("refined", 60, 3, 1 | 8, 1.0, 1),
              ("boundary", 45, 2, 16, 1.0, 0)]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_wls_matches_oracle(P, ctx, oracle, Wo, name):
    make, spec = CASES[name]
    ns = make()
    rp, col = knn_csr(oracle, ns, spec)
    rng = np.random.default_rng(0)
    for cname, n, m, ops, sigma, scale in spec:
        b, e = (0, ns.N) if cname == "all" else ns.classes[cname]
        got, st = run_gpu(ctx, ns, rp, col, b, e, n, m, ops, sigma, scale)
        assert (st[b:e] == P.binding.ST_OK).all(), np.unique(st[b:e], return_counts=True)
        rows = np.arange(b, e) if e - b <= 1500 else np.unique(np.concatenate(
            [rng.choice(np.arange(b, e), 1500, replace=False), [b, e - 1]]))
        names = op_names(ops)
        for i in rows:
            x = ns.pts[col[rp[i]:rp[i + 1]]]
            w_ref, st_ref, s, _ = Wo.stencil_weights(x, m, ops, sigma, scale, ns.normals[i])
            assert st_ref == Wo.OK
            xi = (x - x[0]) / s
            om = np.exp(-(xi ** 2).sum(1) / sigma ** 2)
            kap = np.linalg.cond(om[:, None] * Wo.basis_matrix(xi, m))
            for r, nm in enumerate(names):
                err = rel_err_rows(got[r], np.concatenate([np.zeros(rp[i]), w_ref[r]]), rp, [i])[0]
                assert err <= 100 * kap * U64 + 1e-14, (name, cname, nm, int(i), err, kap)


def test_wls_reproduces_the_basis(P, ctx, oracle, Wo):
    """The GPU weights satisfy B^T w_s = (L b)(0) (consistency of order m)."""
    ns = NS.disk_holes(6000, seed=8)
    spec = [("interior", 25, 4, 1 | 2 | 64, 1.0, 1)]
    rp, col = knn_csr(oracle, ns, spec)
    b, e = ns.classes["interior"]
    got, st = run_gpu(ctx, ns, rp, col, b, e, 25, 4, 1 | 2 | 64, 1.0, 1)
    assert (st[b:e] == 0).all()
    Lb = None
    for i in range(b, b + 300):
        x = ns.pts[col[rp[i]:rp[i + 1]]]
        d = x - x[0]
        s = np.sqrt((d ** 2).sum(1))[1:].min()
        B = Wo.basis_matrix(d / s, 4)
        Lb = Wo.rhs(2, 4, 1 | 2 | 64)
        for r, q in enumerate((2, 1, 2)):
            ws = got[r][rp[i]:rp[i + 1]] * s ** q
            terms = ws[:, None] * B
            res = np.abs(terms.sum(0) - Lb[r]) / np.maximum(1.0, np.abs(terms).sum(0))
            assert res.max() <= 1e-10, (int(i), r, res.max())


@pytest.mark.parametrize("n_max", [8, 40])
def test_wls_statuses_and_errors(P, ctx, Wo, n_max):
    """n < l and rank-deficient (collinear) rows -> SINGULAR, zero weights;
    centre not first or a lone node with the closest-node scale -> BADARG;
    argument errors are reported before anything runs.  n_max = 8 runs one
    stencil per thread, n_max = 40 one per warp (two rows per lane)."""
    g = np.arange(6.0)
    pts = np.concatenate([np.stack([g, np.zeros(6)], 1),                    # 0..5 collinear
                          np.array([[0.0, 1.0], [1.0, 1.0], [2.0, 1.5], [0.5, 2.0], [3.0, 3.0]])])
    rows = [[0, 1, 2, 3, 4, 5],                  # collinear: singular for m = 2
            [1, 0, 2, 6, 7],                     # n = 5 < l = 6: singular
            [2, 3, 1, 8, 7, 6, 9, 0],
            [3, 4, 5, 1, 2, 0],                  # collinear
            [4, 10, 8, 7, 3, 5, 2, 9],
            [5, 0, 1, 2, 3, 4],                  # collinear
            [6, 7, 8, 9, 10, 0, 1],
            [8, 1, 2, 6, 9, 10, 0],              # row 7 does not start with node 7: bad row
            [8, 0, 1, 2, 6, 7, 9, 10],
            [9],                                 # a lone node has no closest other node: bad row
            [10, 9, 8, 7, 6, 2, 1, 0]]
    sizes = [len(r) for r in rows]
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(sizes, out=rp[1:])
    col = np.concatenate(rows).astype(np.int32)
    vals = [torch.full((len(col),), 7.0, dtype=torch.float64, device="cuda")]
    st = torch.full((len(rows),), -1, dtype=torch.int32, device="cuda")
    ctx.wls_weights(1, 2, 3.0, 1, dev(pts), dev(rp), dev(col), vals, n_max=n_max, status=st)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    w = vals[0].cpu().numpy()
    vals_ref, st_ref = Wo.weights(pts, rp, col, 2, 1, 3.0, Wo.SCALE_NEAREST)
    assert list(st) == list(st_ref), (list(st), list(st_ref))
    for i in range(len(rows)):
        seg = slice(rp[i], rp[i + 1])
        if st[i] != 0:
            assert not w[seg].any()
        else:
            assert np.allclose(w[seg], vals_ref[0][seg], rtol=1e-9, atol=1e-9 * np.abs(vals_ref[0][seg]).max())
    with pytest.raises(P.MMError):
        ctx.wls_weights(1, 2, 0.0, 1, dev(pts), dev(rp), dev(col), vals, n_max=8)
    with pytest.raises(P.MMError):
        ctx.wls_weights(1, 2, 1.0, 2, dev(pts), dev(rp), dev(col), vals, n_max=8)
    with pytest.raises(P.MMError):
        ctx.wls_weights(1, 2, 1.0, 1, dev(pts), dev(rp), dev(col), vals, n_max=65)
