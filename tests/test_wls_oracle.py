"""Pins of the weighted least squares (GWLS) oracle (oracle/wls.py) against
facts fixed by Section 2.2.1 and the mathematics; CPU only.

* n = l: W B is square and invertible, so the weights are those of polynomial
  interpolation whatever the weight function -- the closed-form stencils of
  tests/golden/closed_form_stencils.txt.
* The weights reproduce every basis monomial exactly (B^T w_s = (L b)(0)).
* They are the minimum of sum_j w_j^2 / omega_j^2 under those constraints,
  found here from an independent KKT solve (numpy.linalg.solve).
* A hand-derived closed form for a six-node stencil with the degree-1 basis
  pins the Gaussian weight omega = exp(-|x|^2 / sigma^2), W's placement and
  both scale choices.
* Shift invariance and the h^-q dilation law.
"""
import numpy as np
import pytest

import nodesets as NS
from test_oracle_pins import OPBIT, load_closed_forms, lop_monomial, exps_graded


@pytest.fixture(scope="module")
def W(oracle):
    from oracle import wls
    return wls


@pytest.mark.parametrize("case", load_closed_forms(), ids=lambda c: c["name"] + "_" + c["op"])
@pytest.mark.parametrize("sigma,scale", [(1.0, 1), (0.3, 0), (5.0, 1)])
def test_square_systems_give_the_interpolation_stencils(W, case, sigma, scale):
    h = 0.01
    x = np.array(case["nodes"], dtype=float) * h
    w, st, _, _ = W.stencil_weights(x, 2, OPBIT[case["op"]], sigma, scale)
    assert st == W.OK
    expect = np.array(case["w"]) / h ** case["q"]
    assert np.allclose(w[0], expect, rtol=0, atol=1e-9 * np.abs(expect).max())


@pytest.mark.parametrize("dim,m,n", [(2, 2, 9), (2, 4, 25), (3, 2, 20), (3, 3, 35)])
def test_weights_reproduce_the_basis(W, oracle, dim, m, n):
    """kNN stencils of the quasi-uniform node sets (the kernels' inputs)."""
    ns = NS.disk_holes(4000, seed=1) if dim == 2 else NS.ball(4000, seed=1)
    rng = np.random.default_rng(dim * 100 + m)
    q = rng.choice(ns.classes["interior"][1], 6, replace=False)
    idx, _ = oracle.knn(ns.pts, n, queries=q)
    ops = [("lap", 1), ("dx", 2), ("dy", 4)] + ([("dz", 8)] if dim == 3 else []) + [("dxy", 64)]
    bits = sum(b for _, b in ops)
    E = exps_graded(dim, m)
    for t in range(len(q)):
        x = ns.pts[idx[t]]
        for sigma, scale in ((1.0, W.SCALE_NEAREST), (0.7, W.SCALE_FARTHEST)):
            w, st, _, _ = W.stencil_weights(x, m, bits, sigma, scale)
            assert st == W.OK
            d = x - x[0]
            for r, (name, _) in enumerate(ops):
                for e in E:
                    terms = w[r] * np.prod(d ** e, axis=1)
                    ref = lop_monomial(e, name)
                    assert abs(terms.sum() - ref) <= 1e-10 * (np.abs(terms).sum() + 1.0), (name, tuple(e))


def node_set_stencil(oracle, dim, n, t):
    ns = NS.disk_holes(4000, seed=4) if dim == 2 else NS.ball(4000, seed=4)
    q = np.array([37 * t + 11])
    idx, _ = oracle.knn(ns.pts, n, queries=q)
    return ns.pts[idx[0]]


def test_weights_are_the_weighted_minimum_norm_solution(W, oracle):
    """min sum_j w_j^2 / omega_j^2 subject to B^T w = (L b)(0): the KKT system
    [diag(omega^-2) B; B^T 0] [w; -mu] = [0; l] solved directly."""
    for t, (dim, m, n) in enumerate(((2, 2, 12), (2, 3, 20), (3, 2, 18))):
        x = node_set_stencil(oracle, dim, n, t)
        for sigma, scale in ((1.0, W.SCALE_NEAREST), (2.0, W.SCALE_FARTHEST)):
            _, st, s, ws = W.stencil_weights(x, m, 1 | 2, sigma, scale)
            assert st == W.OK
            xi = (x - x[0]) / s
            om = np.exp(-(xi ** 2).sum(1) / sigma ** 2)
            E = exps_graded(dim, m)
            B = np.prod(xi[:, None, :] ** E[None], axis=2)
            l = B.shape[1]
            K = np.zeros((n + l, n + l))
            K[:n, :n] = np.diag(1.0 / om ** 2)
            K[:n, n:] = B
            K[n:, :n] = B.T
            for r, name in enumerate(("lap", "dx")):
                rhs = np.zeros(n + l)
                rhs[n:] = [lop_monomial(e, name) for e in E]
                sol = np.linalg.solve(K, rhs)
                assert np.allclose(ws[r], sol[:n], rtol=1e-9, atol=1e-9 * np.abs(sol[:n]).max())


def closed_form_six_nodes(h, sigma):
    """Scaled d/dx weights for xi = (0,0), (h,0), (-h,0), (0,h), (0,-h), (2h,0)
    with the basis 1, x, y and omega = exp(-|xi|^2 / sigma^2): w_j = omega_j^2
    (mu0 + mu1 x_j + mu2 y_j) with G mu = (0, 1, 0), G = sum_j omega_j^2 b_j b_j^T,
    worked out by hand: mu2 = 0 and a 2 x 2 system for mu0, mu1."""
    A2 = np.exp(-h * h / sigma ** 2) ** 2            # omega^2 of the four nodes at distance h
    C2 = np.exp(-4 * h * h / sigma ** 2) ** 2        # omega^2 of the node at 2h
    S0 = 1 + 4 * A2 + C2
    X1 = 2 * h * C2                                  # sum omega^2 x
    X2 = 2 * h * h * A2 + 4 * h * h * C2             # sum omega^2 x^2
    det = S0 * X2 - X1 * X1
    mu0, mu1 = -X1 / det, S0 / det
    return np.array([mu0, A2 * (mu0 + h * mu1), A2 * (mu0 - h * mu1), A2 * mu0, A2 * mu0,
                     C2 * (mu0 + 2 * h * mu1)])


@pytest.mark.parametrize("sigma", [1.0, 2.0, 0.5])
def test_gaussian_weight_closed_form(W, sigma):
    x = np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1], [2, 0]], dtype=float) * 0.03
    for scale, s in ((W.SCALE_NEAREST, 0.03), (W.SCALE_FARTHEST, 0.06)):
        w, st, s_got, ws = W.stencil_weights(x, 1, 2, sigma, scale)
        assert st == W.OK and abs(s_got - s) < 1e-15
        ref = closed_form_six_nodes(0.03 / s, sigma)
        assert np.allclose(ws[0], ref, rtol=1e-12, atol=1e-14)
        assert np.allclose(w[0], ref / s, rtol=1e-12, atol=1e-12)


def test_shift_and_dilation(W, oracle):
    x = node_set_stencil(oracle, 2, 15, 3)
    w0, _, _, _ = W.stencil_weights(x, 3, 1 | 2 | 32, 1.0, W.SCALE_NEAREST)
    w1, _, _, _ = W.stencil_weights(x + np.array([5.0, -3.0]), 3, 1 | 2 | 32, 1.0, W.SCALE_NEAREST)
    w2, _, _, _ = W.stencil_weights(x * 0.25, 3, 1 | 2 | 32, 1.0, W.SCALE_NEAREST)
    assert np.allclose(w0, w1, rtol=1e-9, atol=1e-9 * np.abs(w0).max())
    for r, q in enumerate((2, 1, 2)):
        assert np.allclose(w2[r], w0[r] / 0.25 ** q, rtol=1e-9, atol=1e-9 * np.abs(w2[r]).max())


def test_rank_deficiency_and_bad_rows(W):
    x = np.array([[0, 0], [1, 0], [2, 0], [3, 0], [4, 0], [5, 0], [6, 0]], dtype=float)   # collinear
    _, st, _, _ = W.stencil_weights(x, 2, 1, 1.0, W.SCALE_NEAREST)
    assert st == W.SINGULAR
    _, st, _, _ = W.stencil_weights(x[:4] + [[0, 0], [0, 1], [1, 1], [1, 3]], 2, 1, 1.0, W.SCALE_NEAREST)
    assert st == W.SINGULAR                                   # n = 4 < l = 6
    pts = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0], [0.5, 0.2]])
    rp = np.array([0, 5, 10])
    col = np.array([0, 1, 2, 3, 4, 0, 1, 2, 3, 4])            # row 1 does not start with itself
    vals, status = W.weights(pts, rp, col, 1, 2, 1.0, W.SCALE_NEAREST)
    assert status[0] == W.OK and status[1] == W.BADARG and not vals[:, 5:].any()


def test_matches_on_a_node_set(W, oracle):
    """CSR front end on a disk patch: rows agree with the single-stencil form."""
    ns = NS.disk_holes(3000, seed=2)
    q = np.arange(0, 40)
    idx, _ = oracle.knn(ns.pts, 9, queries=q)
    rp = np.zeros(ns.N + 1, dtype=np.int64)
    rp[1:41] = np.arange(1, 41) * 9
    rp[41:] = 360
    vals, status = W.weights(ns.pts, rp, idx.ravel(), 2, 1 | 2 | 4, 1.0, W.SCALE_NEAREST, rows=(0, 40))
    assert (status[:40] == W.OK).all()
    for i in (0, 17, 39):
        w, _, _, _ = W.stencil_weights(ns.pts[idx[i]], 2, 1 | 2 | 4, 1.0, W.SCALE_NEAREST)
        assert np.array_equal(vals[:, rp[i]:rp[i + 1]], w)
