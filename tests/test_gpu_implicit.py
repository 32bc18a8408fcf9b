"""The implicit solve on the GPU (Section 2.3.2, the Poisson benchmark of
Section 5) against the oracle: assembly of the implicit matrix, ILU(0)
factors (bit for bit), the preconditioner's triangular solves, BiCGSTAB's
first iterates and its converged solution, and the edge cases (one unknown,
a zero pivot, an unsorted row, a start that already satisfies the
tolerance, no preconditioner)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import torch

import nodesets as NS
from test_oracle_bc import disk_operator

pytestmark = pytest.mark.gpu


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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host_assemble(rp, col, vals, kind):
    """Rows sorted by column, Dirichlet rows the identity on the same pattern."""
    col_s, val_s = col.copy(), vals.copy()
    for i in range(len(rp) - 1):
        a, b = rp[i], rp[i + 1]
        o = np.argsort(col[a:b], kind="stable")
        col_s[a:b] = col[a:b][o]
        val_s[a:b] = vals[a:b][o]
        if kind[i] == 1:
            val_s[a:b] = (col_s[a:b] == i).astype(np.float64)
    return col_s, val_s


def poisson_rhs(ns, kind):
    u = NS.sin_product(ns.pts)
    rhs = NS.sin_product_lap(ns.pts)
    g = NS.sin_product_grad(ns.pts)
    rhs[kind == 1] = u[kind == 1]
    nb = kind == 2
    rhs[nb] = (g[nb] * ns.normals[nb]).sum(1)
    return rhs, u


@pytest.fixture(scope="module")
def disk(oracle):
    ns, rp, col, vals, kind = disk_operator(oracle, N=20000, seed=7)
    return ns, rp, col, vals, kind


@pytest.fixture(scope="module")
def assembled(P, ctx, disk):
    ns, rp, col, vals, kind = disk
    rp_d, col_d, vals_d = dev(rp), dev(col), dev(vals)
    col_o = torch.empty_like(col_d)
    val_o = torch.empty_like(vals_d)
    ctx.implicit_assemble(rp_d, col_d, vals_d, dev(kind), col_o, val_o)
    torch.cuda.synchronize()
    return rp_d, col_o, val_o


def test_assembly_matches_host(disk, assembled):
    ns, rp, col, vals, kind = disk
    _, col_o, val_o = assembled
    col_s, val_s = host_assemble(rp, col, vals, kind)
    assert np.array_equal(col_o.cpu().numpy(), col_s)
    assert np.array_equal(val_o.cpu().numpy(), val_s)


def test_ilu0_factors_bitwise(P, ctx, oracle, disk, assembled):
    """Same operations in the same order with the same roundings as the
    oracle's row-by-row ILU(0): equal bit for bit."""
    ns, rp, col, vals, kind = disk
    rp_d, col_o, val_o = assembled
    f = torch.empty_like(val_o)
    diag = torch.empty(ns.N, dtype=torch.int64, device="cuda")
    ctx.ilu0(rp_d, col_o, val_o, f, diag)
    torch.cuda.synchronize()
    f_ref, d_ref = oracle.ilu0(rp, col_o.cpu().numpy(), val_o.cpu().numpy())
    assert np.array_equal(diag.cpu().numpy(), d_ref)
    got = f.cpu().numpy()
    assert np.array_equal(got, f_ref), np.abs(got - f_ref).max()
    # in place gives the same
    g = val_o.clone()
    ctx.ilu0(rp_d, col_o, g, g, diag)
    torch.cuda.synchronize()
    assert np.array_equal(g.cpu().numpy(), f_ref)


def test_ilu0_solve_matches_oracle(P, ctx, oracle, disk, assembled):
    ns, rp, col, vals, kind = disk
    rp_d, col_o, val_o = assembled
    f = torch.empty_like(val_o)
    diag = torch.empty(ns.N, dtype=torch.int64, device="cuda")
    ctx.ilu0(rp_d, col_o, val_o, f, diag)
    rng = np.random.default_rng(3)
    for trial in range(3):
        b = rng.normal(size=ns.N)
        x = torch.full((ns.N,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.ilu0_solve(rp_d, col_o, f, diag, dev(b), x)
        torch.cuda.synchronize()
        ref = oracle.ilu0_solve(rp, col_o.cpu().numpy(), f.cpu().numpy(), diag.cpu().numpy(), b)
        got = x.cpu().numpy()
        # the two substitutions sum each row in a different order: the
        # difference is rounding amplified by the factors' conditioning
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()


def test_bicgstab_first_iterates_match_oracle(P, ctx, oracle, disk, assembled):
    """After 1, 2 and 5 iterations the GPU iterate equals the oracle's to
    rounding (both start from x = 0 with the same ILU(0) factors)."""
    ns, rp, col, vals, kind = disk
    rp_d, col_o, val_o = assembled
    rhs, _ = poisson_rhs(ns, kind)
    f = torch.empty_like(val_o)
    diag = torch.empty(ns.N, dtype=torch.int64, device="cuda")
    ctx.ilu0(rp_d, col_o, val_o, f, diag)
    col_h, val_h = col_o.cpu().numpy(), val_o.cpu().numpy()
    for k in (1, 2, 5):
        x = torch.zeros(ns.N, dtype=torch.float64, device="cuda")
        rc, it, res = ctx.bicgstab(rp_d, col_o, val_o, dev(rhs), x, f, diag, tol=1e-30, maxit=k)
        assert rc == P.binding.MM_ENOCONV and it == k
        xo, ok, ito, reso = oracle.bicgstab(rp, col_h, val_h, rhs, tol=1e-30, maxit=k)
        assert ito == k
        got = x.cpu().numpy()
        assert np.abs(got - xo).max() <= 1e-8 * np.abs(xo).max(), (k, np.abs(got - xo).max())
        assert abs(res - reso) <= 1e-6 * reso, (k, res, reso)


def test_bicgstab_solves_disk_poisson(P, ctx, oracle, disk, assembled):
    """The converged GPU solution equals the oracle's and a sparse direct
    solve to the solver tolerance, and its error against the manufactured
    solution is the discretisation error."""
    ns, rp, col, vals, kind = disk
    rp_d, col_o, val_o = assembled
    rhs, u = poisson_rhs(ns, kind)
    f = torch.empty_like(val_o)
    diag = torch.empty(ns.N, dtype=torch.int64, device="cuda")
    ctx.ilu0(rp_d, col_o, val_o, f, diag)
    x = torch.zeros(ns.N, dtype=torch.float64, device="cuda")
    rc, it, res = ctx.bicgstab(rp_d, col_o, val_o, dev(rhs), x, f, diag, tol=1e-12, maxit=3000)
    assert rc == P.binding.MM_OK and res <= 1e-12, (rc, it, res)
    col_h, val_h = col_o.cpu().numpy(), val_o.cpu().numpy()
    xo, ok, ito, reso = oracle.bicgstab(rp, col_h, val_h, rhs, tol=1e-12, maxit=3000)
    assert ok
    A = sp.csr_matrix((val_h, col_h, rp), shape=(ns.N, ns.N))
    xd = spla.spsolve(A.tocsc(), rhs)
    got = x.cpu().numpy()
    assert np.abs(got - xd).max() <= 1e-8 * np.abs(xd).max()
    assert np.abs(got - xo).max() <= 1e-8 * np.abs(xd).max()
    assert abs(it - ito) <= max(5, 0.2 * ito), (it, ito)
    assert np.abs(got - u).max() < 1e-3


def test_bicgstab_unpreconditioned_and_trivial_cases(P, ctx, oracle):
    from test_oracle_krylov import random_sparse
    A = random_sparse(150, 5, 3)
    b = np.random.default_rng(4).normal(size=150)
    rp_d, col_d, val_d = dev(A.indptr.astype(np.int64)), dev(A.indices.astype(np.int32)), dev(A.data)
    x = torch.zeros(150, dtype=torch.float64, device="cuda")
    rc, it, res = ctx.bicgstab(rp_d, col_d, val_d, dev(b), x, tol=1e-13, maxit=500)
    assert rc == P.binding.MM_OK and res <= 1e-13
    assert np.allclose(x.cpu().numpy(), np.linalg.solve(A.toarray(), b), rtol=1e-10, atol=1e-12)
    # a start that already meets the tolerance: no iteration, x untouched
    xs = torch.from_numpy(np.linalg.solve(A.toarray(), b)).cuda()
    x0 = xs.clone()
    rc, it, res = ctx.bicgstab(rp_d, col_d, val_d, dev(b), xs, tol=1e-6, maxit=50)
    assert rc == P.binding.MM_OK and it == 0 and torch.equal(xs, x0)
    # one unknown: 4 x = 2, with and without ILU(0)
    rp1, c1, v1 = dev(np.array([0, 1], dtype=np.int64)), dev(np.array([0], dtype=np.int32)), dev(np.array([4.0]))
    f1, d1 = torch.empty(1, dtype=torch.float64, device="cuda"), torch.empty(1, dtype=torch.int64, device="cuda")
    ctx.ilu0(rp1, c1, v1, f1, d1)
    for fac in ((f1, d1), (None, None)):
        x1 = torch.zeros(1, dtype=torch.float64, device="cuda")
        rc, it, res = ctx.bicgstab(rp1, c1, v1, dev(np.array([2.0])), x1, *fac, tol=1e-14, maxit=5)
        assert rc == P.binding.MM_OK and x1.item() == 0.5


def test_ilu0_rejects_bad_matrices(P, ctx):
    # zero pivot: [[0, 1], [1, 1]]
    rp = dev(np.array([0, 2, 4], dtype=np.int64))
    col = dev(np.array([0, 1, 0, 1], dtype=np.int32))
    f = torch.empty(4, dtype=torch.float64, device="cuda")
    d = torch.empty(2, dtype=torch.int64, device="cuda")
    with pytest.raises(P.MMError, match="zero pivot"):
        ctx.ilu0(rp, col, dev(np.array([0.0, 1.0, 1.0, 1.0])), f, d)
    # unsorted row
    col_u = dev(np.array([1, 0, 0, 1], dtype=np.int32))
    with pytest.raises(P.MMError, match="not increasing"):
        ctx.ilu0(rp, col_u, dev(np.array([1.0, 2.0, 1.0, 1.0])), f, d)
    # assembly: a row without its own node
    col_n = dev(np.array([1, 0, 0, 0], dtype=np.int32))
    with pytest.raises(P.MMError):
        ctx.implicit_assemble(rp, col_n, dev(np.ones(4)), None, torch.empty_like(col_n),
                              torch.empty(4, dtype=torch.float64, device="cuda"))
    # the context is still usable afterwards
    ctx.ilu0(rp, col, dev(np.array([2.0, 1.0, 1.0, 3.0])), f, d)
    torch.cuda.synchronize()
    assert np.allclose(f.cpu().numpy(), [2.0, 1.0, 0.5, 2.5])
