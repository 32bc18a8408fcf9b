"""Pins of the oracle's implicit solve (Section 2.3.2: BiCGSTAB with an
incomplete-LU preconditioner; here ILU(0)); CPU only.

* ILU(0)'s defining property: (L U)_ij = A_ij on the pattern of A.
* Without fill-in (a tridiagonal matrix) ILU(0) is the exact LU.
* BiCGSTAB reaches the solution of a direct solver: unpreconditioned on a small
  well-conditioned nonsymmetric system, with ILU(0) on the disk Poisson system
  (interior Laplacian rows, Dirichlet outer circle, Neumann holes).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import nodesets as NS
from test_oracle_bc import disk_operator


def random_sparse(n, per_row, seed):
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        c = np.unique(np.concatenate([[i], rng.choice(n, per_row, replace=False)]))
        rows += [i] * len(c)
        cols += list(c)
    A = sp.csr_matrix((rng.normal(size=len(rows)), (rows, cols)), shape=(n, n))
    A = A + sp.diags(np.abs(A).sum(1).A1 + 1.0)        # diagonally dominant: no zero pivot
    A.sort_indices()
    return A


def test_ilu0_matches_a_on_its_pattern(oracle):
    A = random_sparse(300, 6, 1)
    f, diag = oracle.ilu0(A.indptr, A.indices, A.data)
    n = A.shape[0]
    L = np.eye(n)
    U = np.zeros((n, n))
    for i in range(n):
        for p in range(A.indptr[i], A.indptr[i + 1]):
            j = A.indices[p]
            if j < i:
                L[i, j] = f[p]
            else:
                U[i, j] = f[p]
    LU = L @ U
    Ad = A.toarray()
    mask = Ad != 0
    assert np.allclose(LU[mask], Ad[mask], rtol=1e-12, atol=1e-12 * np.abs(Ad).max())
    assert (diag == np.array([A.indptr[i] + np.searchsorted(A.indices[A.indptr[i]:A.indptr[i + 1]], i)
                              for i in range(n)])).all()


def test_ilu0_of_a_tridiagonal_matrix_is_exact(oracle):
    n = 200
    rng = np.random.default_rng(2)
    A = sp.diags([rng.uniform(-1, 1, n - 1), rng.uniform(3, 4, n), rng.uniform(-1, 1, n - 1)],
                 [-1, 0, 1], format="csr")
    A.sort_indices()
    f, diag = oracle.ilu0(A.indptr, A.indices, A.data)
    b = rng.normal(size=n)
    x = oracle.ilu0_solve(A.indptr, A.indices, f, diag, b)
    assert np.allclose(x, np.linalg.solve(A.toarray(), b), rtol=1e-12, atol=1e-12)


def test_bicgstab_unpreconditioned(oracle):
    A = random_sparse(150, 5, 3)
    b = np.random.default_rng(4).normal(size=150)
    x, ok, it, res = oracle.bicgstab(A.indptr, A.indices, A.data, b, precondition=False, tol=1e-13)
    assert ok and res <= 1e-13
    assert np.allclose(x, np.linalg.solve(A.toarray(), b), rtol=1e-10, atol=1e-12)


def test_bicgstab_ilu0_solves_the_disk_poisson_system(oracle):
    """The implicit Poisson problem of the benchmark (u = sin pi x sin pi y):
    ILU(0)-preconditioned BiCGSTAB agrees with a sparse direct solve."""
    ns, rp, col, vals, kind = disk_operator(oracle, N=5000, seed=7)
    A = sp.csr_matrix((vals, col, rp), shape=(ns.N, ns.N)).tolil()
    u = NS.sin_product(ns.pts)
    rhs = NS.sin_product_lap(ns.pts)
    g = NS.sin_product_grad(ns.pts)
    for i in np.nonzero(kind == 1)[0]:
        A.rows[i] = [int(i)]
        A.data[i] = [1.0]
        rhs[i] = u[i]
    nb = kind == 2
    rhs[nb] = (g[nb] * ns.normals[nb]).sum(1)
    A = A.tocsr()
    A.sort_indices()
    xd = spla.spsolve(A.tocsc(), rhs)
    x, ok, it, res = oracle.bicgstab(A.indptr, A.indices, A.data, rhs, tol=1e-12, maxit=3000)
    assert ok, (it, res)
    assert np.abs(x - xd).max() <= 1e-8 * np.abs(xd).max(), (it, np.abs(x - xd).max())
    assert np.abs(x - u).max() < 1e-3          # the discretisation error, not the solver's
