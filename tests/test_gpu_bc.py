"""GPU parity of mm_diffuse_bc (Neumann update, eq. exp-end) and
mm_combine_operators (eq. gen-op) against the oracle, through the C ABI."""
import numpy as np
import pytest
import torch

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


def gpu_diffuse_bc(ctx, rp, col, vals, kind, g, dt, steps, u):
    ud = dev(u.copy())
    work = torch.empty_like(ud)
    ctx.diffuse_bc(dev(rp), dev(col), dev(vals), dev(kind), None if g is None else dev(g), dt, steps, ud, work)
    torch.cuda.synchronize()
    return ud.cpu().numpy()


def test_neumann_update_by_hand(P, ctx):
    rp = np.array([0, 3, 6, 7, 9])
    col = np.array([0, 1, 2, 1, 0, 3, 2, 3, 2], dtype=np.int32)
    vals = np.array([-2.0, 1.0, 1.0, 4.0, -1.0, -3.0, 1.0, -1.0, 1.0])
    kind = np.array([0, 2, 1, 0], dtype=np.uint8)
    g = np.array([0.0, 0.5, 0.0, 0.0])
    two = gpu_diffuse_bc(ctx, rp, col, vals, kind, g, 0.1, 2, np.array([1.0, 2.0, 3.0, 4.0]))
    assert np.allclose(two, [1.3 + 0.1 * (-2.6 + 3.375 + 3.0), (0.5 + 1.3 + 11.7) / 4, 3.0,
                             3.9 + 0.1 * (-3.9 + 3.0)], rtol=0, atol=1e-14)


def test_diffuse_bc_matches_oracle(P, ctx, oracle):
    """Disk with holes (Laplacian inside, Dirichlet outer circle, Neumann
    holes): one step from a rough field against the oracle, per node within
    rounding of the row's terms; and without Neumann rows, 30 steps equal
    mm_diffuse bit for bit."""
    ns, rp, col, vals, kind = disk_operator(oracle)
    rng = np.random.default_rng(2)
    u = rng.normal(size=ns.N)
    g = rng.normal(size=ns.N)
    got = gpu_diffuse_bc(ctx, rp, col, vals, kind, g, 1e-6, 1, u)
    ref = oracle.diffuse_bc(rp, col, vals, kind, g, 1e-6, 1, u)
    absrow = oracle.spmv(rp, col, np.abs(vals), np.abs(u))
    w1 = np.abs(vals[rp[:-1]])
    bound = 64 * np.finfo(float).eps * np.where(kind == 2, (absrow + np.abs(g)) / w1, 1e-6 * absrow + np.abs(u))
    assert (np.abs(got - ref) <= bound + 1e-300).all(), np.abs(got - ref).max()
    held = np.where(kind == 2, 1, kind).astype(np.uint8)
    a = gpu_diffuse_bc(ctx, rp, col, vals, held, None, 1e-7, 30, u)
    ud, work = dev(u.copy()), torch.empty(ns.N, dtype=torch.float64, device="cuda")
    ctx.diffuse(dev(rp), dev(col), dev(vals), dev(held), 1e-7, 30, ud, work)
    torch.cuda.synchronize()
    assert np.array_equal(a, ud.cpu().numpy())


def test_combine_operators_matches_definition(P, ctx, oracle):
    rng = np.random.default_rng(4)
    N, n = 5000, 25
    rp = np.arange(N + 1, dtype=np.int64) * n
    col = rng.integers(0, N, N * n).astype(np.int32)
    terms = [rng.normal(size=N * n) for _ in range(7)]
    coefs = [rng.normal(size=N) if t % 3 else None for t in range(7)]
    b, e = 123, 4567
    out = torch.full((N * n,), 9.0, dtype=torch.float64, device="cuda")
    ctx.combine_operators(dev(rp), dev(col), [dev(t) for t in terms],
                          [None if a is None else dev(a) for a in coefs], out, row_begin=b, row_end=e)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = oracle.combine_operators(rp, terms, coefs, rows=(b, e))
    sl = slice(rp[b], rp[e])
    scale = sum(np.abs(t) * (1.0 if a is None else np.abs(a[np.repeat(np.arange(N), n)]))
                for t, a in zip(terms, coefs))
    assert (np.abs(got[sl] - ref[sl]) <= 16 * np.finfo(float).eps * scale[sl]).all()
    assert (got[:rp[b]] == 9.0).all() and (got[rp[e]:] == 9.0).all()
    # the result may overwrite one of the terms; all coefficients 1
    t0 = dev(terms[0])
    ctx.combine_operators(dev(rp), dev(col), [t0, dev(terms[1])], None, t0)
    torch.cuda.synchronize()
    assert np.allclose(t0.cpu().numpy(), terms[0] + terms[1], rtol=1e-15, atol=1e-15)
    with pytest.raises(P.MMError):
        ctx.combine_operators(dev(rp), dev(col), [], None, out)
