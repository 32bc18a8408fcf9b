"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

kNN rows must be identical (integer work); weights must match per node and
operator within 1e-10 (FP64 path; larger only where the oracle's own
conditioning bound 20 kappa_1 u64 exceeds it) and 1e-7 (FP32 + FP64
refinement), with monomials reproduced to 1e-12 in scaled units; operator
application within the rounding bound of the sum.
"""
import numpy as np
import pytest
import torch

import nodesets as NS
from _helpers import monomial_residual, op_names, rel_err_rows

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


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


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gpu_knn(ctx, P, pts_d, ranges, method):
    outs = []
    spec = []
    for qb, qe, n in ranges:
        o = torch.empty((qe - qb, n), dtype=torch.int32, device="cuda")
        outs.append(o)
        spec.append((qb, qe, n, o))
    st = torch.full((pts_d.shape[0],), -7, dtype=torch.int32, device="cuda")
    ctx.knn_stencils(pts_d, spec, method=method, status=st)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], st.cpu().numpy()


def csr_from_blocks(blocks):
    col = np.concatenate([b.ravel() for b in blocks]).astype(np.int32)
    sizes = np.concatenate([np.full(b.shape[0], b.shape[1]) for b in blocks])
    rp = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=rp[1:])
    return rp, col


# ----------------------------------------------------------------------- kNN
KNN_CASES = [
    ("square", lambda: NS.square(0.02), [("all", 12)]),
    ("disk", lambda: NS.disk_holes(30000, seed=1), [("interior", 25), ("boundary", 30)]),
    ("ball", lambda: NS.ball(30000, seed=2), [("interior", 35), ("refined", 60), ("boundary", 45)]),
    ("patches", lambda: NS.patches(400, seed=3), [("centre", 25)]),
]


@pytest.mark.parametrize("case", KNN_CASES, ids=[c[0] for c in KNN_CASES])
@pytest.mark.parametrize("method", ["grid", "brute"])
def test_knn_matches_oracle(P, ctx, oracle, case, method):
    name, make, classes = case
    ns = make()
    pts_d = dev(ns.pts)
    ranges = []
    for cname, n in classes:
        b, e = (0, ns.N) if cname == "all" else ns.classes[cname]
        ranges.append((b, e, n))
    m = P.KNN_GRID if method == "grid" else P.KNN_BRUTE
    got, st = gpu_knn(ctx, P, pts_d, ranges, m)
    for (b, e, n), g in zip(ranges, got):
        ref, rst = oracle.knn(ns.pts, n, queries=np.arange(b, e), nthreads=8)
        assert np.array_equal(g, ref), f"{name} rows differ: {np.argwhere(g != ref)[:5]}"
        assert (st[b:e] == 0).all() and (rst == 0).all()


def test_knn_ragged_and_edge_sizes(P, ctx, oracle):
    rng = np.random.default_rng(4)
    pts = rng.uniform(size=(1237, 2))
    pts_d = dev(pts)
    for method in (P.KNN_GRID, P.KNN_BRUTE):
        # the top list holds n - 1 entries: n = 33 is the largest one-slot
        # list, n = 34 the smallest two-slot one, n = 64 the largest allowed
        ranges = [(7, 1000, 1), (1000, 1237, 64), (3, 5, 33), (20, 400, 34), (400, 900, 64), (900, 1100, 33)]
        got, _ = gpu_knn(ctx, P, pts_d, ranges, method)
        for (b, e, n), g in zip(ranges, got):
            ref, _ = oracle.knn(pts, n, queries=np.arange(b, e))
            assert np.array_equal(g, ref)
    tiny = rng.uniform(size=(40, 3))
    got, st = gpu_knn(ctx, P, dev(tiny), [(0, 40, 40)], P.KNN_GRID)
    ref, _ = oracle.knn(tiny, 40)
    assert np.array_equal(got[0], ref) and (st == 0).all()


def test_knn_ties_and_duplicates(P, ctx, oracle):
    g = np.arange(30.0)
    X, Y = np.meshgrid(g, g, indexing="ij")
    grid = np.stack([X.ravel(), Y.ravel()], 1) * 0.1       # exact ties everywhere
    for method in (P.KNN_GRID, P.KNN_BRUTE):
        got, _ = gpu_knn(ctx, P, dev(grid), [(0, len(grid), 21)], method)
        ref, _ = oracle.knn(grid, 21)
        assert np.array_equal(got[0], ref)
    dup = np.concatenate([grid[:200], grid[10:11]])
    got, st = gpu_knn(ctx, P, dev(dup), [(0, len(dup), 9)], P.KNN_GRID)
    assert st[10] == P.binding.ST_DUPLICATE and st[200] == P.binding.ST_DUPLICATE
    assert (np.delete(st, [10, 200]) == 0).all()


# ------------------------------------------------------------------- weights
def oracle_rows(oracle, pts, normals, rp, col, rows, k, m, ops):
    """Oracle weights for arbitrary rows of a CSR stencil pattern: returns a
    dict row -> [R, n] array."""
    rows = np.asarray(rows)
    st_list = [col[rp[i]:rp[i + 1]] for i in rows]
    centres = rows
    others = np.setdiff1d(np.unique(np.concatenate(st_list)), centres)
    order = np.concatenate([centres, others])
    remap = np.full(pts.shape[0], -1, dtype=np.int64)
    remap[order] = np.arange(len(order))
    Pl = pts[order]
    Nl = None if normals is None else normals[order]
    lcol = np.concatenate([remap[s] for s in st_list]).astype(np.int32)
    sizes = np.array([len(s) for s in st_list])
    lrp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(sizes, out=lrp[1:])
    vals, status, _ = oracle.weights(Pl, lrp, lcol, k, m, ops, normals=Nl, rows=(0, len(rows)),
                                     nthreads=8)
    assert (status == 0).all()
    return {int(i): vals[:, lrp[t]:lrp[t + 1]] for t, i in enumerate(rows)}


def run_gpu_weights(ctx, P, ns, rp, col, cls, precision):
    """cls: list of (row_begin, row_end, n_max, k, m, ops).  One value array
    per operator name across classes."""
    pts_d, nrm_d = dev(ns.pts), dev(ns.normals)
    rp_d, col_d = dev(rp), dev(col)
    names = sorted({nm for *_, ops in cls for nm in op_names(ops)})
    vals = {nm: torch.zeros(len(col), dtype=torch.float64, device="cuda") for nm in names}
    status = torch.full((len(rp) - 1,), -1, dtype=torch.int32, device="cuda")
    for b, e, n_max, k, m, ops in cls:
        ctx.rbffd_weights(ops, k, m, pts_d, rp_d, col_d, [vals[nm] for nm in op_names(ops)],
                          row_begin=b, row_end=e, n_max=n_max, precision=precision,
                          normals=nrm_d, status=status)
    torch.cuda.synchronize()
    return {nm: v.cpu().numpy() for nm, v in vals.items()}, status.cpu().numpy()


def weight_case(name):
    if name == "square":
        ns = NS.square(0.01)
        spec = [("all", 12, 3, 2, 1 | 2 | 4)]
    elif name == "square_d2":
        # all 2D operators (6 columns: two launches of at most 5), r^3 and r^5
        ns = NS.square(0.02)
        spec = [("all", 12, 3, 2, 1 | 2 | 4 | 32 | 64 | 128)]
    elif name == "disk_d2":
        ns = NS.disk_holes(20000, seed=5)
        spec = [("interior", 25, 5, 4, 32 | 64 | 128), ("boundary", 30, 5, 4, 16 | 32 | 128)]
    elif name == "ball_d2":
        ns = NS.ball(15000, seed=6)
        spec = [("interior", 35, 3, 2, 32 | 64 | 128 | 256 | 512 | 1024), ("refined", 60, 3, 3, 1 | 256 | 1024),
                ("boundary", 45, 3, 2, 16 | 32)]
    elif name == "disk":
        ns = NS.disk_holes(20000, seed=5)
        spec = [("interior", 25, 5, 4, 1 | 2 | 4), ("boundary", 30, 5, 4, 16)]
    elif name.startswith("disk_r"):
        # every operator count R = 1..5 of the solvers (each R is its own
        # kernel instance): 25-node interior rows (M = 40, register inverse)
        # and 30-node boundary rows (M = 45)
        ops = {"disk_r1": 1, "disk_r2": 2 | 4, "disk_r4": 1 | 2 | 4 | 32, "disk_r5": 1 | 2 | 4 | 32 | 128}[name]
        ns = NS.disk_holes(20000, seed=8)
        spec = [("interior", 25, 5, 4, ops), ("boundary", 30, 5, 4, ops if name != "disk_r1" else 16)]
    else:
        ns = NS.ball(15000, seed=6)
        spec = [("interior", 35, 3, 2, 1 | 2 | 4 | 8), ("refined", 60, 3, 3, 1 | 2 | 4 | 8),
                ("boundary", 45, 3, 2, 16)]
    return ns, spec


@pytest.fixture(scope="module")
def weight_inputs(P, ctx):
    cache = {}

    def get(name):
        if name not in cache:
            ns, spec = weight_case(name)
            pts_d = dev(ns.pts)
            ranges = []
            for cname, n, *_ in spec:
                b, e = (0, ns.N) if cname == "all" else ns.classes[cname]
                ranges.append((b, e, n))
            blocks, _ = gpu_knn(ctx, P, pts_d, ranges, P.KNN_GRID)
            rp, col = csr_from_blocks(blocks)
            cls = [(b, e, n, k, m, ops) for (b, e, n), (_, _, k, m, ops) in zip(ranges, spec)]
            cache[name] = (ns, rp, col, cls)
        return cache[name]
    return get


@pytest.mark.parametrize("name", ["square", "disk", "ball", "square_d2", "disk_d2", "ball_d2", "disk_r1",
                                  "disk_r2", "disk_r4", "disk_r5"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_ir", "fp32_ir_wide64"])
def test_weights_match_oracle(P, ctx, oracle, weight_inputs, name, precision):
    """fp32_ir refines with double-FP32 residuals (the default), fp32_ir_wide64
    with native FP64 residuals; both meet the same bar."""
    ns, rp, col, cls = weight_inputs(name)
    prec = P.FP64 if precision == "fp64" else P.FP32_IR
    ctx.set_option(P.binding.OPT_WIDE, P.binding.WIDE_FP64 if precision.endswith("wide64") else P.binding.WIDE_FF)
    try:
        got, status = run_gpu_weights(ctx, P, ns, rp, col, cls, prec)
    finally:
        ctx.set_option(P.binding.OPT_WIDE, P.binding.WIDE_FF)
    ok_codes = {0} if precision == "fp64" else {0, P.binding.ST_FALLBACK}
    assert set(np.unique(status)) <= ok_codes, np.unique(status, return_counts=True)
    rng = np.random.default_rng(0)
    for b, e, n_max, k, m, ops in cls:
        # every row of small classes, a sample of large ones (plus both ends)
        rows = np.arange(b, e) if e - b <= 4000 else np.unique(np.concatenate(
            [rng.choice(np.arange(b, e), 4000, replace=False), [b, e - 1]]))
        ref = oracle_rows(oracle, ns.pts, ns.normals, rp, col, rows, k, m, ops)
        for oi, nm in enumerate(op_names(ops)):
            w_ref = np.zeros_like(got[nm])
            for i in rows:
                w_ref[rp[i]:rp[i + 1]] = ref[int(i)][oi]
            err = rel_err_rows(got[nm], w_ref, rp, rows)
            if precision == "fp64":
                bad = rows[err > 1e-10]
                for i in bad:      # only conditioning may explain a larger difference
                    kap = oracle.kkt_cond1(ns.pts, col[rp[i]:rp[i + 1]], k, m)
                    e_i = err[np.searchsorted(rows, i)]
                    assert e_i <= 20 * kap * U64, (name, nm, int(i), e_i, kap)
            else:
                assert err.max() <= 1e-7, (name, nm, err.max())
            mono = monomial_residual(ns.pts, ns.normals, rp, col, got[nm], nm, m, rows[:800])
            assert mono <= 1e-12, (name, nm, mono)


def test_mixed_fallback_path_is_exercised(P, ctx, oracle, weight_inputs):
    """Forcing every stencil through the condition-estimate gate must route
    them all to the FP64 solve and still match the oracle."""
    ns, rp, col, cls = weight_inputs("disk")
    c2 = P.Context(0)
    c2.set_option(P.binding.OPT_KAPPA_MAX, 1e-12)
    got, status = run_gpu_weights(c2, P, ns, rp, col, cls, P.FP32_IR)
    c2.close()
    assert (status == P.binding.ST_FALLBACK).all()
    ref64, _ = run_gpu_weights(ctx, P, ns, rp, col, cls, P.FP64)
    for nm in got:
        assert np.array_equal(got[nm], ref64[nm])


@pytest.mark.parametrize("name", ["disk", "ball", "disk_d2"])
def test_register_and_shared_inverse_agree_bitwise(P, ctx, weight_inputs, name):
    """Systems of 33..48 unknowns invert with each lane's rows in registers
    (disk interior M = 40, disk boundary and ball interior M = 45); the
    shared-memory form performs the same operations in the same order, so
    weights and statuses are identical."""
    ns, rp, col, cls = weight_inputs(name)
    got, st = run_gpu_weights(ctx, P, ns, rp, col, cls, P.FP32_IR)
    c2 = P.Context(0)
    c2.set_option(P.binding.OPT_GJ, P.binding.GJ_SHARED)
    ref, st2 = run_gpu_weights(c2, P, ns, rp, col, cls, P.FP32_IR)
    c2.close()
    assert np.array_equal(st, st2)
    for nm in got:
        assert np.array_equal(got[nm], ref[nm]), nm


def test_register_inverse_ragged_stencils(P, ctx, oracle, weight_inputs):
    """Rows of 20..25 nodes in a class of n_max = 25 (M = 35..40 in a
    40-column register frame: the inverse lands 0..5 columns from the left
    edge) and a few rows of odd M: identical to the shared-memory form and
    within 1e-7 of the oracle."""
    ns, rp, col, cls = weight_inputs("disk")
    b, e = ns.classes["interior"]
    rows = np.arange(b, b + 6000)
    n_i = 20 + (rows % 6)
    sizes = np.zeros(ns.N, dtype=np.int64)          # rows outside the range stay empty
    sizes[rows] = n_i
    rp2 = np.zeros(ns.N + 1, dtype=np.int64)
    np.cumsum(sizes, out=rp2[1:])
    col2 = np.concatenate([col[rp[i]:rp[i] + n] for i, n in zip(rows, n_i)]).astype(np.int32)
    pts_d, rp_d, col_d = dev(ns.pts), dev(rp2), dev(col2)
    out = []
    for form in (P.binding.GJ_AUTO, P.binding.GJ_SHARED):
        c = P.Context(0)
        c.set_option(P.binding.OPT_GJ, form)
        vals = [torch.zeros(len(col2), dtype=torch.float64, device="cuda") for _ in range(3)]
        st = torch.full((ns.N,), -1, dtype=torch.int32, device="cuda")
        c.rbffd_weights(1 | 2 | 4, 5, 4, pts_d, rp_d, col_d, vals, row_begin=int(rows[0]),
                        row_end=int(rows[-1]) + 1, n_max=25, precision=P.FP32_IR, status=st)
        torch.cuda.synchronize()
        out.append(([v.cpu().numpy() for v in vals], st.cpu().numpy()[rows]))
        c.close()
    (w_reg, st_reg), (w_sh, st_sh) = out
    assert np.array_equal(st_reg, st_sh) and set(np.unique(st_reg)) <= {0, P.binding.ST_FALLBACK}
    for a, r in zip(w_reg, w_sh):
        assert np.array_equal(a, r)
    sample = rows[::7]
    ref = oracle_rows(oracle, ns.pts, ns.normals, rp2, col2, sample, 5, 4, 1 | 2 | 4)
    for oi in range(3):
        w_ref = np.zeros_like(w_reg[oi])
        for i in sample:
            w_ref[rp2[i]:rp2[i + 1]] = ref[int(i)][oi]
        err = rel_err_rows(w_reg[oi], w_ref, rp2, sample)
        assert err.max() <= 1e-7, (oi, err.max())


def test_condition_gate_agrees_with_oracle_kappa(P, ctx, oracle, weight_inputs):
    """The mixed solver's condition number (||K||_1 times the exact norm of
    its FP32 inverse) matches the oracle's explicit-inverse kappa_1: with the
    gate threshold at the median kappa_1 of a sample, the rows clearly above it
    go to the FP64 solve and the rows clearly below it do not."""
    ns, rp, col, cls = weight_inputs("disk")
    b, e, n_max, k, m, ops = cls[0]                      # interior class
    rng = np.random.default_rng(3)
    rows = np.sort(rng.choice(np.arange(b, e), 300, replace=False))
    kap = np.array([oracle.kkt_cond1(ns.pts, col[rp[i]:rp[i + 1]], k, m) for i in rows])
    med = float(np.median(kap))
    c2 = P.Context(0)
    c2.set_option(P.binding.OPT_KAPPA_MAX, med * 2.0 ** -24)
    got, status = run_gpu_weights(c2, P, ns, rp, col, [cls[0]], P.FP32_IR)
    c2.close()
    st = status[rows]
    hi, lo = kap > 1.1 * med, kap < med / 1.1
    assert hi.sum() >= 20 and lo.sum() >= 20, (hi.sum(), lo.sum())
    assert (st[hi] == P.binding.ST_FALLBACK).all(), kap[hi][st[hi] != P.binding.ST_FALLBACK]
    assert (st[lo] == P.binding.ST_OK).all(), kap[lo][st[lo] != P.binding.ST_OK]


def test_bad_rows_get_status_and_zero_weights(P, ctx):
    rng = np.random.default_rng(7)
    pts = rng.uniform(size=(64, 2))
    pts[40:52] = np.stack([np.linspace(0, 1, 12), np.full(12, 0.5)], 1)   # collinear
    n = 12
    col = np.stack([np.concatenate([[i], rng.choice(np.delete(np.arange(64), i), n - 1,
                                                     replace=False)]) for i in range(64)])
    col[3, 5] = 999                     # out of range index
    col[4, 0] = 5                       # centre is not the row's node
    col[40:52] = np.stack([np.concatenate([[i], np.delete(np.arange(40, 52), i - 40)])
                           for i in range(40, 52)])
    rp = NS.csr_uniform(64, n)
    for prec in (P.FP64, P.FP32_IR):
        ns = NS.NodeSet(pts, np.zeros_like(pts), {"all": (0, 64)}, 0.1)
        got, status = run_gpu_weights(ctx, P, ns, rp, col.ravel().astype(np.int32),
                                      [(0, 64, n, 3, 2, 1)], prec)
        assert status[3] == P.binding.ST_BADARG and status[4] == P.binding.ST_BADARG
        assert (status[40:52] == P.binding.ST_SINGULAR).all()
        for i in [3, 4] + list(range(40, 52)):
            assert (got["lap"][rp[i]:rp[i + 1]] == 0).all()


# --------------------------------------------------------- operator application
def test_spmv_and_diffuse_match_oracle(P, ctx, oracle, weight_inputs):
    ns, rp, col, cls = weight_inputs("disk")
    got, _ = run_gpu_weights(ctx, P, ns, rp, col, cls, P.FP64)
    vals = got["lap"].copy()
    b0, b1 = ns.classes["boundary"]
    vals[rp[b0]:] = got["dn"][rp[b0]:]
    u = NS.sin_product(ns.pts)
    y0 = np.cos(ns.pts[:, 0])
    rp_d, col_d, v_d, u_d = dev(rp), dev(col), dev(vals), dev(u)
    y_d = dev(y0)
    ctx.apply_operator(rp_d, col_d, v_d, u_d, y_d, alpha=0.7, beta=-1.3)
    torch.cuda.synchronize()
    y = y_d.cpu().numpy()
    ref = oracle.spmv(rp, col, vals, u, alpha=0.7, beta=-1.3, y=y0)
    absw = oracle.spmv(rp, col, np.abs(vals), np.abs(u))
    n = np.diff(rp)
    bound = 2 * (n + 2) * U64 * (0.7 * absw + 1.3 * np.abs(y0))
    assert (np.abs(y - ref) <= bound).all()
    # explicit diffusion, boundary held
    fixed = np.zeros(ns.N, dtype=np.uint8)
    fixed[b0:b1] = 1
    lap = got["lap"]
    dt = 0.1 * ns.h ** 2
    u_d = dev(u)
    work = torch.empty_like(u_d)
    ctx.diffuse(rp_d, col_d, dev(lap), dev(fixed), dt, 20, u_d, work)
    torch.cuda.synchronize()
    ref = oracle.diffuse(rp, col, lap, fixed, dt, 20, u)
    assert np.abs(u_d.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("max_len", [60, 200])
def test_spmv_ragged_rows_match_oracle(P, ctx, oracle, max_len):
    """Random CSR rows of 0..max_len entries (mean ~30 or ~100, so both the
    2-lane and the 4-lane row groups run), covering every split of a lane's
    entries into batches of 8, 4, 2 and 1 and empty rows; y = alpha L u + beta
    y and y = L u within the rounding bound of the oracle's sum."""
    rng = np.random.default_rng(17 + max_len)
    nrows, ncols = 20011, 5003
    lens = rng.integers(0, max_len + 1, nrows)
    lens[::97] = 0
    rp = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    col = rng.integers(0, ncols, rp[-1]).astype(np.int32)
    vals = rng.standard_normal(rp[-1])
    u = rng.standard_normal(ncols)
    y0 = rng.standard_normal(nrows)
    absw = oracle.spmv(rp, col, np.abs(vals), np.abs(u))
    for alpha, beta in ((1.0, 0.0), (-0.6, 2.5)):
        y_d = dev(y0)
        ctx.apply_operator(dev(rp), dev(col), dev(vals), dev(u), y_d, alpha=alpha, beta=beta)
        torch.cuda.synchronize()
        y = y_d.cpu().numpy()
        ref = oracle.spmv(rp, col, vals, u, alpha=alpha, beta=beta, y=y0.copy())
        bound = 2 * (lens + 2) * U64 * (abs(alpha) * absw + abs(beta) * np.abs(y0))
        assert (np.abs(y - ref) <= bound).all(), (alpha, beta, np.abs(y - ref).max())
        if beta == 0.0:
            assert (y[lens == 0] == 0.0).all()


def test_full_size_disk_sampled(P, ctx, oracle):
    """The 1,000,000-node disk-with-holes workload in the launch
    configuration the benchmark times: grid kNN + FP32/FP64-refined weights;
    sampled rows against the oracle."""
    ns = NS.disk_holes(1_000_000, seed=0)
    (ib, ie), (bb, be) = ns.classes["interior"], ns.classes["boundary"]
    pts_d = dev(ns.pts)
    blocks, st = gpu_knn(ctx, P, pts_d, [(ib, ie, 25), (bb, be, 30)], P.KNN_GRID)
    assert (st == 0).all()
    rng = np.random.default_rng(11)
    qi = np.sort(rng.choice(np.arange(ib, ie), 300, replace=False))
    qb = np.sort(rng.choice(np.arange(bb, be), 100, replace=False))
    ref_i, _ = oracle.knn(ns.pts, 25, queries=qi, nthreads=16)
    ref_b, _ = oracle.knn(ns.pts, 30, queries=qb, nthreads=16)
    assert np.array_equal(blocks[0][qi - ib], ref_i)
    assert np.array_equal(blocks[1][qb - bb], ref_b)
    rp, col = csr_from_blocks(blocks)
    cls = [(ib, ie, 25, 5, 4, 1 | 2 | 4), (bb, be, 30, 5, 4, 16)]
    got, status = run_gpu_weights(ctx, P, ns, rp, col, cls, P.FP32_IR)
    assert set(np.unique(status)) <= {0, P.binding.ST_FALLBACK}
    for rows, (b, e, n, k, m, ops) in ((qi, cls[0]), (qb, cls[1])):
        ref = oracle_rows(oracle, ns.pts, ns.normals, rp, col, rows, k, m, ops)
        for oi, nm in enumerate(op_names(ops)):
            w_ref = np.zeros_like(got[nm])
            for i in rows:
                w_ref[rp[i]:rp[i + 1]] = ref[int(i)][oi]
            assert rel_err_rows(got[nm], w_ref, rp, rows).max() <= 1e-7
            assert monomial_residual(ns.pts, ns.normals, rp, col, got[nm], nm, m, rows) <= 1e-12
