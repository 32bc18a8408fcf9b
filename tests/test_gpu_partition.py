"""The range partition on the GPU kernels: a node set split into 4 Morton
ranges, each range's stencils (grid kNN), FP32 + refinement weights and 10
explicit diffusion steps computed from range + halo only (the ranks emulated
one after another on one GPU, the halo values copied between them after
every step), equal bit for bit to the single-set run."""
import numpy as np
import pytest
import torch

import nodesets as NS

pytestmark = pytest.mark.gpu

N_ST, K, M, OPS = 25, 5, 4, 1 | 2 | 4


def runs(mask):
    """Maximal runs [b, e) of True in a boolean array."""
    d = np.diff(np.concatenate([[0], mask.astype(np.int8), [0]]))
    return list(zip(np.nonzero(d == 1)[0], np.nonzero(d == -1)[0]))


def stencils_and_weights(P, ctx, pts, rows_mask):
    """kNN stencils (N_ST nodes) and weights of the rows in rows_mask (other
    rows empty) on the node set pts (device)."""
    N = pts.shape[0]
    sizes = np.where(rows_mask, N_ST, 0).astype(np.int64)
    rp = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(sizes, out=rp[1:])
    rp_d = torch.from_numpy(rp).cuda()
    col = torch.zeros(int(rp[-1]), dtype=torch.int32, device="cuda")
    ranges = [(int(b), int(e), N_ST, col[int(rp[b]):int(rp[e])]) for b, e in runs(rows_mask)]
    ctx.knn_stencils(pts, ranges, method=P.KNN_GRID)
    vals = [torch.zeros(int(rp[-1]), dtype=torch.float64, device="cuda") for _ in range(3)]
    for b, e in runs(rows_mask):
        ctx.rbffd_weights(OPS, K, M, pts, rp_d, col, vals, row_begin=int(b), row_end=int(e), n_max=N_ST,
                          precision=P.FP32_IR)
    torch.cuda.synchronize()
    return rp, rp_d, col, vals


def test_partitioned_run_equals_single_set():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1912_13282_gb300 import _build
    _build.build()
    import paper_1912_13282_gb300 as P
    ctx = P.Context(0)
    ns = NS.disk_holes(200_000, seed=12)
    N = ns.N
    fixed = np.zeros(N, dtype=np.uint8)
    fixed[ns.classes["boundary"][0]:ns.classes["boundary"][1]] = 1
    u0 = NS.sin_product(ns.pts)
    dt = 0.1 * ns.h ** 2

    # the whole set
    pts = torch.from_numpy(ns.pts).cuda()
    grp, grp_d, gcol, gvals = stencils_and_weights(P, ctx, pts, np.ones(N, dtype=bool))
    gu = torch.from_numpy(u0).cuda()
    ctx.diffuse(grp_d, gcol, gvals[0], torch.from_numpy(fixed).cuda(), dt, 10, gu, torch.empty_like(gu))
    torch.cuda.synchronize()
    gcol_h = gcol.cpu().numpy()
    gv_h = [v.cpu().numpy() for v in gvals]

    # four ranges with their halos
    nparts, radius = 4, 6.0 * ns.h
    perm, starts = P.partition_morton(ns.pts, nparts)
    parts = []
    for p in range(nparts):
        own = np.sort(perm[starts[p]:starts[p + 1]])
        halo = P.partition_halo(ns.pts, perm, starts[p], starts[p + 1], radius)
        local = np.sort(np.concatenate([own, halo]))       # global index order: same tie ranking
        is_own = np.isin(local, own)
        lpts = torch.from_numpy(ns.pts[local]).cuda()
        rp, rp_d, col, vals = stencils_and_weights(P, ctx, lpts, is_own)
        col_h = col.cpu().numpy()
        own_pos = np.nonzero(is_own)[0]
        # the halo criterion: every stencil's farthest node within the radius
        last = col_h[rp[own_pos] + N_ST - 1]
        far = np.sqrt(((ns.pts[local[last]] - ns.pts[local[own_pos]]) ** 2).sum(1))
        assert (far <= radius).all()
        # stencils and weights equal the whole set's, bit for bit
        gpos = (grp[local[own_pos]][:, None] + np.arange(N_ST)).ravel()
        lpos = (rp[own_pos][:, None] + np.arange(N_ST)).ravel()
        assert np.array_equal(local[col_h[lpos]], gcol_h[gpos])
        for v, gv in zip(vals, gv_h):
            assert np.array_equal(v.cpu().numpy()[lpos], gv[gpos])
        # diffusion: the halo rows are empty and held; own boundary rows held
        kind = np.where(is_own, fixed[local], 1).astype(np.uint8)
        parts.append({"local": local, "own_pos": own_pos, "rp_d": rp_d, "col": col, "lap": vals[0],
                      "fixed": torch.from_numpy(kind).cuda(), "u": torch.from_numpy(u0[local]).cuda(),
                      "halo_pos": np.nonzero(~is_own)[0]})
    owner = np.empty(N, dtype=np.int64)
    where = np.empty(N, dtype=np.int64)
    for p in range(nparts):
        owner[parts[p]["local"][parts[p]["own_pos"]]] = p
        where[parts[p]["local"][parts[p]["own_pos"]]] = parts[p]["own_pos"]
    for step in range(10):
        for q in parts:
            ctx.diffuse(q["rp_d"], q["col"], q["lap"], q["fixed"], dt, 1, q["u"], torch.empty_like(q["u"]))
        # halo exchange: each halo value from its owner's new field
        for q in parts:
            g = q["local"][q["halo_pos"]]
            for p in np.unique(owner[g]):
                sel = owner[g] == p
                src = torch.from_numpy(where[g[sel]]).cuda()
                dst = torch.from_numpy(q["halo_pos"][sel]).cuda()
                q["u"].index_copy_(0, dst, parts[p]["u"].index_select(0, src))
    torch.cuda.synchronize()
    gu_h = gu.cpu().numpy()
    for q in parts:
        got = q["u"].cpu().numpy()[q["own_pos"]]
        assert np.array_equal(got, gu_h[q["local"][q["own_pos"]]])
    ctx.close()
