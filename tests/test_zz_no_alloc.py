"""mm_rbffd_weights_ir_noalloc (the allocation-free variant of the FP32 +
FP64-refinement weights call) gives the same weights and statuses as
mm_rbffd_weights(..., MM_FP32_IR, ...), on two calls in a row.

Collected last on purpose; it must pass both alone and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import nodesets as NS

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_entry_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1912_13282_gb300 import _build
    _build.build()
    import paper_1912_13282_gb300 as P
    B = P.binding
    ctx = P.Context(0)
    ns = NS.disk_holes(30000, seed=21)
    (ib, ie), (bb, be) = ns.classes["interior"], ns.classes["boundary"]
    sizes = np.concatenate([np.full(ie - ib, 25), np.full(be - bb, 30)])
    rp = np.zeros(ns.N + 1, dtype=np.int64)
    np.cumsum(sizes, out=rp[1:])
    pts = torch.from_numpy(ns.pts).cuda()
    nrm = torch.from_numpy(ns.normals).cuda()
    rp_d = torch.from_numpy(rp).cuda()
    col = torch.empty(int(rp[-1]), dtype=torch.int32, device="cuda")
    ctx.knn_stencils(pts, [(ib, ie, 25, col[:(ie - ib) * 25]), (bb, be, 30, col[int(rp[bb]):])],
                     method=P.KNN_GRID)
    classes = [(ib, ie, 25, P.LAP | P.DX | P.DY), (bb, be, 30, P.DN)]

    def run(entry):
        vals = [torch.full((int(rp[-1]),), float("nan"), dtype=torch.float64, device="cuda")
                for _ in range(3)]
        status = torch.full((ns.N,), -1, dtype=torch.int32, device="cuda")
        for b, e, n, ops in classes:
            vv = vals if ops != P.DN else [vals[0]]
            if entry == "regular":
                ctx.rbffd_weights(ops, 5, 4, pts, rp_d, col, vv, row_begin=b, row_end=e, n_max=n,
                                  precision=P.FP32_IR, normals=nrm, status=status)
            else:
                ctx.rbffd_weights_ir_noalloc(ops, 5, 4, pts, rp_d, col, vv, row_begin=b,
                                             row_end=e, n_max=n, normals=nrm, status=status)
        torch.cuda.synchronize()
        return [v.cpu().numpy() for v in vals], status.cpu().numpy()

    ref_vals, ref_status = run("regular")
    assert set(np.unique(ref_status)) <= {B.ST_OK, B.ST_FALLBACK}
    for call in range(2):
        vals, status = run("noalloc")
        assert np.array_equal(status, ref_status), f"call {call}: statuses differ"
        for v, r in zip(vals, ref_vals):
            written = ~np.isnan(r)
            assert np.array_equal(np.isnan(v), np.isnan(r))
            per_row = np.abs(v[written] - r[written]).max() / np.abs(r[written]).max()
            assert per_row <= 1e-7, (call, per_row)

    # a range above the fixed queue's capacity is refused before any work
    big = B.CsrPattern((1 << 20) + 1, 1, rp_d.data_ptr(), col.data_ptr())
    dummy = torch.empty(1, dtype=torch.float64, device="cuda")
    vp = (C.c_void_p * 1)(dummy.data_ptr())
    lib = B.load()
    rc = lib.mm_rbffd_weights_ir_noalloc(ctx._h, P.LAP, 5, 4, 2, (1 << 20) + 2,
                                         C.c_void_p(pts.data_ptr()), None, C.byref(big), 0,
                                         (1 << 20) + 1, 25, vp, None)
    assert rc == B.MM_EUNSUPPORTED
    assert b"at most" in lib.mm_last_error(ctx._h)
    ctx.close()
