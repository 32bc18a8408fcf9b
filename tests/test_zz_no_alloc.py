"""mm_rbffd_weights_ir_noalloc, the FP32 + FP64-refinement weights call for
callers that cannot allocate device memory when they call in (a memory pool
that already holds the GPU, or a loop where a cudaFree would synchronise the
device), gives the same weights and statuses as
mm_rbffd_weights(..., MM_FP32_IR, ...), bit for bit per row, on two calls in
a row, from a context that never allocates a workspace.

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
    ns = NS.disk_holes(30000, seed=21)
    (ib, ie), (bb, be) = ns.classes["interior"], ns.classes["boundary"]
    sizes = np.concatenate([np.full(ie - ib, 25), np.full(be - bb, 30)])
    rp = np.zeros(ns.N + 1, dtype=np.int64)
    np.cumsum(sizes, out=rp[1:])
    pts = torch.from_numpy(ns.pts).cuda()
    nrm = torch.from_numpy(ns.normals).cuda()
    rp_d = torch.from_numpy(rp).cuda()
    col = torch.empty(int(rp[-1]), dtype=torch.int32, device="cuda")
    classes = [(ib, ie, 25, P.LAP | P.DX | P.DY), (bb, be, 30, P.DN)]

    # stencils from a context of their own (the kNN grid uses a workspace)
    knn_ctx = P.Context(0)
    knn_ctx.knn_stencils(pts, [(ib, ie, 25, col[:(ie - ib) * 25]), (bb, be, 30, col[int(rp[bb]):])],
                         method=P.KNN_GRID)
    torch.cuda.synchronize()
    knn_ctx.close()

    def run(ctx, entry):
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

    # the allocation-free calls come first, on a context that never makes any
    # other call, so nothing else could have provided a workspace for them
    na_ctx = P.Context(0)
    assert na_ctx.workspace_bytes() == 0
    results = [run(na_ctx, "noalloc")]
    free_before = torch.cuda.mem_get_info()[0]
    results.append(run(na_ctx, "noalloc"))
    free_after = torch.cuda.mem_get_info()[0]
    assert na_ctx.workspace_bytes() == 0
    # the second call allocated nothing on the device (the result tensors of
    # run() come from torch's cache, which already held them after call 1)
    assert free_after >= free_before, (free_before, free_after)

    reg_ctx = P.Context(0)
    ref_vals, ref_status = run(reg_ctx, "regular")
    assert reg_ctx.workspace_bytes() > 0
    assert set(np.unique(ref_status)) <= {B.ST_OK, B.ST_FALLBACK}
    for call, (vals, status) in enumerate(results):
        assert np.array_equal(status, ref_status), f"call {call}: statuses differ"
        for v, r in zip(vals, ref_vals):
            # same kernels on the same inputs: every written entry is equal
            # bit for bit (NaN marks entries neither call writes)
            assert np.array_equal(v, r, equal_nan=True), f"call {call}: weights differ"

    # a range above the fixed queue's capacity is refused before any work
    big = B.CsrPattern((1 << 20) + 1, 1, rp_d.data_ptr(), col.data_ptr())
    dummy = torch.empty(1, dtype=torch.float64, device="cuda")
    vp = (C.c_void_p * 1)(dummy.data_ptr())
    lib = B.load()
    rc = lib.mm_rbffd_weights_ir_noalloc(na_ctx._h, P.LAP, 5, 4, 2, (1 << 20) + 2,
                                         C.c_void_p(pts.data_ptr()), None, C.byref(big), 0,
                                         (1 << 20) + 1, 25, vp, None)
    assert rc == B.MM_EUNSUPPORTED
    assert b"at most" in lib.mm_last_error(na_ctx._h)
    assert na_ctx.workspace_bytes() == 0
    na_ctx.close()
    reg_ctx.close()
