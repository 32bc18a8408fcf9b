"""Balanced stencils on the GPU (mm_balanced_stencils) equal the oracle's bit
for bit: 2D and 3D node sets, several stencil sizes and candidate counts,
ragged query ranges, K = n (plain kNN), grid and brute-force candidates."""
import numpy as np
import pytest
import torch

import nodesets as NS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1912_13282_gb300 import _build
    _build.build()
    import paper_1912_13282_gb300 as pkg
    return pkg


@pytest.mark.parametrize("case", [("disk", 25, 48), ("disk", 30, 64), ("square", 12, 32), ("ball", 35, 64),
                                  ("ball", 45, 60), ("disk", 9, 9)])
def test_balanced_matches_oracle(P, oracle, case):
    name, n, K = case
    ns = {"disk": lambda: NS.disk_holes(20000, seed=9), "square": lambda: NS.square(0.01, seed=9),
          "ball": lambda: NS.ball(20000, seed=9)}[name]()
    ctx = P.Context(0)
    pts = torch.from_numpy(ns.pts).cuda()
    # two ragged ranges covering a prefix and a suffix of the nodes
    r1 = (0, ns.N // 3 + 7)
    r2 = (ns.N // 2 + 3, ns.N)
    outs = []
    for method in (P.KNN_GRID, P.KNN_BRUTE):
        o1 = torch.full(((r1[1] - r1[0]), n), -7, dtype=torch.int32, device="cuda")
        o2 = torch.full(((r2[1] - r2[0]), n), -7, dtype=torch.int32, device="cuda")
        st = torch.full((ns.N,), -1, dtype=torch.int32, device="cuda")
        ctx.balanced_stencils(pts, [(r1[0], r1[1], n, o1), (r2[0], r2[1], n, o2)], K, method=method, status=st)
        torch.cuda.synchronize()
        outs.append((o1.cpu().numpy(), o2.cpu().numpy(), st.cpu().numpy()))
        if ns.N > 20000:
            break
    q = np.concatenate([np.arange(*r1), np.arange(*r2)])
    ref, rst = oracle.balanced(ns.pts, n, K, queries=q, nthreads=8)
    for o1, o2, st in outs:
        got = np.concatenate([o1, o2])
        assert np.array_equal(got, ref), np.argwhere(got != ref)[:5]
        assert np.array_equal(st[q], rst)
    if n == K:
        knn, _ = oracle.knn(ns.pts, n, queries=q, nthreads=8)
        assert np.array_equal(np.concatenate(outs[0][:2]), knn)
    ctx.close()
