"""Pins of the oracle's balanced stencils (Section 3.1, FindBalancedSupport:
stencils balanced around the central node; the rule is the library's
reading: a quota of (n - 1) / 2^dim candidates per orthant among the K
nearest, then the nearest of the rest).  CPU only."""
import numpy as np
import pytest

import nodesets as NS


def orthant(pts, c, j):
    d = pts[j] - pts[c]
    return sum(1 << a for a in range(pts.shape[1]) if d[a] < 0.0)


def test_hand_worked_one_sided_cluster(oracle):
    # centre at the origin, six close nodes to the right (alternating above
    # and below the axis), three far ones to the left; n = 5: one per quadrant
    pts = np.array([[0, 0], [1, 0.1], [1.1, -0.1], [1.2, 0.2], [1.3, -0.2], [1.4, 0.3], [1.5, -0.3],
                    [-3, 0.5], [-3.1, -0.5], [-3.2, 0.4]], dtype=float)
    knn, _ = oracle.knn(pts, 5, queries=[0])
    bal, st = oracle.balanced(pts, 5, 10, queries=[0])
    assert list(knn[0]) == [0, 1, 2, 3, 4]
    # quadrants: 1 (+,+), 2 (+,-), 7 (-,+), 8 (-,-): the left ones displace 3 and 4
    assert list(bal[0]) == [0, 1, 2, 7, 8] and st[0] == 0
    # with K too small to reach the left nodes the quota cannot be met: the
    # nearest fill the slots, i.e. plain kNN
    bal, _ = oracle.balanced(pts, 5, 7, queries=[0])
    assert list(bal[0]) == [0, 1, 2, 3, 4]
    # n = 9 (quota 2): two per quadrant where available, the rest by distance
    bal, _ = oracle.balanced(pts, 9, 10, queries=[0])
    assert list(bal[0]) == [0, 1, 2, 3, 4, 5, 7, 8, 9]


def test_k_equal_n_is_knn(oracle):
    ns = NS.disk_holes(3000, seed=3)
    q = np.arange(0, ns.N, 7)
    a, _ = oracle.knn(ns.pts, 12, queries=q)
    b, _ = oracle.balanced(ns.pts, 12, 12, queries=q)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("case", [("disk", 25, 48), ("disk", 13, 40), ("ball", 35, 64), ("ball", 17, 40)])
def test_balanced_invariants(oracle, case):
    """Every row: the node first, distinct nodes, all among the K nearest and
    in their ranking order; each orthant holds min(quota, its candidates)
    nodes or more; no candidate left out is closer than the nodes that filled
    the slots beyond the quotas."""
    name, n, K = case
    ns = NS.disk_holes(4000, seed=5) if name == "disk" else NS.ball(4000, seed=5)
    dim = ns.pts.shape[1]
    quota = (n - 1) // 2 ** dim
    q = np.arange(0, ns.N, 11)
    cand, _ = oracle.knn(ns.pts, K, queries=q)
    bal, st = oracle.balanced(ns.pts, n, K, queries=q)
    assert (st == 0).all()
    gained = 0
    for t, c in enumerate(q):
        row, cr = bal[t], cand[t]
        assert row[0] == c and len(set(row)) == n
        pos = [int(np.nonzero(cr == j)[0][0]) for j in row[1:]]
        assert pos == sorted(pos)                          # a subsequence of the ranking
        o_c = np.array([orthant(ns.pts, c, j) for j in cr[1:]])
        o_r = np.array([orthant(ns.pts, c, j) for j in row[1:]])
        for o in range(2 ** dim):
            assert (o_r == o).sum() >= min(quota, (o_c == o).sum())
        # the quota takes: first `quota` of each orthant in ranking order
        quota_taken = set()
        for o in range(2 ** dim):
            quota_taken |= set(cr[1:][o_c == o][:quota].tolist())
        assert quota_taken <= set(row[1:].tolist())
        fill = [j for j in row[1:] if j not in quota_taken]
        left = [j for j in cr[1:] if j not in set(row.tolist())]
        if fill and left:
            last_fill = max(int(np.nonzero(cr == j)[0][0]) for j in fill)
            first_left = min(int(np.nonzero(cr == j)[0][0]) for j in left)
            assert last_fill < first_left
        gained += int(not np.array_equal(row, cr[:n]))
    assert gained > 0          # the balancing changes some stencils (boundary ones)
