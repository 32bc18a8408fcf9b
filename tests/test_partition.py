"""Range partition of one node set over several ranks (CPU; gloo for the
multi-rank part): Morton ranges and halos, and a world-size-2 run in which
each rank forms the stencils, weights and explicit diffusion steps of its own
range from range + halo (oracle arithmetic, halo values exchanged with
send/recv every step) and gets exactly the single-process result."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import nodesets as NS


@pytest.fixture(scope="module")
def B():
    from paper_1912_13282_gb300 import _build
    _build.build()
    from paper_1912_13282_gb300 import binding
    return binding


def test_morton_ranges(B):
    ns = NS.disk_holes(5000, seed=2)
    perm, starts = B.partition_morton(ns.pts, 4)
    assert np.array_equal(np.sort(perm), np.arange(ns.N))
    assert starts[0] == 0 and starts[-1] == ns.N and (np.diff(starts) >= ns.N // 4).all()
    # Z-order ranges are compact: each range's bounding box is well below the domain's
    total = np.prod(ns.pts.max(0) - ns.pts.min(0))
    for p in range(4):
        x = ns.pts[perm[starts[p]:starts[p + 1]]]
        assert np.prod(x.max(0) - x.min(0)) < 0.6 * total
    # deterministic, and the order of a 2x2 grid is the Z curve
    assert np.array_equal(B.partition_morton(ns.pts, 4)[0], perm)
    g = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    assert list(B.partition_morton(g[[3, 1, 2, 0]], 1)[0]) == [3, 1, 2, 0]
    with pytest.raises(B.MMError):
        B.partition_morton(ns.pts, 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_halo_matches_brute_force(B, dim):
    ns = NS.disk_holes(3000, seed=4) if dim == 2 else NS.ball(3000, seed=4)
    perm, starts = B.partition_morton(ns.pts, 3)
    r = 3.5 * ns.h
    for p in range(3):
        own = perm[starts[p]:starts[p + 1]]
        halo = B.partition_halo(ns.pts, perm, starts[p], starts[p + 1], r)
        d2 = ((ns.pts[:, None, :] - ns.pts[None, own, :]) ** 2).sum(-1).min(1)
        ref = np.setdiff1d(np.nonzero(d2 <= r * r)[0], own)
        assert np.array_equal(halo, ref), p


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


CLASSES = (("interior", 25, 1), ("boundary", 30, 16))   # (class, n, ops) with k = 5, m = 4


def local_problem(oracle, ns, own, halo):
    """Range + halo of one rank in local numbering (the nodes in increasing
    global index, so exact distance ties rank as in the whole set): its
    stencils and weights (rows for its own nodes, empty rows for the halo)
    and the distance of each own stencil's farthest node."""
    from _helpers import oracle_rows
    local = np.sort(np.concatenate([own, halo]))
    own_pos = np.nonzero(np.isin(local, own))[0]
    lpts, lnrm = ns.pts[local], ns.normals[local]
    b, e = ns.classes["boundary"]
    cls = ((local >= b) & (local < e)).astype(np.int64)
    sizes = np.zeros(len(local), dtype=np.int64)
    sizes[own_pos] = np.where(cls[own_pos] == 1, CLASSES[1][1], CLASSES[0][1])
    rp = np.zeros(len(local) + 1, dtype=np.int64)
    np.cumsum(sizes, out=rp[1:])
    col = np.zeros(rp[-1], dtype=np.int32)
    far = np.zeros(len(local))
    vals = np.zeros(rp[-1])
    for c, (_, n, ops) in enumerate(CLASSES):
        rows = own_pos[cls[own_pos] == c]
        idx, _ = oracle.knn(lpts, n, queries=rows, nthreads=4)
        for t, i in enumerate(rows):
            col[rp[i]:rp[i + 1]] = idx[t]
            far[i] = np.sqrt(((lpts[idx[t][-1]] - lpts[i]) ** 2).sum())
        w = oracle_rows(oracle, lpts, lnrm, rp, col, rows, 5, 4, ops, nthreads=4)
        for i in rows:
            vals[rp[i]:rp[i + 1]] = w[int(i)][0]
    return local, own_pos, rp, col, vals, far[own_pos]


def global_problem(oracle, ns):
    b, e = ns.classes["boundary"]
    n_of = np.where((np.arange(ns.N) >= b) & (np.arange(ns.N) < e), 30, 25)
    rp = np.zeros(ns.N + 1, dtype=np.int64)
    np.cumsum(n_of, out=rp[1:])
    col = np.zeros(rp[-1], dtype=np.int32)
    for (cname, n, ops) in CLASSES:
        cb, ce = ns.classes[cname]
        idx, _ = oracle.knn(ns.pts, n, queries=np.arange(cb, ce), nthreads=4)
        col[rp[cb]:rp[ce]] = idx.ravel()
    vals = np.zeros(rp[-1])
    for (cname, n, ops) in CLASSES:
        cb, ce = ns.classes[cname]
        v, st, _ = oracle.weights(ns.pts, rp, col, 5, 4, ops, normals=ns.normals, rows=(cb, ce), nthreads=4)
        vals[rp[cb]:rp[ce]] = v[0][rp[cb]:rp[ce]]
    return rp, col, vals


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch
    import torch.distributed as dist
    from oracle import oracle
    from paper_1912_13282_gb300 import binding as Bd
    try:
        dist.init_process_group("gloo")
        ns = NS.disk_holes(6000, seed=3)
        radius = 6.0 * ns.h
        perm, starts = Bd.partition_morton(ns.pts, world)
        owns = [perm[starts[p]:starts[p + 1]] for p in range(world)]
        halos = [Bd.partition_halo(ns.pts, perm, starts[p], starts[p + 1], radius) for p in range(world)]
        own, halo = owns[rank], halos[rank]
        local, own_pos, rp, col, vals, far = local_problem(oracle, ns, own, halo)
        # every stencil's farthest node within the radius: the local stencils
        # are the whole set's (the halo criterion of mm_partition_halo)
        exact = bool((far <= radius).all())
        grp, gcol, gvals = global_problem(oracle, ns)
        same_st = all(np.array_equal(local[col[rp[i]:rp[i + 1]]], gcol[grp[g]:grp[g + 1]])
                      for i, g in zip(own_pos, local[own_pos]))
        same_w = all(np.array_equal(vals[rp[i]:rp[i + 1]], gvals[grp[g]:grp[g + 1]])
                     for i, g in zip(own_pos, local[own_pos]))
        # explicit diffusion (boundary nodes fixed), 10 steps; after each step
        # every rank sends the new values its neighbours hold as halo
        fixed = np.zeros(ns.N, dtype=np.uint8)
        fixed[ns.classes["boundary"][0]:ns.classes["boundary"][1]] = 1
        u0 = NS.sin_product(ns.pts)
        dt = 0.1 * ns.h ** 2
        owner = np.empty(ns.N, dtype=np.int64)
        for p in range(world):
            owner[owns[p]] = p
        u = u0[local].copy()
        upd = own_pos[fixed[local[own_pos]] == 0]
        for step in range(10):
            y = oracle.spmv(rp, col, vals, u)
            u[upd] = u[upd] + dt * y[upd]
            reqs = []
            for p in range(world):
                if p != rank:
                    send = halos[p][owner[halos[p]] == rank]
                    buf = torch.from_numpy(u[np.searchsorted(local, send)].copy())
                    reqs.append(dist.isend(buf, dst=p))
            for p in range(world):
                if p != rank:
                    recv_nodes = halo[owner[halo] == p]
                    buf = torch.empty(len(recv_nodes), dtype=torch.float64)
                    dist.recv(buf, src=p)
                    u[np.searchsorted(local, recv_nodes)] = buf.numpy()
            for r_ in reqs:
                r_.wait()
        ref = oracle.diffuse(grp, gcol, gvals, fixed, dt, 10, u0)
        same_u = bool(np.array_equal(u[own_pos], ref[local[own_pos]]))
        dist.barrier()
        q.put((rank, len(own), len(halo), exact, same_st, same_w, same_u))
        dist.destroy_process_group()
    except Exception as exc:   # report instead of hanging the parent
        q.put((rank, -1, -1, False, False, False, repr(exc)))


@pytest.mark.timeout(300)
def test_two_ranks_match_single_process(B, oracle):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=280) for _ in procs)
    for p in procs:
        p.join(timeout=30)
    for rank, nown, nhalo, exact, same_st, same_w, same_u in out:
        assert nown > 0 and nhalo > 0, (rank, same_u)
        assert exact and same_st and same_w, (rank, exact, same_st, same_w)
        assert same_u is True, (rank, same_u)
    assert out[0][1] + out[1][1] == NS.disk_holes(6000, seed=3).N
