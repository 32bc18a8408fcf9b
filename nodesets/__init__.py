"""Seeded synthetic node sets and manufactured fields.

This module only places points, labels them and evaluates analytic test
functions.  It holds none of the method's arithmetic (no stencil selection, no
weights, no operator application), so both the CUDA path and the CPU oracle can
be fed from it without sharing any code with each other.

The workloads stand in for the paper's analytic domains: the jittered regular
grid on the unit square (Section 3.2, the Laplacian approximation test), the
annulus-like domains of the Poisson benchmark (Section 5), and the 3D ball.
No public dataset is involved.

Node order inside every set is grouped by class, so a class is a contiguous
index range ``classes[name] = (begin, end)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class NodeSet:
    pts: np.ndarray                 # [N, d] float64
    normals: np.ndarray             # [N, d] float64, outward unit normal, zero inside
    classes: dict                   # name -> (begin, end)
    h: float                        # nominal spacing
    dirichlet: np.ndarray = None    # [N] bool, boundary nodes with Dirichlet data
    neumann: np.ndarray = None      # [N] bool, boundary nodes with Neumann data
    info: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.pts.shape[0]

    @property
    def dim(self) -> int:
        return self.pts.shape[1]


# --------------------------------------------------------------- 2D square
def square(h: float = 0.01, jitter: float = 0.25, seed: int = 0) -> NodeSet:
    """Unit square [0,1]^2 on the grid x = i h, i = 0..1/h.

    Interior nodes are moved by U(-jitter h, +jitter h) per coordinate; edge
    nodes move only along their edge, corners stay.  Order: interior, boundary.
    All boundary nodes are Dirichlet.
    """
    nx = int(round(1.0 / h))
    rng = np.random.default_rng(seed)
    g = np.arange(nx + 1) * h
    X, Y = np.meshgrid(g, g, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel()], axis=1)
    I, J = np.meshgrid(np.arange(nx + 1), np.arange(nx + 1), indexing="ij")
    I, J = I.ravel(), J.ravel()
    onx = (I == 0) | (I == nx)
    ony = (J == 0) | (J == nx)
    interior = ~(onx | ony)
    jit = rng.uniform(-jitter * h, jitter * h, size=P.shape)
    P = P.copy()
    P[interior] += jit[interior]
    # edges: tangential jitter only (x-edge nodes move in y and vice versa), corners fixed
    ex = onx & ~ony
    ey = ony & ~onx
    P[ex, 1] += jit[ex, 1]
    P[ey, 0] += jit[ey, 0]
    nrm = np.zeros_like(P)
    nrm[I == 0, 0] = -1.0
    nrm[I == nx, 0] = 1.0
    nrm[J == 0, 1] = -1.0
    nrm[J == nx, 1] = 1.0
    ln = np.linalg.norm(nrm, axis=1)
    nrm[ln > 0] /= ln[ln > 0, None]
    order = np.concatenate([np.nonzero(interior)[0], np.nonzero(~interior)[0]])
    P, nrm = P[order], nrm[order]
    ni = int(interior.sum())
    N = P.shape[0]
    bnd = np.zeros(N, dtype=bool)
    bnd[ni:] = True
    return NodeSet(P, nrm, {"interior": (0, ni), "boundary": (ni, N)}, h,
                   dirichlet=bnd, neumann=np.zeros(N, dtype=bool),
                   info={"domain": "unit square", "seed": seed, "jitter": jitter})


def regular_grid(h: float) -> np.ndarray:
    """The plain grid G_h covering [0,1]^2 (no jitter), row-major."""
    nx = int(round(1.0 / h))
    g = np.arange(nx + 1) * h
    X, Y = np.meshgrid(g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


# ----------------------------------------------------- 2D disk minus holes
def disk_holes(N_target: int = 1_000_000, nholes: int = 5, seed: int = 0,
               jitter: float = 0.25) -> NodeSet:
    """Unit disk minus ``nholes`` circular holes.

    Hole radii U(0.05, 0.15); centres uniform in |c| <= 0.8, rejected unless
    every hole keeps a gap >= 0.02 to the others and to the outer circle.
    Spacing h = sqrt(area / N_target).  Interior: a jittered square grid
    (U(+-jitter h)) masked to the domain, nodes closer than h/2 to a boundary
    dropped.  Boundary: nodes at arclength spacing h with analytic outward
    normals (into the holes on hole boundaries).  Order: interior, boundary
    (outer circle, then the holes).  Outer circle Dirichlet, holes Neumann.
    """
    rng = np.random.default_rng(seed)
    holes = []
    while len(holes) < nholes:
        r = rng.uniform(0.05, 0.15)
        c = rng.uniform(-0.8, 0.8, size=2)
        if np.hypot(*c) > 0.8:
            continue
        if np.hypot(*c) + r > 1.0 - 0.02:
            continue
        if any(np.hypot(*(c - c2)) < r + r2 + 0.02 for c2, r2 in holes):
            continue
        holes.append((c, r))
    area = math.pi * (1.0 - sum(r * r for _, r in holes))
    h = math.sqrt(area / N_target)
    nx = int(math.ceil(2.0 / h)) + 1
    g = -1.0 + np.arange(nx) * h
    X, Y = np.meshgrid(g, g, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel()], axis=1)
    P += rng.uniform(-jitter * h, jitter * h, size=P.shape)
    keep = np.hypot(P[:, 0], P[:, 1]) < 1.0 - 0.5 * h
    for c, r in holes:
        keep &= np.hypot(P[:, 0] - c[0], P[:, 1] - c[1]) > r + 0.5 * h
    Pi = P[keep]
    bp, bn, bd = [], [], []
    K = int(round(2 * math.pi / h))
    t = rng.uniform(0, 2 * math.pi) + 2 * math.pi * np.arange(K) / K
    bp.append(np.stack([np.cos(t), np.sin(t)], 1))
    bn.append(np.stack([np.cos(t), np.sin(t)], 1))
    bd.append(np.ones(K, dtype=bool))
    for c, r in holes:
        K = max(8, int(round(2 * math.pi * r / h)))
        t = rng.uniform(0, 2 * math.pi) + 2 * math.pi * np.arange(K) / K
        u = np.stack([np.cos(t), np.sin(t)], 1)
        bp.append(c[None, :] + r * u)
        bn.append(-u)
        bd.append(np.zeros(K, dtype=bool))
    Pb = np.concatenate(bp)
    Nb = np.concatenate(bn)
    ni, nb = Pi.shape[0], Pb.shape[0]
    pts = np.concatenate([Pi, Pb])
    nrm = np.concatenate([np.zeros_like(Pi), Nb])
    N = ni + nb
    dmask = np.zeros(N, dtype=bool)
    dmask[ni:] = np.concatenate(bd)
    nmask = np.zeros(N, dtype=bool)
    nmask[ni:] = ~np.concatenate(bd)
    return NodeSet(np.ascontiguousarray(pts), np.ascontiguousarray(nrm),
                   {"interior": (0, ni), "boundary": (ni, N)}, h,
                   dirichlet=dmask, neumann=nmask,
                   info={"domain": "unit disk minus holes", "seed": seed,
                         "holes": [(c.tolist(), r) for c, r in holes]})


# ------------------------------------------------------------------ 3D ball
def ball(N_target: int = 4_000_000, seed: int = 0, jitter: float = 0.25,
         refined_radius: float = 0.5) -> NodeSet:
    """Unit ball: jittered cubic grid with h = (vol / N_target)^(1/3), nodes
    within h/2 of the sphere dropped, plus a Fibonacci lattice on the sphere at
    spacing h (outward normals).  Nodes with |x| < refined_radius form the
    'refined' class (same density; a class label).  Order: interior, refined,
    boundary.  All boundary nodes Dirichlet."""
    rng = np.random.default_rng(seed)
    h = (4.0 / 3.0 * math.pi / N_target) ** (1.0 / 3.0)
    nx = int(math.ceil(2.0 / h)) + 1
    g = (-1.0 + np.arange(nx) * h).astype(np.float64)
    parts = []
    for i in range(nx):          # slab by slab to bound memory
        Y, Z = np.meshgrid(g, g, indexing="ij")
        P = np.stack([np.full(Y.size, g[i]), Y.ravel(), Z.ravel()], 1)
        P += rng.uniform(-jitter * h, jitter * h, size=P.shape)
        parts.append(P[np.linalg.norm(P, axis=1) < 1.0 - 0.5 * h])
    P = np.concatenate(parts)
    r = np.linalg.norm(P, axis=1)
    ref = r < refined_radius
    Pint, Pref = P[~ref], P[ref]
    K = int(round(4 * math.pi / (h * h)))
    i = np.arange(K) + 0.5
    phi = np.arccos(1 - 2 * i / K)
    th = math.pi * (1 + 5 ** 0.5) * i
    B = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    pts = np.concatenate([Pint, Pref, B])
    nrm = np.concatenate([np.zeros_like(Pint), np.zeros_like(Pref), B])
    a, b = Pint.shape[0], Pint.shape[0] + Pref.shape[0]
    N = pts.shape[0]
    dmask = np.zeros(N, dtype=bool)
    dmask[b:] = True
    return NodeSet(np.ascontiguousarray(pts), np.ascontiguousarray(nrm),
                   {"interior": (0, a), "refined": (a, b), "boundary": (b, N)}, h,
                   dirichlet=dmask, neumann=np.zeros(N, dtype=bool),
                   info={"domain": "unit ball", "seed": seed})


# --------------------------------------------------------- training patches
def patches(count: int, seed: int, side: int = 9, max_jitter: float = 0.3,
            spacing: float = 12.0) -> NodeSet:
    """``count`` independent jittered grid patches of side x side nodes (unit
    spacing), each with its own jitter amplitude a ~ U(0, max_jitter) and node
    offsets U(-a, a) per coordinate.  Patches sit on a lattice ``spacing``
    apart, so the 25 nearest nodes of a patch centre all come from its own
    patch.  Order: the ``count`` patch centres first (class 'centre'), then the
    other nodes.  Used to make surrogate training and evaluation stencils."""
    rng = np.random.default_rng(seed)
    L = int(math.ceil(math.sqrt(count)))
    half = side // 2
    gi = np.arange(side) - half
    GX, GY = np.meshgrid(gi, gi, indexing="ij")
    G = np.stack([GX.ravel(), GY.ravel()], 1).astype(np.float64)   # [side^2, 2]
    ci = int(np.nonzero((G[:, 0] == 0) & (G[:, 1] == 0))[0][0])
    amp = rng.uniform(0.0, max_jitter, size=count)
    off = rng.uniform(-1.0, 1.0, size=(count, G.shape[0], 2)) * amp[:, None, None]
    p = np.arange(count)
    origin = np.stack([(p % L) * spacing, (p // L) * spacing], 1).astype(np.float64)
    P = origin[:, None, :] + G[None, :, :] + off                      # [count, side^2, 2]
    centres = P[:, ci, :]
    others = np.delete(P, ci, axis=1).reshape(-1, 2)
    pts = np.ascontiguousarray(np.concatenate([centres, others]))
    return NodeSet(pts, np.zeros_like(pts), {"centre": (0, count), "other": (count, pts.shape[0])},
                   1.0, info={"domain": "jittered patches", "seed": seed, "amplitude": amp})


# ------------------------------------------------------------ mixed batches
def batch_geometries(count: int = 64, seed: int = 0, n_min: float = 1e4, n_max: float = 2e6,
                     scale: float = 1.0):
    """Specs of ``count`` independent geometries: each a 2D disk with holes or
    a 3D ball (probability 1/2), node count log-uniform in [n_min, n_max]
    (times ``scale``).  Returns a list of dicts (dim, N_target, seed); build
    each with ``make_geometry``."""
    rng = np.random.default_rng(seed)
    out = []
    for g in range(count):
        dim = 2 if rng.uniform() < 0.5 else 3
        N = int(math.exp(rng.uniform(math.log(n_min), math.log(n_max))) * scale)
        out.append({"dim": dim, "N_target": max(N, 500), "seed": seed * 1000 + g + 1,
                    "stencil_choice": int(rng.integers(0, 2))})
    return out


def make_geometry(spec) -> NodeSet:
    if spec["dim"] == 2:
        return disk_holes(spec["N_target"], seed=spec["seed"])
    return ball(spec["N_target"], seed=spec["seed"])


# -------------------------------------------------------- manufactured fields
def sin_product(pts: np.ndarray) -> np.ndarray:
    """u = prod_a sin(pi x_a)."""
    return np.prod(np.sin(np.pi * pts), axis=1)


def sin_product_lap(pts: np.ndarray) -> np.ndarray:
    """Laplacian of sin_product: -d pi^2 u."""
    return -pts.shape[1] * np.pi ** 2 * sin_product(pts)


def sin_product_grad(pts: np.ndarray) -> np.ndarray:
    """Gradient of sin_product, [N, d]."""
    d = pts.shape[1]
    s = np.sin(np.pi * pts)
    c = np.cos(np.pi * pts)
    g = np.empty_like(pts)
    for a in range(d):
        f = np.pi * c[:, a]
        for b in range(d):
            if b != a:
                f = f * s[:, b]
        g[:, a] = f
    return g


def csr_uniform(N: int, n: int) -> np.ndarray:
    """row_ptr of N rows of n entries."""
    return np.arange(N + 1, dtype=np.int64) * n


def csr_classes(classes, sizes) -> np.ndarray:
    """row_ptr for nodes grouped by class: rows of class c have sizes[c] entries.
    ``classes`` maps name -> (begin, end) and must tile 0..N."""
    spans = sorted(classes.items(), key=lambda kv: kv[1][0])
    counts = []
    for name, (b, e) in spans:
        counts.append(np.full(e - b, sizes[name], dtype=np.int64))
    rp = np.zeros(sum(len(c) for c in counts) + 1, dtype=np.int64)
    np.cumsum(np.concatenate(counts), out=rp[1:])
    return rp
