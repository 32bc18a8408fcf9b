"""Benchmark: RBF-FD stencil-weight throughput (nodes/s).

Default workload (the one the headline metric is quoted on): the 1,000,000-node
2D unit disk minus 5 holes; interior nodes get 25-node stencils with PHS r^5 +
degree-4 monomials (Laplacian, d/dx, d/dy), boundary nodes 30-node stencils
with d/dn.  One step = the whole hot path over the node set: grid binning +
kNN stencils, weights for both classes in the chosen form (FP32 Gauss-Jordan
inverse with double-FP32 refinement and FP64 fallback), one application of
each assembled operator.  The same form with native FP64 residuals is timed
too.
The plain FP64 GPU path is timed the same way beside it; the sampled error
against the CPU oracle and the Poisson solution error of both weight sets are
reported with it.

Other workloads (--workload):
  ball       4,000,000-node 3D unit ball, three stencil classes (interior
             n=35 deg 2, refined n=60 deg 3, boundary n=45 d/dn) in one
             persistent launch with autotuned tiles.
  batch      64 independent 2D/3D node sets (10^4..2*10^6 nodes, log-uniform),
             all Laplacian weights + 100 explicit diffusion steps in one
             captured CUDA graph.
  surrogate  MLP surrogate trained on 2^20 patch stencils, evaluated on
             10^6 held-out stencils against the FP64 and FP32+IR paths, and
             at equal Poisson solution error on a 10^5-node disk.
  wls        GWLS weights (Section 2.2.1) on the 10^6-node disk.
  poisson    the implicit Poisson solve (Section 2.3.2) on a 2*10^4-node
             disk: assembly, ILU(0), BiCGSTAB.
  square     the small configuration: 10,201 nodes on the unit square, n=12
             r^3 deg 2, FP64 and FP32+IR, every row against the oracle,
             Dirichlet Poisson through the GPU implicit solve.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload disk|ball|batch|surrogate|wls|poisson|square]
Prints one JSON line (rank 0).  Under torchrun every rank runs its own
independent node set (seed = rank): weak scaling, no data-path collective;
the step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import shutil
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stencil weights nodes/s at stated error vs FP64 oracle; chosen form vs plain FP64 GPU"
DISK = {
    "workload": "disk minus 5 holes, 1e6 nodes: interior n=25 PHS r^5 + deg-4 monomials "
                "(lap, dx, dy); boundary n=30 d/dn",
    "N_target": 1_000_000,
    "interior": {"n": 25, "k": 5, "m": 4, "ops": 1 | 2 | 4},
    "boundary": {"n": 30, "k": 5, "m": 4, "ops": 16},
}
# kernels of one disk step: kNN (bbox, grid params, cell count, 3 scan passes,
# scatter, 2 queries) + per class (solve, FP64 fallback) x 2 + 3 SpMV
DISK_LAUNCHES_PER_STEP = 9 + 4 + 3


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="disk", choices=["disk", "ball", "batch", "surrogate", "wls", "poisson",
                                                          "square", "balanced", "convdiff"])
    ap.add_argument("--n-target", type=int, default=None, help="override the node count")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched-config", default=None,
                    help="ball: fixed launch shape 'warps_per_block,blocks_per_sm,chunk_rows' for both "
                         "precisions instead of the autotuner's")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-error", action="store_true")
    ap.add_argument("--no-poisson", action="store_true")
    ap.add_argument("--train-samples", type=int, default=1 << 20, help="surrogate: training stencils")
    ap.add_argument("--train-epochs", type=int, default=120, help="surrogate: training epochs")
    ap.add_argument("--train-batch", type=int, default=4096, help="surrogate: training batch (<= 65536)")
    return ap.parse_args(argv)


# --------------------------------------------------------------- ranks
class Ranks:
    """RANK / WORLD_SIZE / LOCAL_RANK from the environment, process group
    (NCCL on GPUs, gloo for the CPU tests) when WORLD_SIZE > 1."""

    def __init__(self, backend="nccl"):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            if backend == "nccl":
                dist.init_process_group("nccl", device_id=torch.device(f"cuda:{self.local}"))
            else:
                dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, values):
        """Element-wise maximum of a list of floats over all ranks."""
        if self.dist is None:
            return [float(v) for v in values]
        import torch
        dev = "cuda" if self.dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return [float(v) for v in t.cpu()]

    def sum(self, values):
        """Element-wise sum of a list of floats over all ranks."""
        if self.dist is None:
            return [float(v) for v in values]
        import torch
        dev = "cuda" if self.dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return [float(v) for v in t.cpu()]

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def throughput(units_all_ranks, ms_total_max, steps):
    """Whole-job units/s: the units all ranks process per step, over the
    slowest rank's time."""
    return units_all_ranks * steps / (ms_total_max * 1e-3)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        self.proc = subprocess.Popen([exe, f"--id={self.device}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits", "-lms", "200"],
                                     stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)

        def reader():
            for line in self.proc.stdout:
                self.samples.append([x.strip() for x in line.split(",")])
        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                smax.append(float(s[2]))
                for nm, v in zip(names, s[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------- roofline helpers
def mixed_fp32_flops(n, l, R, dim, k, residuals=2):
    """Algorithmic FP32 flops of the FP32+IR solve of one stencil (2 per
    multiply-add): the Gauss-Jordan inverse of the M x M system (every row
    updated at every step: M^3 multiply-adds), the products with the inverse
    (x0, one per refinement step, the constraint correction), the double-FP32
    residuals (15 FP32 flops per term of the compensated dot product) and the
    double-FP32 assembly (per pair: differences, squares, square root and
    powers of r; Q by products)."""
    M = n + l
    pairs = n * (n - 1) // 2
    gj = 2 * M ** 3
    applies = (residuals + 2) * 2 * M * M * R
    terms = residuals * R * (n * M + l * n) + R * n * l
    assembly = pairs * (18 * dim + 11 * (dim - 1) + 10 + 7 * ((k - 1) // 2)) + n * (l - 1) * 7
    return gj + applies + 15 * terms + assembly


def method_flops(n, l, R):
    """The method's algorithmic flops for one stencil, whatever the solver:
    an LU of the M x M augmented matrix ((2/3) M^3), forward and back
    substitution for R right-hand sides (2 R M^2) and the assembly (8 flops
    per node pair for the distance power, 4 per entry of Q, 6 per node and
    operator for the right-hand side): (2/3) M^3 + 2 R M^2 + 8 n(n-1)/2 +
    4 n l + 6 n R.  The same count serves the FP64 and the FP32 + refinement
    forms, so their roofline fractions compare the same work."""
    M = n + l
    return 2.0 * M ** 3 / 3 + 2 * R * M * M + 8 * n * (n - 1) / 2 + 4 * n * l + 6 * n * R


def fp64_solve_flops(n, l, R, dim, k):
    """Algorithmic FP64 flops of the plain solve: assembly, LU of the M x M
    augmented matrix applied to R right-hand sides, back substitution."""
    M = n + l
    pairs = n * (n - 1) // 2
    assembly = pairs * (2 * dim + 1 + (k + 1) // 2) + n * (l - 1) + n * (dim + 2 + R * (dim + 1))
    lu = sum(2 * (M - kk - 1) * (M + R - kk - 1) + (M - kk - 1) for kk in range(M))
    back = R * M * M
    return assembly + lu + back


def peaks_file():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def kernel_source_hash():
    """Hash of the weights kernel sources, to tie a stored ncu traffic figure
    to the kernel it was measured on."""
    h = hashlib.sha256()
    for f in ("rbffd_dev.cuh", "rbffd.cu", "mixed_launch.cuh", "mixed2d.cu"):
        with open(os.path.join(ROOT, "paper_1912_13282_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored_traffic(name):
    """(bytes per row, source hash) stored under profiles/ for a kernel, if the
    kernel source is unchanged since; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)[name]
    except Exception:
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d


# ------------------------------------------------------------ disk workload
def make_disk(seed: int, n_target: int):
    import nodesets as NS
    ns = NS.disk_holes(n_target, seed=seed)
    (ib, ie), (bb, be) = ns.classes["interior"], ns.classes["boundary"]
    sizes = np.concatenate([np.full(ie - ib, DISK["interior"]["n"]),
                            np.full(be - bb, DISK["boundary"]["n"])])
    rp = np.zeros(ns.N + 1, dtype=np.int64)
    np.cumsum(sizes, out=rp[1:])
    return ns, rp


class DiskPipeline:
    """Device buffers and calls of one disk step."""

    def __init__(self, P, ctx, ns, rp, device):
        import torch
        self.P, self.ctx, self.ns = P, ctx, ns
        self.N = ns.N
        (self.ib, self.ie), (self.bb, self.be) = ns.classes["interior"], ns.classes["boundary"]
        self.rp_h = rp
        self.nnz = int(rp[-1])
        dv = f"cuda:{device}"
        self.pts = torch.from_numpy(ns.pts).to(dv)
        self.nrm = torch.from_numpy(ns.normals).to(dv)
        self.rp = torch.from_numpy(rp).to(dv)
        self.col = torch.empty(self.nnz, dtype=torch.int32, device=dv)
        # one operator array: Laplacian rows (interior) and d/dn rows (boundary)
        self.op = torch.zeros(self.nnz, dtype=torch.float64, device=dv)
        self.dx = torch.zeros(self.nnz, dtype=torch.float64, device=dv)
        self.dy = torch.zeros(self.nnz, dtype=torch.float64, device=dv)
        self.status = torch.empty(self.N, dtype=torch.int32, device=dv)
        self.u = torch.from_numpy(np.sin(np.pi * ns.pts[:, 0]) * np.sin(np.pi * ns.pts[:, 1])).to(dv)
        self.y = torch.empty(self.N, dtype=torch.float64, device=dv)
        self.gy = torch.empty(self.N, dtype=torch.float64, device=dv)
        ni, nb = DISK["interior"]["n"], DISK["boundary"]["n"]
        self.ranges = [(self.ib, self.ie, ni, self.col[:(self.ie - self.ib) * ni]),
                       (self.bb, self.be, nb, self.col[int(rp[self.bb]):])]

    def knn(self):
        self.ctx.knn_stencils(self.pts, self.ranges, method=self.P.KNN_GRID)

    def weights_interior(self, precision):
        wi = DISK["interior"]
        self.ctx.rbffd_weights(wi["ops"], wi["k"], wi["m"], self.pts, self.rp, self.col,
                               [self.op, self.dx, self.dy], row_begin=self.ib, row_end=self.ie,
                               n_max=wi["n"], precision=precision, normals=self.nrm,
                               status=self.status)

    def weights_boundary(self, precision):
        wb = DISK["boundary"]
        self.ctx.rbffd_weights(wb["ops"], wb["k"], wb["m"], self.pts, self.rp, self.col, [self.op],
                               row_begin=self.bb, row_end=self.be, n_max=wb["n"],
                               precision=precision, normals=self.nrm, status=self.status)

    def apply(self):
        self.ctx.apply_operator(self.rp, self.col, self.op, self.u, self.y)
        self.ctx.apply_operator(self.rp, self.col, self.dx, self.u, self.gy)
        self.ctx.apply_operator(self.rp, self.col, self.dy, self.u, self.gy, beta=1.0)

    def step(self, precision):
        self.knn()
        self.weights_interior(precision)
        self.weights_boundary(precision)
        self.apply()

    def step_host(self, precision, h_pts, h_nrm, h_out, copy_stream, chunks=8):
        """The same step with host inputs and outputs: points and normals
        copied in, then the interior weights in row chunks, each chunk's three
        value ranges copied to the pinned host arrays h_out on copy_stream
        while the next chunk computes (the step ends when every copy has)."""
        import torch
        cur = torch.cuda.current_stream(self.pts.device)
        self.pts.copy_(h_pts, non_blocking=True)
        self.nrm.copy_(h_nrm, non_blocking=True)
        self.knn()

        def fetch(b, e):
            ev = torch.cuda.Event()
            ev.record(cur)
            copy_stream.wait_event(ev)
            lo, hi = int(self.rp_h[b]), int(self.rp_h[e])
            with torch.cuda.stream(copy_stream):
                for h, d in zip(h_out, (self.op, self.dx, self.dy)):
                    h[lo:hi].copy_(d[lo:hi], non_blocking=True)

        wi = DISK["interior"]
        bounds = np.linspace(self.ib, self.ie, chunks + 1).astype(np.int64)
        for b, e in zip(bounds[:-1], bounds[1:]):
            self.ctx.rbffd_weights(wi["ops"], wi["k"], wi["m"], self.pts, self.rp, self.col,
                                   [self.op, self.dx, self.dy], row_begin=int(b), row_end=int(e),
                                   n_max=wi["n"], precision=precision, normals=self.nrm,
                                   status=self.status)
            fetch(b, e)
        self.weights_boundary(precision)
        fetch(self.bb, self.be)
        self.apply()
        cur.wait_stream(copy_stream)


def timed_disk_steps(pipe, precision, steps, stream, flush):
    """Per-step CUDA-event times (L2 flushed between steps): whole step,
    weights, and the dominant launch (interior weights); the operator
    applications' and the kNN's times are left in timed_disk_steps.apply_ms
    and timed_disk_steps.knn_ms."""
    import torch
    tot, wts, dom, app, kn = [], [], [], [], []
    for _ in range(steps):
        flush.add_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        pipe.knn()
        ev[1].record(stream)
        pipe.weights_interior(precision)
        ev[2].record(stream)
        pipe.weights_boundary(precision)
        ev[3].record(stream)
        pipe.apply()
        ev[4].record(stream)
        ev[4].synchronize()
        tot.append(ev[0].elapsed_time(ev[4]))
        wts.append(ev[1].elapsed_time(ev[3]))
        dom.append(ev[1].elapsed_time(ev[2]))
        app.append(ev[3].elapsed_time(ev[4]))
        kn.append(ev[0].elapsed_time(ev[1]))
    timed_disk_steps.apply_ms = np.array(app)
    timed_disk_steps.knn_ms = np.array(kn)
    return np.array(tot), np.array(wts), np.array(dom)


def oracle_rows(ns, rp, col, rows, k, m, ops, nthreads=None):
    """Oracle weights of arbitrary CSR rows (local renumbering, rows first);
    returns {row: [R, n]}."""
    from oracle import oracle as O
    sts = [col[rp[i]:rp[i + 1]] for i in rows]
    others = np.setdiff1d(np.unique(np.concatenate(sts)), rows)
    order = np.concatenate([rows, others])
    remap = np.full(ns.N, -1, dtype=np.int64)
    remap[order] = np.arange(len(order))
    lcol = np.concatenate([remap[s] for s in sts]).astype(np.int32)
    lrp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum([len(s) for s in sts], out=lrp[1:])
    vals, st, _ = O.weights(ns.pts[order], lrp, lcol, k, m, ops, normals=ns.normals[order],
                            rows=(0, len(rows)), nthreads=nthreads or O.nthreads_default())
    return {int(i): vals[:, lrp[t]:lrp[t + 1]] for t, i in enumerate(rows)}


def sampled_error(pipe, rows_per_class=200, seed=0):
    """Max / median relative weight error per operator and the scaled
    monomial-reproduction residual on sampled rows, against the oracle."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from _helpers import monomial_residual, rel_err_rows
    ns, rp = pipe.ns, pipe.rp_h
    col = pipe.col.cpu().numpy()
    got = {"lap": pipe.op.cpu().numpy(), "dx": pipe.dx.cpu().numpy(),
           "dy": pipe.dy.cpu().numpy(), "dn": pipe.op.cpu().numpy()}
    rng = np.random.default_rng(seed)
    out = {}
    for (b, e), spec, names in (((pipe.ib, pipe.ie), DISK["interior"], ["lap", "dx", "dy"]),
                                ((pipe.bb, pipe.be), DISK["boundary"], ["dn"])):
        rows = np.sort(rng.choice(np.arange(b, e), min(rows_per_class, e - b), replace=False))
        ref = oracle_rows(ns, rp, col, rows, spec["k"], spec["m"], spec["ops"])
        for oi, nm in enumerate(names):
            w_ref = np.zeros_like(got[nm])
            for i in rows:
                w_ref[rp[i]:rp[i + 1]] = ref[int(i)][oi]
            err = rel_err_rows(got[nm], w_ref, rp, rows)
            mono = monomial_residual(ns.pts, ns.normals, rp, col, got[nm], nm, spec["m"], rows)
            out[nm] = {"max_rel_err": float(err.max()), "median_rel_err": float(np.median(err)),
                       "monomial_residual": float(mono), "rows": int(len(rows))}
    return out


def poisson_error(ns, rp, col, op_vals):
    """Max-norm error of the manufactured Poisson problem on the disk with
    holes (Section 2.3.2 assembly): interior rows  Laplacian weights, u_xx +
    u_yy = f; outer circle Dirichlet rows (identity), hole boundaries Neumann
    rows (d/dn weights), u = sin(pi x) sin(pi y).  Solved with scipy (not
    timed)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    import nodesets as NS
    # copies: scipy keeps the given arrays and sorts their rows in place
    A = sp.csr_matrix((np.array(op_vals, dtype=np.float64), np.array(col), np.array(rp)),
                      shape=(ns.N, ns.N)).tolil()
    u = NS.sin_product(ns.pts)
    rhs = NS.sin_product_lap(ns.pts)
    g = NS.sin_product_grad(ns.pts)
    for i in np.nonzero(ns.dirichlet)[0]:
        A.rows[i] = [int(i)]
        A.data[i] = [1.0]
        rhs[i] = u[i]
    nb = np.nonzero(ns.neumann)[0]
    rhs[nb] = (g[nb] * ns.normals[nb]).sum(1)
    sol = spla.spsolve(A.tocsc(), rhs)
    return float(np.abs(sol - u).max())


def poisson_comparison(P, ctx, device, n_target=100_000):
    """Poisson error with plain FP64 weights and with the chosen form on a
    smaller disk (the sparse direct solve of the full size is not needed to
    compare them): 'equal' means within 1% relative."""
    import torch
    ns, rp = make_disk(7, n_target)
    pipe = DiskPipeline(P, ctx, ns, rp, device)
    out = {}
    for name, prec in (("fp64", P.FP64), ("fp32_ir", P.FP32_IR)):
        pipe.knn()
        pipe.weights_interior(prec)
        pipe.weights_boundary(prec)
        torch.cuda.synchronize()
        out[name] = poisson_error(ns, rp, pipe.col.cpu().numpy(), pipe.op.cpu().numpy())
    out["N"] = ns.N
    out["note"] = "a smaller instance of the same disk workload (the host direct solve is untimed)"
    out["relative_difference"] = abs(out["fp32_ir"] - out["fp64"]) / out["fp64"]
    out["equal_within_1pct"] = out["relative_difference"] <= 0.01
    return out


def cpu_baseline_disk(ns, rp, col_h, seconds=15.0, seed=0):
    """The oracle timed on the host cores on a bounded sample of the disk
    workload: brute-force kNN of S_k queries and weights of S_w rows (interior
    and boundary in proportion), all cores.  nodes/s of kNN + weights."""
    from oracle import oracle as O
    threads = O.nthreads_default()
    rng = np.random.default_rng(seed)
    (ib, ie), (bb, be) = ns.classes["interior"], ns.classes["boundary"]
    frac_b = (be - bb) / ns.N
    q = rng.choice(np.arange(ib, ie), 64, replace=False)
    t0 = time.perf_counter()
    O.knn(ns.pts, 25, queries=q, nthreads=threads)
    per = (time.perf_counter() - t0) / 64
    sk = int(max(64, min(20000, seconds / 3 / max(per, 1e-9))))
    qi = rng.choice(np.arange(ib, ie), sk, replace=False)
    t0 = time.perf_counter()
    O.knn(ns.pts, 25, queries=qi, nthreads=threads)
    t_knn = (time.perf_counter() - t0) / sk
    sw = 20000
    t_w = 0.0
    for (b, e), spec, share in (((ib, ie), DISK["interior"], 1 - frac_b),
                                ((bb, be), DISK["boundary"], frac_b)):
        rows = np.sort(rng.choice(np.arange(b, e), max(1, int(sw * share)), replace=False))
        t0 = time.perf_counter()
        oracle_rows(ns, rp, col_h, rows, spec["k"], spec["m"], spec["ops"])
        t_w += (time.perf_counter() - t0) / len(rows) * share
    # one thread: a smaller sample of the same mix
    q1 = rng.choice(np.arange(ib, ie), 32, replace=False)
    t0 = time.perf_counter()
    O.knn(ns.pts, 25, queries=q1, nthreads=1)
    t_knn1 = (time.perf_counter() - t0) / len(q1)
    t_w1 = 0.0
    for (b, e), spec, share in (((ib, ie), DISK["interior"], 1 - frac_b),
                                ((bb, be), DISK["boundary"], frac_b)):
        rows = np.sort(rng.choice(np.arange(b, e), max(1, int(1000 * share)), replace=False))
        t0 = time.perf_counter()
        oracle_rows(ns, rp, col_h, rows, spec["k"], spec["m"], spec["ops"], nthreads=1)
        t_w1 += (time.perf_counter() - t0) / len(rows) * share
    return {"value": 1.0 / (t_knn + t_w), "unit": "nodes/s", "cores": threads, "kind": "oracle",
            "sample": f"{sk} brute-force kNN queries over all {ns.N} nodes + {sw} weight rows "
                      f"(interior/boundary in proportion), all host cores",
            "knn_s_per_node": t_knn, "weights_s_per_node": t_w,
            "single_thread": {"value": 1.0 / (t_knn1 + t_w1), "unit": "nodes/s", "cores": 1,
                              "sample": f"{len(q1)} kNN queries + 1000 weight rows, one thread",
                              "knn_s_per_node": t_knn1, "weights_s_per_node": t_w1}}


def cpu_baseline_classes(ns, rp, col_h, spans, seconds=15.0, seed=0):
    """The oracle timed on the host cores on a bounded sample of a workload
    with several stencil classes (spans: (row_begin, row_end, n, k, m, ops)): per class,
    brute-force kNN of some of its queries and weights of some of its rows,
    weighted by the class's share of the nodes; all cores, and one thread on
    a smaller sample.  nodes/s of kNN + weights."""
    from oracle import oracle as O
    threads = O.nthreads_default()
    rng = np.random.default_rng(seed)
    shares = [(e - b) / ns.N for b, e, *_ in spans]

    def timed(nthreads, queries_total, rows_total):
        t_knn = t_w = 0.0
        q_used = r_used = 0
        for (b, e, n, k, m, ops), share in zip(spans, shares):
            nq = max(1, min(e - b, int(queries_total * share)))
            q = rng.choice(np.arange(b, e), nq, replace=False)
            t0 = time.perf_counter()
            O.knn(ns.pts, n, queries=q, nthreads=nthreads)
            t_knn += (time.perf_counter() - t0) / nq * share
            nr = max(1, min(e - b, int(rows_total * share)))
            rows = np.sort(rng.choice(np.arange(b, e), nr, replace=False))
            t0 = time.perf_counter()
            oracle_rows(ns, rp, col_h, rows, k, m, ops, nthreads=nthreads)
            t_w += (time.perf_counter() - t0) / nr * share
            q_used += nq
            r_used += nr
        return t_knn, t_w, q_used, r_used

    # size the all-core sample from a short probe so it takes about `seconds`
    tk, tw, _, _ = timed(threads, 64, 256)
    scale = max(1.0, seconds / max((tk * 64 + tw * 256), 1e-9))
    t_knn, t_w, nq, nr = timed(threads, int(min(20000, 64 * scale)), int(min(20000, 256 * scale)))
    t_knn1, t_w1, nq1, nr1 = timed(1, 32, 256)
    return {"value": 1.0 / (t_knn + t_w), "unit": "nodes/s", "cores": threads, "kind": "oracle",
            "sample": f"{nq} brute-force kNN queries over all {ns.N} nodes + {nr} weight rows "
                      f"(classes in proportion to their nodes), all host cores",
            "knn_s_per_node": t_knn, "weights_s_per_node": t_w,
            "single_thread": {"value": 1.0 / (t_knn1 + t_w1), "unit": "nodes/s", "cores": 1,
                              "sample": f"{nq1} kNN queries + {nr1} weight rows, one thread",
                              "knn_s_per_node": t_knn1, "weights_s_per_node": t_w1}}


def run_disk(args, rk):
    import torch
    import paper_1912_13282_gb300 as P
    device = rk.local
    stream = torch.cuda.current_stream(device)
    ctx = P.Context(device, stream)
    n_target = args.n_target or DISK["N_target"]
    ns, rp = make_disk(rk.rank, n_target)
    pipe = DiskPipeline(P, ctx, ns, rp, device)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=f"cuda:{device}")
    fp64_peak = ctx.measure_fma_peak(0)
    fp32_peak = ctx.measure_fma_peak(1)
    for _ in range(max(3, args.warmup)):
        pipe.step(P.FP64)
        pipe.step(P.FP32_IR)
    torch.cuda.synchronize()
    clocks = ClockSampler(device)
    clocks.start()
    rk.barrier()
    torch.cuda.synchronize()
    t64, w64, d64 = timed_disk_steps(pipe, P.FP64, args.steps, stream, flush)
    rk.barrier()
    torch.cuda.synchronize()
    tot, wts, dom = timed_disk_steps(pipe, P.FP32_IR, args.steps, stream, flush)
    apply_ms = float(np.median(timed_disk_steps.apply_ms))
    knn_ms = float(np.mean(timed_disk_steps.knn_ms))
    torch.cuda.synchronize()
    # the same chosen form with native FP64 refinement residuals (MM_WIDE_FP64)
    ctx.set_option(P.binding.OPT_WIDE, P.binding.WIDE_FP64)
    pipe.step(P.FP32_IR)
    rk.barrier()
    torch.cuda.synchronize()
    tw, ww, dw = timed_disk_steps(pipe, P.FP32_IR, args.steps, stream, flush)
    ctx.set_option(P.binding.OPT_WIDE, P.binding.WIDE_FF)
    pipe.step(P.FP32_IR)
    torch.cuda.synchronize()
    rk.barrier()
    clk = clocks.stop()
    ms, ms64, msw = rk.max([tot.sum(), t64.sum(), tw.sum()])
    status = pipe.status.cpu().numpy()
    fallback = float((status == P.binding.ST_FALLBACK).mean())
    (n_all,) = rk.sum([ns.N])
    value = throughput(n_all, ms, args.steps)

    e2e = None
    if not args.no_e2e:
        h_pts = torch.from_numpy(ns.pts).pin_memory()
        h_nrm = torch.from_numpy(ns.normals).pin_memory()
        h_out = [torch.empty(pipe.nnz, dtype=torch.float64).pin_memory() for _ in range(3)]
        copy_stream = torch.cuda.Stream(device)
        pipe.step_host(P.FP32_IR, h_pts, h_nrm, h_out, copy_stream)
        torch.cuda.synchronize()
        e_ms = []
        for _ in range(args.steps):
            flush.add_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pipe.step_host(P.FP32_IR, h_pts, h_nrm, h_out, copy_stream)
            b.record(stream)
            b.synchronize()
            e_ms.append(a.elapsed_time(b))
        (e_tot,) = rk.max([float(np.sum(e_ms))])
        e2e = {"value": throughput(n_all, e_tot, args.steps), "unit": "nodes/s",
               "h2d_bytes_per_step": int((h_pts.numel() + h_nrm.numel()) * 8),
               "d2h_bytes_per_step": int(sum(h.numel() * 8 for h in h_out)),
               "overlap": "interior weights in 8 row chunks; each chunk's values copied to pinned "
                          "host memory on a second stream while the next chunk computes"}
        # the host copies must equal the device weights of the same step
        for h, d in zip(h_out, (pipe.op, pipe.dx, pipe.dy)):
            if not torch.equal(h, d.cpu()):
                raise RuntimeError("host copy of the weights differs from the device arrays")

    # general second-order operator (eq. gen-op) from the three weight arrays
    # with per-node coefficients, timed alone: HBM-bound, (terms + 1) x 8 bytes
    # per nonzero plus the coefficients and row pointers
    coefs = [torch.ones(ns.N, dtype=torch.float64, device=pipe.pts.device) * c for c in (1.0, 0.5, -0.25)]
    wl = torch.empty_like(pipe.op)
    cm = []
    for t in range(max(3, args.warmup) + args.steps):
        flush.add_(1.0)
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.combine_operators(pipe.rp, pipe.col, [pipe.op, pipe.dx, pipe.dy], coefs, wl)
        z.record(stream)
        z.synchronize()
        if t >= max(3, args.warmup):
            cm.append(a.elapsed_time(z))
    comb_bytes = 4 * 8 * pipe.nnz + 3 * 8 * ns.N + 8 * (ns.N + 1)
    hbm = peaks_file().get("hbm_gbs")
    comb_gbs = comb_bytes / (float(np.mean(cm)) * 1e-3) / 1e9
    comb_roof = {"bound": "hbm", "kernel": "k_combine (3 weight arrays, per-node coefficients)",
                 "achieved": comb_gbs, "unit": "GB/s", "peak": hbm, "frac": comb_gbs / hbm if hbm else None,
                 "ms": float(np.mean(cm)), "bytes": comb_bytes,
                 "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}

    wi = DISK["interior"]
    Ni = pipe.ie - pipe.ib
    alg = method_flops(wi["n"], 15, 3) * Ni
    issued = mixed_fp32_flops(wi["n"], 15, 3, 2, wi["k"]) * Ni
    dom_ms = float(np.mean(dom))
    achieved = alg / (dom_ms * 1e-3)
    traffic = stored_traffic("k_weights_mixed<2,2,3,40>")
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": fp32_peak / 1e12,
            "unit": "TFLOP/s", "frac": achieved / fp32_peak,
            "traffic": None if traffic is None else traffic.get("full_size", traffic)["bytes_per_row"] * Ni,
            "traffic_source": "profiles/traffic.json: one-pass ncu dram__bytes_read.sum + dram__bytes_write.sum "
                              "of this launch on this workload, per row x rows",
            "kernel": "k_weights_mixed<2,2,3,40> (interior rows; FP32 Gauss-Jordan inverse with the "
                      "rows in registers + double-FP32 refinement)",
            "algorithmic": "the method's flops per interior stencil, (2/3)M^3 + 2RM^2 + 8n(n-1)/2 + 4nl "
                           "+ 6nR = %.0f (M=40, R=3, n=25, l=15) x %d rows per launch (bench.method_flops)"
                           % (method_flops(wi["n"], 15, 3), Ni),
            "issued_flops": issued,
            "issued_tflops": issued / (dom_ms * 1e-3) / 1e12,
            "issued_note": "FP32 flops the implementation executes (explicit inverse 2M^3, products with "
                           "it, 15-flop compensated residual terms, double-FP32 assembly; "
                           "bench.mixed_fp32_flops); not the method's work",
            "frac_of_fp64_peak": achieved / fp64_peak,
            "ms": dom_ms, "units": Ni,
            "peak_source": "FP32 FMA peak measured in this run (mm_measure_fma_peak); "
                           "MEASURED_PEAKS.json has no FP32 CUDA-core figure"}
    f64_plain = method_flops(wi["n"], 15, 3) * Ni
    # operator application (3 SpMVs, the last with beta = 1): values and column
    # indices once, row pointers, x and y once per row (algorithmic bytes)
    N = ns.N
    spmv_bytes = 3 * (12 * pipe.nnz + 8 * (N + 1) + 16 * N) + 8 * N
    hbm = peaks_file().get("hbm_gbs")
    spmv_roof = {"bound": "hbm", "kernel": "k_spmv (3 operator applications per step)",
                 "achieved": spmv_bytes / (apply_ms * 1e-3) / 1e9, "unit": "GB/s",
                 "peak": hbm, "frac": (spmv_bytes / (apply_ms * 1e-3) / 1e9 / hbm) if hbm else None,
                 "bytes": spmv_bytes, "ms": apply_ms,
                 "fp64_pipe_frac": 3 * 2.0 * pipe.nnz / (apply_ms * 1e-3) / fp64_peak,
                 "note": "one FP64 multiply-add per nonzero: fp64_pipe_frac is their rate against the measured "
                         "FP64 peak; on GB300 the FP64 pipe co-bounds this kernel with HBM",
                 "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}
    # the method's flops delivered per second by the chosen form, against FP64
    fp64_equiv = {"tflops": f64_plain / (dom_ms * 1e-3) / 1e12,
                  "frac_of_fp64_peak": f64_plain / (dom_ms * 1e-3) / fp64_peak}
    # kNN stencils (grid build + ring search): the output rows and the
    # coordinates once (n x 4 + 8 d bytes per node, plus 8 d for the sorted copy
    # and 12 for the cell keys, counts and permutation)
    knn_bytes = ns.N * (DISK["interior"]["n"] * 4 + 8 * 2 * 2 + 12)
    knn_roof = {"bound": "hbm", "kernel": "k_knn_grid<2> + grid build (whole kNN phase)",
                "achieved": knn_bytes / (knn_ms * 1e-3) / 1e9, "unit": "GB/s", "peak": hbm,
                "frac": (knn_bytes / (knn_ms * 1e-3) / 1e9 / hbm) if hbm else None,
                "bytes": knn_bytes, "ms": knn_ms, "nodes_per_s": ns.N / (knn_ms * 1e-3),
                "note": "HBM reference of the survey; the ring search is bound by integer/ALU issue "
                        "(keys compared as integers), with the exact FP64 keys on full batches keeping "
                        "the FP64 pipe about half busy; not by HBM",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}
    line = {"metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": rk.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": DISK["workload"], "N": ns.N,
                       "precision": "fp32 Gauss-Jordan inverse + double-fp32 refinement (fp64 fallback)",
                       "l2": "256 MiB buffer written between timed steps",
                       "step": "grid kNN + weights (2 classes) + 3 operator applications"},
            "fp64_plain": {"value": throughput(n_all, ms64, args.steps), "unit": "nodes/s",
                           "ms_per_step": ms64 / args.steps, "weights_ms": float(np.mean(w64)),
                           "dominant_ms": float(np.mean(d64)),
                           "roofline_frac": f64_plain / (float(np.mean(d64)) * 1e-3) / fp64_peak,
                           "roofline_note": "bench.method_flops x interior rows / dominant_ms / "
                                            "measured FP64 FMA peak"},
            "fp32_ir_wide64": {"value": throughput(n_all, msw, args.steps), "unit": "nodes/s",
                               "ms_per_step": msw / args.steps, "weights_ms": float(np.mean(ww)),
                               "dominant_ms": float(np.mean(dw)),
                               "note": "same form, refinement residuals in native FP64"},
            "fp64_equivalent": fp64_equiv,
            "speedup_vs_fp64_plain": ms64 / ms, "weights_ms": float(np.mean(wts)),
            "weights_only": {"value": n_all / (float(np.mean(wts)) * 1e-3), "unit": "nodes/s",
                             "fp64_plain": n_all / (float(np.mean(w64)) * 1e-3),
                             "note": "both classes' weights without the kNN and the operator "
                                     "applications (the headline value is kNN + weights + applications)"},
            "fallback_fraction": fallback, "roofline": roof, "roofline_spmv": spmv_roof,
            "roofline_knn": knn_roof,
            "roofline_combine": comb_roof,
            "peaks_measured": {"fp64_flops": fp64_peak, "fp32_flops": fp32_peak},
            "e2e": e2e, "clocks": clk, "gpu_launches": DISK_LAUNCHES_PER_STEP * args.steps}
    if rk.rank == 0 and not args.no_error:
        line["error"] = sampled_error(pipe)
    if rk.rank == 0 and not args.no_poisson:
        line["poisson"] = poisson_comparison(P, ctx, device)
    if rk.rank == 0 and rk.world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_disk(ns, rp, pipe.col.cpu().numpy())
    ctx.close()
    return line


# ------------------------------------------------------------ ball workload
BALL = {"workload": "unit ball, 4e6 nodes: interior n=35 r^3 deg 2, refined |x|<0.5 n=60 r^3 deg 3, "
                    "boundary n=45 d/dn; one persistent launch, autotuned tiles",
        "N_target": 4_000_000,
        "classes": [("interior", 35, 3, 2, 1 | 2 | 4 | 8), ("refined", 60, 3, 3, 1 | 2 | 4 | 8),
                    ("boundary", 45, 3, 2, 16)]}


def run_ball(args, rk):
    import torch

    import nodesets as NS
    import paper_1912_13282_gb300 as P
    device = rk.local
    stream = torch.cuda.current_stream(device)
    ctx = P.Context(device, stream)
    ns = NS.ball(args.n_target or BALL["N_target"], seed=rk.rank)
    sizes = np.zeros(ns.N, dtype=np.int64)
    for cname, n, *_ in BALL["classes"]:
        b, e = ns.classes[cname]
        sizes[b:e] = n
    rp = np.zeros(ns.N + 1, dtype=np.int64)
    np.cumsum(sizes, out=rp[1:])
    dv = f"cuda:{device}"
    pts, nrm = torch.from_numpy(ns.pts).to(dv), torch.from_numpy(ns.normals).to(dv)
    rp_d = torch.from_numpy(rp).to(dv)
    nnz = int(rp[-1])
    col = torch.empty(nnz, dtype=torch.int32, device=dv)
    vals = [torch.zeros(nnz, dtype=torch.float64, device=dv) for _ in range(4)]   # lap/dn, dx, dy, dz
    status = torch.empty(ns.N, dtype=torch.int32, device=dv)
    ranges = []
    classes = []
    for cname, n, k, m, ops in BALL["classes"]:
        b, e = ns.classes[cname]
        ranges.append((b, e, n, col[int(rp[b]):int(rp[e])]))
        vv = vals if ops != 16 else [vals[0]]
        classes.append(P.Context.weights_class(ops, k, m, pts, rp_d, col, vv, row_begin=b,
                                               row_end=e, n_max=n, normals=nrm, status=status))
    u = torch.from_numpy(NS.sin_product(ns.pts)).to(dv)
    y = torch.empty_like(u)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=dv)

    fixed = tuple(int(v) for v in args.batched_config.split(",")) if args.batched_config else None

    def weights(prec):
        ctx.rbffd_weights_batched(classes, precision=prec, config=fixed)

    def step(prec):
        ctx.knn_stencils(pts, ranges, method=P.KNN_GRID)
        weights(prec)
        for v in vals:
            ctx.apply_operator(rp_d, col, v, u, y)

    ctx.knn_stencils(pts, ranges, method=P.KNN_GRID)
    tuned = {}
    for name, prec in (("fp64", P.FP64), ("fp32_ir", P.FP32_IR)):
        if fixed:
            tuned[name] = {"warps_per_block": fixed[0], "blocks_per_sm": fixed[1], "chunk_rows": fixed[2],
                           "fixed": True}
            continue
        cfg, t = ctx.autotune_batched(classes, precision=prec, sample_rows=32768)
        tuned[name] = {"warps_per_block": cfg[0], "blocks_per_sm": cfg[1], "chunk_rows": cfg[2],
                       "sample_ms": t}
    for _ in range(max(3, args.warmup)):
        step(P.FP64)
        step(P.FP32_IR)
    torch.cuda.synchronize()
    res = {}
    clocks = ClockSampler(device)
    clocks.start()
    for name, prec in (("fp64", P.FP64), ("fp32_ir", P.FP32_IR)):
        rk.barrier()
        tt, ww = [], []
        for _ in range(args.steps):
            flush.add_(1.0)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            ctx.knn_stencils(pts, ranges, method=P.KNN_GRID)
            ev[1].record(stream)
            weights(prec)
            ev[2].record(stream)
            for v in vals:
                ctx.apply_operator(rp_d, col, v, u, y)
            ev[3].record(stream)
            ev[3].synchronize()
            tt.append(ev[0].elapsed_time(ev[3]))
            ww.append(ev[1].elapsed_time(ev[2]))
        (ms,) = rk.max([float(np.sum(tt))])
        (n_all,) = rk.sum([ns.N])
        res[name] = {"ms_per_step": ms / args.steps, "weights_ms": float(np.mean(ww)),
                     "value": throughput(n_all, ms, args.steps)}
    clk = clocks.stop()
    st = status.cpu().numpy()
    line = {"metric": METRIC, "value": res["fp32_ir"]["value"], "unit": "nodes/s",
            "n_gpus": rk.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["fp32_ir"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": BALL["workload"], "N": ns.N,
                       "classes": {c: ns.classes[c] for c, *_ in BALL["classes"]}},
            "fp64_plain": res["fp64"], "fp32_ir": res["fp32_ir"],
            "speedup_vs_fp64_plain": res["fp64"]["ms_per_step"] / res["fp32_ir"]["ms_per_step"],
            "fallback_fraction": float((st == P.binding.ST_FALLBACK).mean()),
            "autotuned": tuned, "clocks": clk,
            "gpu_launches": (11 + 2 + 4) * args.steps}
    if rk.rank == 0 and rk.world == 1 and not args.no_cpu_baseline:
        spans = [(ns.classes[c][0], ns.classes[c][1], n, k, m, ops) for c, n, k, m, ops in BALL["classes"]]
        line["cpu_baseline"] = cpu_baseline_classes(ns, rp, col.cpu().numpy(), spans)
    ctx.close()
    return line


# ----------------------------------------------------------- GWLS workload
WLS = {"workload": "GWLS weights (Section 2.2.1) on the disk minus 5 holes, 1e6 nodes: interior rows, "
                   "9 closest nodes, monomials of degree <= 2, Gaussian weight sigma = 1, closest-node "
                   "scale (the paper's GWLS example setup); lap, dx, dy",
       "N_target": 1_000_000, "n": 9, "m": 2, "sigma": 1.0, "ops": 1 | 2 | 4}


def wls_fp64_flops(n, l, R):
    """Algorithmic FP64 flops of one GWLS stencil: Householder QR of the n x l
    matrix W B (2 n l^2 - 2 l^3 / 3), R forward substitutions (l^2 each),
    R products with Q (4 n l - 2 l^2 each) and W B itself (n l)."""
    return 2 * n * l * l - 2 * l ** 3 / 3 + R * l * l + R * (4 * n * l - 2 * l * l) + n * l


def cpu_baseline_wls(ns, col_h, rp_h, rows, seconds=10.0):
    """oracle/wls.py (numpy, one stencil at a time) on a bounded sample."""
    from oracle import wls as Wo
    import time as _t
    t0 = _t.perf_counter()
    done = 0
    for i in rows:
        x = ns.pts[col_h[rp_h[i]:rp_h[i + 1]]]
        Wo.stencil_weights(x, WLS["m"], WLS["ops"], WLS["sigma"], Wo.SCALE_NEAREST)
        done += 1
        if _t.perf_counter() - t0 > seconds:
            break
    dt = _t.perf_counter() - t0
    return {"value": done / dt, "unit": "nodes/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} interior stencils of the same node set (numpy SVD pseudoinverse, one thread)"}


def run_wls(args, rk):
    import torch

    import nodesets as NS
    import paper_1912_13282_gb300 as P
    device = rk.local
    stream = torch.cuda.current_stream(device)
    ctx = P.Context(device, stream)
    ns = NS.disk_holes(args.n_target or WLS["N_target"], seed=rk.rank)
    b, e = ns.classes["interior"]
    n, m, R = WLS["n"], WLS["m"], 3
    rp = np.zeros(ns.N + 1, dtype=np.int64)
    rp[b + 1:e + 1] = np.arange(1, e - b + 1) * n
    rp[e + 1:] = rp[e]
    dv = f"cuda:{device}"
    pts = torch.from_numpy(ns.pts).to(dv)
    rp_d = torch.from_numpy(rp).to(dv)
    nnz = int(rp[-1])
    col = torch.empty(nnz, dtype=torch.int32, device=dv)
    vals = [torch.zeros(nnz, dtype=torch.float64, device=dv) for _ in range(R)]
    status = torch.empty(ns.N, dtype=torch.int32, device=dv)
    ranges = [(b, e, n, col)]
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=dv)
    fp64_peak = ctx.measure_fma_peak(0)

    def weights():
        ctx.wls_weights(WLS["ops"], m, WLS["sigma"], P.SCALE_NEAREST, pts, rp_d, col, vals, row_begin=b,
                        row_end=e, n_max=n, status=status)

    for _ in range(max(3, args.warmup)):
        ctx.knn_stencils(pts, ranges, method=P.KNN_GRID)
        weights()
    torch.cuda.synchronize()
    clocks = ClockSampler(device)
    clocks.start()
    rk.barrier()
    tt, ww = [], []
    for _ in range(args.steps):
        flush.add_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        ctx.knn_stencils(pts, ranges, method=P.KNN_GRID)
        ev[1].record(stream)
        weights()
        ev[2].record(stream)
        ev[2].synchronize()
        tt.append(ev[0].elapsed_time(ev[2]))
        ww.append(ev[1].elapsed_time(ev[2]))
    clk = clocks.stop()
    (ms,) = rk.max([float(np.sum(tt))])
    (msw,) = rk.max([float(np.sum(ww))])
    Ni = e - b
    (n_all,) = rk.sum([Ni])
    # end to end through the public calls: host points in, weights out (pinned)
    e2e = None
    if not args.no_e2e:
        h_pts = torch.from_numpy(ns.pts).pin_memory()
        h_out = [torch.empty(nnz, dtype=torch.float64).pin_memory() for _ in range(R)]
        e_ms = []
        for _ in range(args.steps):
            flush.add_(1.0)
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pts.copy_(h_pts, non_blocking=True)
            ctx.knn_stencils(pts, ranges, method=P.KNN_GRID)
            weights()
            for h, d in zip(h_out, vals):
                h.copy_(d, non_blocking=True)
            z.record(stream)
            z.synchronize()
            e_ms.append(a.elapsed_time(z))
        (e_tot,) = rk.max([float(np.sum(e_ms))])
        e2e = {"value": throughput(n_all, e_tot, args.steps), "unit": "nodes/s",
               "h2d_bytes_per_step": int(h_pts.numel() * 8), "d2h_bytes_per_step": int(nnz * 8 * R)}
    st = status.cpu().numpy()[b:e]
    l = 6
    flops = wls_fp64_flops(n, l, R) * Ni
    w_ms = msw / args.steps
    roof = {"bound": "alu", "kernel": "k_wls_thread<2> (FP64 Householder QR, one stencil per thread)",
            "achieved": flops / (w_ms * 1e-3) / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
            "frac": flops / (w_ms * 1e-3) / fp64_peak, "traffic": None,
            "algorithmic": "bench.wls_fp64_flops: %.0f FP64 flops per stencil" % wls_fp64_flops(n, l, R),
            "peak_source": "FP64 FMA peak measured in this run (mm_measure_fma_peak)"}
    line = {"metric": "GWLS stencil weights nodes/s", "value": throughput(n_all, msw, args.steps),
            "unit": "nodes/s", "n_gpus": rk.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": w_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WLS["workload"], "N": ns.N, "rows": Ni,
                       "l2": "256 MiB buffer written between timed steps"},
            "with_knn": {"value": throughput(n_all, ms, args.steps), "unit": "nodes/s",
                         "ms_per_step": ms / args.steps},
            "status_ok_fraction": float((st == 0).mean()), "roofline": roof, "e2e": e2e,
            "clocks": clk, "gpu_launches": 6 * args.steps}
    if rk.rank == 0 and rk.world == 1 and not args.no_cpu_baseline:
        rng = np.random.default_rng(0)
        sample = rng.choice(np.arange(b, e), 4000, replace=False)
        # the rows before b are empty, so col is indexed by the full row pointer
        line["cpu_baseline"] = cpu_baseline_wls(ns, col.cpu().numpy(), rp, sample)
    ctx.close()
    return line


# ----------------------------------------------------------- batch workload
def run_batch(args, rk):
    import torch

    import nodesets as NS
    import paper_1912_13282_gb300 as P
    device = rk.local
    dv = f"cuda:{device}"
    ctx = P.Context(device, torch.cuda.current_stream(device))
    scale = (args.n_target / 2.4e7) if args.n_target else 1.0
    specs = NS.batch_geometries(64, seed=rk.rank, scale=scale)
    params = {2: [(12, 3, 2), (25, 5, 4)], 3: [(35, 3, 2), (60, 3, 3)]}
    geoms = []
    t0 = time.time()
    for sp in specs:
        ns = NS.make_geometry(sp)
        n, k, m = params[sp["dim"]][sp["stencil_choice"]]
        rp = np.arange(ns.N + 1, dtype=np.int64) * n
        g = {"ns": ns, "n": n, "k": k, "m": m, "pts": torch.from_numpy(ns.pts).to(dv),
             "rp": torch.from_numpy(rp).to(dv), "col": torch.empty(ns.N * n, dtype=torch.int32, device=dv),
             "lap": torch.zeros(ns.N * n, dtype=torch.float64, device=dv),
             "fixed": torch.from_numpy(ns.normals.any(axis=1).astype(np.uint8)).to(dv),
             "u0": torch.from_numpy(NS.sin_product(ns.pts)).to(dv),
             "dt": 0.1 * ns.h ** 2}
        g["u"] = g["u0"].clone()
        g["work"] = torch.empty_like(g["u"])
        ctx.knn_stencils(g["pts"], [(0, ns.N, n, g["col"])], method=P.KNN_GRID)
        geoms.append(g)
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    N = sum(g["ns"].N for g in geoms)
    classes = [P.Context.weights_class(1, g["k"], g["m"], g["pts"], g["rp"], g["col"], [g["lap"]],
                                       n_max=g["n"]) for g in geoms]
    res = {}
    for name, prec in (("fp64", P.FP64), ("fp32_ir", P.FP32_IR)):
        ctx.autotune_batched(classes, precision=prec, sample_rows=8192)

        def run():
            ctx.rbffd_weights_batched(classes, precision=prec)
            for g in geoms:
                ctx.diffuse(g["rp"], g["col"], g["lap"], g["fixed"], g["dt"], 100, g["u"], g["work"])

        for g in geoms:
            g["u"].copy_(g["u0"])
        run()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(device)
        side.wait_stream(torch.cuda.current_stream(device))
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                ctx.set_stream(side)
                run()
        ctx.set_stream(torch.cuda.current_stream(device))
        torch.cuda.synchronize()
        for _ in range(max(1, args.warmup)):
            graph.replay()
        torch.cuda.synchronize()
        rk.barrier()
        times = []
        stream = torch.cuda.current_stream(device)
        for _ in range(args.steps):
            for g in geoms:
                g["u"].copy_(g["u0"])
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            graph.replay()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        (ms,) = rk.max([float(np.sum(times))])
        (n_all,) = rk.sum([N])
        res[name] = {"ms_per_step": ms / args.steps, "value": throughput(n_all, ms, args.steps)}
        del graph
    line = {"metric": METRIC, "value": res["fp32_ir"]["value"], "unit": "nodes/s",
            "n_gpus": rk.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["fp32_ir"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "64 2D/3D node sets, log-uniform 1e4..2e6 nodes, n in {12,25,35,60}: "
                                   "all Laplacian weights (one persistent launch) + 100 explicit "
                                   "diffusion steps each, one CUDA graph", "N_total": N,
                       "node_generation_s": gen_s},
            "fp64_plain": res["fp64"], "fp32_ir": res["fp32_ir"],
            "speedup_vs_fp64_plain": res["fp64"]["ms_per_step"] / res["fp32_ir"]["ms_per_step"]}
    ctx.close()
    return line


# ------------------------------------------------------- surrogate workload
def run_surrogate(args, rk):
    import torch

    import paper_1912_13282_gb300 as P
    from paper_1912_13282_gb300 import surrogate as S
    device = rk.local
    ctx = P.Context(device, torch.cuda.current_stream(device))
    n, k, m = 25, 5, 4
    ntrain = args.train_samples
    neval = args.n_target or 1_000_000
    t0 = time.time()
    data = S.make_dataset(ctx, ntrain, seed=1 + 1000 * rk.rank)
    torch.cuda.synchronize()
    t_data = time.time() - t0
    net = P.MLP(ctx, 2 * n, n, seed=rk.rank)
    t0 = time.time()
    losses = S.train(net, data["x"], data["t"], epochs=args.train_epochs, batch=args.train_batch, lr=3e-3,
                     lr_final=1e-4)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    del data
    pts, rp, col = S.make_stencils(ctx, neval, seed=10 ** 6 + rk.rank)
    vals = {nm: torch.zeros(neval * n, dtype=torch.float64, device="cuda")
            for nm in ("fp64", "ir", "sur", "surir")}
    status = torch.empty(neval, dtype=torch.int32, device="cuda")
    rho = torch.empty(neval, dtype=torch.float32, device="cuda")
    tau = 1e-3
    stream = torch.cuda.current_stream(device)

    def run(name):
        if name in ("sur", "surir"):
            P.rbffd_weights_surrogate(ctx, net, k, m, pts, rp, col, 0, neval, n, tau, vals[name],
                                      status, rho, fallback=P.FP64 if name == "sur" else P.FP32_IR)
        else:
            ctx.rbffd_weights(P.LAP, k, m, pts, rp, col, [vals[name]], row_end=neval, n_max=n,
                              precision=P.FP64 if name == "fp64" else P.FP32_IR)

    res = {}
    for name in ("fp64", "ir", "surir", "sur"):
        for _ in range(max(1, args.warmup)):
            run(name)
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run(name)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        (ms,) = rk.max([float(np.sum(ts))])
        (n_all,) = rk.sum([neval])
        res[name] = {"ms": ms / args.steps, "value": throughput(n_all, ms, args.steps)}
    st = status.cpu().numpy()
    acc = st == P.binding.ST_ACCEPTED
    w = vals["sur"].view(neval, n).cpu().numpy()
    r = vals["fp64"].view(neval, n).cpu().numpy()
    err = np.abs(w - r).max(1) / np.abs(r).max(1)
    # headline: the surrogate with the FP32+IR solve as fallback; the form
    # whose fallback is the plain FP64 solve is reported beside it
    line = {"metric": METRIC, "value": res["surir"]["value"], "unit": "nodes/s", "n_gpus": rk.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["surir"]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16+f32+f64", "data": "synthetic",
            "config": {"workload": f"surrogate: MLP 50-256x3-25 trained ({args.train_epochs} epochs) on {ntrain} jittered-patch "
                                   f"stencils, {neval} held-out stencils (n=25, r^5, deg 4)",
                       "tau": tau},
            "fp64_plain": res["fp64"], "fp32_ir": res["ir"], "surrogate_fp64_fallback": res["sur"],
            "surrogate_fp32ir_fallback": res["surir"],
            "speedup_vs_fp64_plain": res["fp64"]["ms"] / res["surir"]["ms"],
            "speedup_vs_fp32_ir": res["ir"]["ms"] / res["surir"]["ms"],
            "speedup_fp64_fallback_vs_fp64_plain": res["fp64"]["ms"] / res["sur"]["ms"],
            "accept_fraction": float(acc.mean()),
            "error_vs_fp64": {"accepted_median": float(np.median(err[acc])) if acc.any() else None,
                              "accepted_p99": float(np.quantile(err[acc], 0.99)) if acc.any() else None,
                              "fallback_max": float(err[~acc].max()) if (~acc).any() else None},
            "training": {"samples": ntrain, "steps": int(len(losses)), "seconds": t_train,
                         "data_seconds": t_data, "loss_first": float(losses[:20].mean()),
                         "loss_last": float(losses[-50:].mean()),
                         "samples_per_s": float(len(losses)) * args.train_batch / t_train,
                         "tflops": float(len(losses)) * args.train_batch * MLP_TRAIN_FLOPS_PER_SAMPLE / t_train / 1e12,
                         "gemms": "tcgen05 (BF16 operands, FP32 accumulators in tensor memory), batch %d"
                                  % args.train_batch}}
    if rk.rank == 0 and not args.no_poisson:
        line["poisson"] = surrogate_poisson(P, ctx, net, (1e-3, 3e-4, 1e-4, 3e-5))
    ctx.close()
    return line


# BF16 GEMM flops of one training sample (2 per multiply-add): forward
# 50(64 padded) -> 256 -> 256 -> 256 -> 25(32 padded), the backward data
# products of the three upper layers, and the four weight gradients
MLP_TRAIN_FLOPS_PER_SAMPLE = (2 * (64 * 256 + 2 * 256 * 256 + 256 * 32) + 2 * (32 * 256 + 2 * 256 * 256)
                              + 2 * (32 * 256 + 2 * 256 * 256 + 256 * 64))


def surrogate_poisson(P, ctx, net, taus, n_target=100_000, seed=7, reps=5):
    """The surrogate at equal Poisson solution error (Section 5's benchmark
    problem on the disk with holes): the interior Laplacian rows from the
    surrogate (FP32 + refinement fallback for rejected stencils) for each
    tau, the boundary d/dn rows from the FP32 + refinement solve, against
    the same rows from the plain FP64 and the FP32 + refinement solves; each
    weight set goes through the same host sparse direct solve (untimed).
    Also the interior rows' weight time of each form (mean of `reps`)."""
    import torch
    ns, rp = make_disk(seed, n_target)
    pipe = DiskPipeline(P, ctx, ns, rp, torch.cuda.current_device())
    pipe.knn()
    wi, wb = DISK["interior"], DISK["boundary"]
    stream = torch.cuda.current_stream()
    status = torch.empty(ns.N, dtype=torch.int32, device=pipe.pts.device)
    rho = torch.empty(ns.N, dtype=torch.float32, device=pipe.pts.device)

    def interior(form, tau=None):
        if form == "surrogate":
            P.rbffd_weights_surrogate(ctx, net, wi["k"], wi["m"], pipe.pts, pipe.rp, pipe.col, pipe.ib,
                                      pipe.ie, wi["n"], tau, pipe.op, status, rho, fallback=P.FP32_IR)
        else:
            ctx.rbffd_weights(P.LAP, wi["k"], wi["m"], pipe.pts, pipe.rp, pipe.col, [pipe.op],
                              row_begin=pipe.ib, row_end=pipe.ie, n_max=wi["n"],
                              precision=P.FP64 if form == "fp64" else P.FP32_IR, status=status)

    def timed(form, tau=None):
        interior(form, tau)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            interior(form, tau)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.mean(ts))

    col = pipe.col.cpu().numpy()
    out = {"N": ns.N, "interior_rows": pipe.ie - pipe.ib, "forms": {}}
    runs = [("fp64", None), ("fp32_ir", None)] + [("surrogate", t) for t in taus]
    for form, tau in runs:
        ms = timed(form, tau)
        ctx.rbffd_weights(wb["ops"], wb["k"], wb["m"], pipe.pts, pipe.rp, pipe.col, [pipe.op],
                          row_begin=pipe.bb, row_end=pipe.be, n_max=wb["n"], precision=P.FP32_IR,
                          normals=pipe.nrm)
        torch.cuda.synchronize()
        err = poisson_error(ns, rp, col, pipe.op.cpu().numpy())
        key = form if tau is None else f"surrogate_tau_{tau:g}"
        rec = {"poisson_max_error": err, "interior_weights_ms": ms}
        if form == "surrogate":
            st = status.cpu().numpy()[pipe.ib:pipe.ie]
            rec["tau"] = tau
            rec["accept_fraction"] = float((st == P.binding.ST_ACCEPTED).mean())
        out["forms"][key] = rec
    e64 = out["forms"]["fp64"]["poisson_max_error"]
    for rec in out["forms"].values():
        rec["relative_to_fp64"] = abs(rec["poisson_max_error"] - e64) / e64
        rec["equal_within_1pct"] = rec["relative_to_fp64"] <= 0.01
    ir_ms = out["forms"]["fp32_ir"]["interior_weights_ms"]
    for rec in out["forms"].values():
        rec["speedup_vs_fp32_ir"] = ir_ms / rec["interior_weights_ms"]
    ok = [r for k, r in out["forms"].items() if k.startswith("surrogate") and r["equal_within_1pct"]
          and r["speedup_vs_fp32_ir"] > 1.0]
    out["gain_at_equal_error"] = max((r["speedup_vs_fp32_ir"] for r in ok), default=None)
    return out


# ------------------------------------------------------------ unit square
SQUARE = {"workload": "unit square, h = 0.01 (10,201 nodes, jittered interior, Dirichlet edges): n=12 PHS r^3 + "
                      "deg-2 monomials, lap/dx/dy on every node; Poisson u = sin(pi x) sin(pi y) solved with the "
                      "GPU implicit solve",
          "h": 0.01, "n": 12, "k": 3, "m": 2, "ops": 1 | 2 | 4}


def run_square(args, rk):
    """The small configuration: whole step (kNN + weights of every node + 3
    operator applications) in FP64 and in the FP32 + refinement form, the
    weights' error against the oracle on every row, and the Dirichlet Poisson
    error of both weight sets through the GPU implicit solve."""
    import torch

    import nodesets as NS
    import paper_1912_13282_gb300 as P
    device = rk.local
    stream = torch.cuda.current_stream(device)
    ctx = P.Context(device, stream)
    ns = NS.square(SQUARE["h"], seed=rk.rank)
    n, k, m, ops = SQUARE["n"], SQUARE["k"], SQUARE["m"], SQUARE["ops"]
    N = ns.N
    dv = f"cuda:{device}"
    pts = torch.from_numpy(ns.pts).to(dv)
    rp_h = np.arange(N + 1, dtype=np.int64) * n
    rp = torch.from_numpy(rp_h).to(dv)
    col = torch.empty(N * n, dtype=torch.int32, device=dv)
    vals = [torch.zeros(N * n, dtype=torch.float64, device=dv) for _ in range(3)]
    u = torch.from_numpy(NS.sin_product(ns.pts)).to(dv)
    y = torch.empty_like(u)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=dv)

    def step(prec):
        ctx.knn_stencils(pts, [(0, N, n, col)], method=P.KNN_GRID)
        ctx.rbffd_weights(ops, k, m, pts, rp, col, vals, n_max=n, precision=prec)
        for v in vals:
            ctx.apply_operator(rp, col, v, u, y)

    for _ in range(max(3, args.warmup)):
        step(P.FP64)
        step(P.FP32_IR)
    torch.cuda.synchronize()
    clocks = ClockSampler(device)
    clocks.start()
    res = {}
    for name, prec in (("fp64", P.FP64), ("fp32_ir", P.FP32_IR)):
        rk.barrier()
        ts = []
        for _ in range(args.steps):
            flush.add_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(prec)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        (ms,) = rk.max([float(np.sum(ts))])
        (n_all,) = rk.sum([N])
        res[name] = {"ms_per_step": ms / args.steps, "value": throughput(n_all, ms, args.steps)}
    clk = clocks.stop()
    # accuracy: every row against the oracle, and the Poisson error of both weight sets
    out_err, poisson = {}, {}
    kind = torch.from_numpy(ns.dirichlet.astype(np.uint8)).to(dv)
    rhs = np.where(ns.dirichlet, NS.sin_product(ns.pts), NS.sin_product_lap(ns.pts))
    b = torch.from_numpy(rhs).to(dv)
    for name, prec in (("fp64", P.FP64), ("fp32_ir", P.FP32_IR)):
        step(prec)
        torch.cuda.synchronize()
        if rk.rank == 0 and not args.no_error:
            from oracle import oracle as O
            ref, st, _ = O.weights(ns.pts, rp_h, col.cpu().numpy(), k, m, ops, nthreads=O.nthreads_default())
            errs = []
            for r in range(3):
                g = vals[r].cpu().numpy().reshape(N, n)
                w = ref[r].reshape(N, n)
                errs.append(float((np.abs(g - w).max(1) / np.abs(w).max(1)).max()))
            out_err[name] = {"max_rel_err_lap_dx_dy": errs, "rows": N}
        cs, vs = torch.empty_like(col), torch.empty_like(vals[0])
        ctx.implicit_assemble(rp, col, vals[0], kind, cs, vs)
        f = torch.empty_like(vs)
        diag = torch.empty(N, dtype=torch.int64, device=dv)
        ctx.ilu0(rp, cs, vs, f, diag)
        x = torch.zeros(N, dtype=torch.float64, device=dv)
        rc, it, rr = ctx.bicgstab(rp, cs, vs, b, x, f, diag, tol=1e-12, maxit=5000)
        poisson[name] = {"max_error": float(np.abs(x.cpu().numpy() - NS.sin_product(ns.pts)).max()),
                         "bicgstab_iterations": it, "converged": rc == P.binding.MM_OK}
    poisson["relative_difference"] = abs(poisson["fp32_ir"]["max_error"] - poisson["fp64"]["max_error"]) / \
        poisson["fp64"]["max_error"]
    line = {"metric": METRIC, "value": res["fp64"]["value"], "unit": "nodes/s", "n_gpus": rk.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["fp64"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": SQUARE["workload"], "N": N,
                       "l2": "256 MiB buffer written between timed steps",
                       "note": "10^4 nodes: the step is launch-bound (16 launches)"},
            "fp64_plain": res["fp64"], "fp32_ir": res["fp32_ir"], "error": out_err, "poisson": poisson,
            "clocks": clk, "gpu_launches": 16 * args.steps * 2}
    if rk.rank == 0 and rk.world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_classes(ns, rp_h, col.cpu().numpy(), [(0, N, n, k, m, ops)])
    ctx.close()
    return line


# ------------------------------------------------------- implicit Poisson
POISSON = {"workload": "implicit Poisson solve (Section 2.3.2, the benchmark problem of Section 5) on the "
                       "disk minus 5 holes, 2e4 nodes: interior Laplacian rows n=25 r^5 deg 4, Dirichlet "
                       "outer circle, Neumann holes (n=30 d/dn), u = sin(pi x) sin(pi y); ILU(0)-preconditioned "
                       "BiCGSTAB to ||r|| <= 1e-10 ||b||",
           "N_target": 20_000, "tol": 1e-10}


def dependency_depth(rp, col, lower=True):
    """Longest dependency chain of a sorted CSR factor's triangular solve
    (host, for the report only)."""
    n = len(rp) - 1
    lev = np.zeros(n, dtype=np.int64)
    rng = range(n) if lower else range(n - 1, -1, -1)
    for i in rng:
        r = col[rp[i]:rp[i + 1]]
        r = r[r < i] if lower else r[r > i]
        lev[i] = 1 + (lev[r].max() if len(r) else 0)
    return int(lev.max())


def run_poisson(args, rk):
    import torch

    import nodesets as NS
    import paper_1912_13282_gb300 as P
    device = rk.local
    stream = torch.cuda.current_stream(device)
    ctx = P.Context(device, stream)
    ns, rp = make_disk(7 + rk.rank, args.n_target or POISSON["N_target"])
    pipe = DiskPipeline(P, ctx, ns, rp, device)
    kind = np.zeros(ns.N, dtype=np.uint8)
    kind[ns.dirichlet] = 1
    kind[ns.neumann] = 2
    u = NS.sin_product(ns.pts)
    rhs = NS.sin_product_lap(ns.pts)
    g = NS.sin_product_grad(ns.pts)
    rhs[kind == 1] = u[kind == 1]
    rhs[kind == 2] = (g[kind == 2] * ns.normals[kind == 2]).sum(1)
    dv = pipe.pts.device
    kd = torch.from_numpy(kind).to(dv)
    b = torch.from_numpy(rhs).to(dv)
    cs = torch.empty_like(pipe.col)
    vs = torch.empty_like(pipe.op)
    f = torch.empty_like(pipe.op)
    diag = torch.empty(ns.N, dtype=torch.int64, device=dv)
    x = torch.zeros(ns.N, dtype=torch.float64, device=dv)
    tmp = torch.empty_like(x)
    wi, wb = DISK["interior"], DISK["boundary"]

    def step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        ev[0].record(stream)
        pipe.knn()
        ctx.rbffd_weights(P.LAP, wi["k"], wi["m"], pipe.pts, pipe.rp, pipe.col, [pipe.op], row_begin=pipe.ib,
                          row_end=pipe.ie, n_max=wi["n"], precision=P.FP32_IR)
        pipe.weights_boundary(P.FP32_IR)
        ev[1].record(stream)
        ctx.implicit_assemble(pipe.rp, pipe.col, pipe.op, kd, cs, vs)
        ev[2].record(stream)
        ctx.ilu0(pipe.rp, cs, vs, f, diag)
        ev[3].record(stream)
        x.zero_()
        rc, it, res = ctx.bicgstab(pipe.rp, cs, vs, b, x, f, diag, tol=POISSON["tol"], maxit=20000)
        ev[4].record(stream)
        ev[4].synchronize()
        if rc != P.binding.MM_OK:
            raise RuntimeError(f"BiCGSTAB did not converge: rc={rc} it={it} res={res}")
        return [ev[0].elapsed_time(ev[4]), ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]),
                ev[2].elapsed_time(ev[3]), ev[3].elapsed_time(ev[4]), it, res]

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(device)
    clocks.start()
    rk.barrier()
    rows = [step() for _ in range(args.steps)]
    clk = clocks.stop()
    R = np.array(rows)
    (ms,) = rk.max([float(R[:, 0].sum())])
    (n_all,) = rk.sum([ns.N])
    iters = int(R[0, 5])
    # one preconditioner application (forward + back substitution), timed alone
    ts = []
    for _ in range(5):
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.ilu0_solve(pipe.rp, cs, f, diag, b, tmp)
        z.record(stream)
        z.synchronize()
        ts.append(a.elapsed_time(z))
    pair_ms = float(np.median(ts))
    cs_h = cs.cpu().numpy()
    depth_l = dependency_depth(rp, cs_h, True) if ns.N <= 300_000 else None
    depth_u = dependency_depth(rp, cs_h, False) if ns.N <= 300_000 else None
    nnz = int(rp[-1])
    tri_bytes = 12 * nnz + 8 * (ns.N + 1) + 8 * ns.N + 3 * 8 * ns.N   # factors + columns, row/diag ptrs, b, y, x
    hbm = peaks_file().get("hbm_gbs")
    err = float(np.abs(x.cpu().numpy() - u).max())
    line = {"metric": "implicit Poisson solve unknowns/s (kNN + weights + assembly + ILU(0) + BiCGSTAB)",
            "value": throughput(n_all, ms, args.steps), "unit": "unknowns/s", "n_gpus": rk.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": POISSON["workload"], "N": ns.N, "nnz": nnz, "tol": POISSON["tol"],
                       "l2": "working set ~10 MB (L2-resident between steps: the solve is latency-bound)"},
            "breakdown_ms": {"knn_and_weights": float(R[:, 1].mean()), "assemble": float(R[:, 2].mean()),
                             "ilu0": float(R[:, 3].mean()), "bicgstab": float(R[:, 4].mean())},
            "iterations": iters, "relative_residual": float(R[0, 6]),
            "ms_per_iteration": float(R[:, 4].mean()) / max(iters, 1),
            "preconditioner_apply_ms": pair_ms,
            "dependency_depth": {"lower": depth_l, "upper": depth_u,
                                 "us_per_level": (pair_ms * 1e3 / (depth_l + depth_u)) if depth_l else None},
            "roofline": {"bound": "latency", "kernel": "k_lower + k_upper (one preconditioner application)",
                         "achieved": tri_bytes / (pair_ms * 1e-3) / 1e9, "unit": "GB/s", "peak": hbm,
                         "frac": (tri_bytes / (pair_ms * 1e-3) / 1e9 / hbm) if hbm else None,
                         "traffic": None,
                         "note": "sync-free substitutions: time ~ dependency depth x one L2 round trip, "
                                 "not bandwidth"},
            "poisson_max_error": err, "clocks": clk,
            "gpu_launches": (13 + 3 + 3 + 2 + 2 + 10 * iters) * args.steps}
    ctx.close()
    return line


# ------------------------------------------------------- balanced stencils
BALANCED = {"workload": "disk minus 5 holes, 1e6 nodes, balanced stencils (FindBalancedSupport reading: "
                        "per-quadrant quota among the K closest, then the closest of the rest): interior "
                        "n=25 of K=48, boundary n=30 of K=60; FP32 + refinement weights and 3 operator "
                        "applications as in the default workload",
            "K": {"interior": 48, "boundary": 60}}


def run_balanced(args, rk):
    """The default disk step with balanced stencils in place of plain kNN:
    the selection alone and against plain kNN, the whole step, and sampled
    rows against the oracle (bit for bit)."""
    import torch
    import paper_1912_13282_gb300 as P
    from oracle import oracle as O
    device = rk.local
    stream = torch.cuda.current_stream(device)
    ctx = P.Context(device, stream)
    ns, rp = make_disk(rk.rank, args.n_target or DISK["N_target"])
    pipe = DiskPipeline(P, ctx, ns, rp, device)
    ni, nb = DISK["interior"]["n"], DISK["boundary"]["n"]
    Ki, Kb = BALANCED["K"]["interior"], BALANCED["K"]["boundary"]
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=pipe.pts.device)

    def balanced():
        ctx.balanced_stencils(pipe.pts, [pipe.ranges[0]], Ki, method=P.KNN_GRID)
        ctx.balanced_stencils(pipe.pts, [pipe.ranges[1]], Kb, method=P.KNN_GRID)

    def timed(fn):
        flush.add_(1.0)
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        z.record(stream)
        z.synchronize()
        return a.elapsed_time(z)

    def step():
        balanced()
        pipe.weights_interior(P.FP32_IR)
        pipe.weights_boundary(P.FP32_IR)
        pipe.apply()

    for _ in range(max(3, args.warmup)):
        step()
        pipe.knn()
    torch.cuda.synchronize()
    clocks = ClockSampler(device)
    clocks.start()
    rk.barrier()
    sel = [timed(balanced) for _ in range(args.steps)]
    knn = [timed(pipe.knn) for _ in range(args.steps)]
    tt = [timed(step) for _ in range(args.steps)]
    clk = clocks.stop()
    (ms,) = rk.max([float(np.sum(tt))])
    (n_all,) = rk.sum([ns.N])
    # the last step's rows: a sample against the oracle's balanced selection
    balanced()
    torch.cuda.synchronize()
    col = pipe.col.cpu().numpy()
    rng = np.random.default_rng(3)
    checked, same = 0, True
    for (b, e, n, _), K in ((pipe.ranges[0], Ki), (pipe.ranges[1], Kb)):
        q = np.sort(rng.choice(np.arange(b, e), min(e - b, 400), replace=False))
        ref, _ = O.balanced(ns.pts, n, K, queries=q, nthreads=O.nthreads_default())
        got = np.stack([col[rp[i]:rp[i + 1]] for i in q])
        same &= bool(np.array_equal(got, ref))
        checked += len(q)
    st = pipe.status.cpu().numpy()
    line = {"metric": METRIC + " (balanced stencils)", "value": throughput(n_all, ms, args.steps),
            "unit": "nodes/s", "n_gpus": rk.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": BALANCED["workload"], "N": ns.N,
                       "l2": "256 MiB buffer written before every timed launch",
                       "step": "balanced stencils + weights (2 classes) + 3 operator applications"},
            "selection_ms": float(np.mean(sel)), "plain_knn_ms": float(np.mean(knn)),
            "selection_nodes_per_s": ns.N / (float(np.mean(sel)) * 1e-3),
            "rows_checked_against_oracle": checked, "rows_equal": same,
            "fallback_fraction": float((st == P.binding.ST_FALLBACK).mean()),
            "clocks": clk}
    ctx.close()
    return line


# ----------------------------------------------- 3D convection-diffusion
CONVDIFF = {"workload": "implicit 3D convection-diffusion (Section 3.3 example), -2 lap u + 8 (2, 1, -1) . "
                        "grad u = f on the unit ball, Dirichlet sphere, u = sin(pi x) sin(pi y) sin(pi z) "
                        "manufactured: n=35 r^3 deg 2 stencils, lap/dx/dy/dz weights (FP32 + refinement) "
                        "combined by eq. gen-op, identity Dirichlet rows, ILU(0) + BiCGSTAB to 1e-10",
            "N_target": 50_000, "n": 35, "k": 3, "m": 2, "coef": (-2.0, 16.0, 8.0, -8.0), "tol": 1e-10}


def run_convdiff(args, rk):
    import torch

    import nodesets as NS
    import paper_1912_13282_gb300 as P
    device = rk.local
    stream = torch.cuda.current_stream(device)
    ctx = P.Context(device, stream)
    ns = NS.ball(args.n_target or CONVDIFF["N_target"], seed=rk.rank)
    N, n = ns.N, CONVDIFF["n"]
    nb = ns.classes["boundary"][0]
    dv = f"cuda:{device}"
    pts = torch.from_numpy(ns.pts).to(dv)
    rp = torch.arange(N + 1, dtype=torch.int64, device=dv) * n
    col = torch.empty(N * n, dtype=torch.int32, device=dv)
    terms = [torch.zeros(N * n, dtype=torch.float64, device=dv) for _ in range(4)]
    coefs = [torch.full((N,), c, dtype=torch.float64, device=dv) for c in CONVDIFF["coef"]]
    L = torch.zeros(N * n, dtype=torch.float64, device=dv)
    kind = torch.from_numpy(ns.dirichlet.astype(np.uint8)).to(dv)
    cs, vs = torch.empty_like(col), torch.empty_like(L)
    fac = torch.empty_like(vs)
    diag = torch.empty(N, dtype=torch.int64, device=dv)
    x = torch.zeros(N, dtype=torch.float64, device=dv)
    u = NS.sin_product(ns.pts)
    g = NS.sin_product_grad(ns.pts)
    c0, c1, c2, c3 = CONVDIFF["coef"]
    f = c0 * NS.sin_product_lap(ns.pts) + c1 * g[:, 0] + c2 * g[:, 1] + c3 * g[:, 2]
    b = torch.from_numpy(np.where(ns.dirichlet, u, f)).to(dv)

    def step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        ctx.knn_stencils(pts, [(0, N, n, col)], method=P.KNN_GRID)
        ctx.rbffd_weights(P.LAP | P.DX | P.DY | P.DZ, CONVDIFF["k"], CONVDIFF["m"], pts, rp, col, terms,
                          row_begin=0, row_end=nb, n_max=n, precision=P.FP32_IR)
        ctx.combine_operators(rp, col, terms, coefs, L, row_begin=0, row_end=nb)
        ev[1].record(stream)
        ctx.implicit_assemble(rp, col, L, kind, cs, vs)
        ctx.ilu0(rp, cs, vs, fac, diag)
        ev[2].record(stream)
        x.zero_()
        rc, it, res = ctx.bicgstab(rp, cs, vs, b, x, fac, diag, tol=CONVDIFF["tol"], maxit=20000)
        ev[3].record(stream)
        ev[3].synchronize()
        if rc != P.binding.MM_OK:
            raise RuntimeError(f"BiCGSTAB did not converge: rc={rc} it={it} res={res}")
        return [ev[0].elapsed_time(ev[3]), ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]),
                ev[2].elapsed_time(ev[3]), it, res]

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(device)
    clocks.start()
    rk.barrier()
    rows = [step() for _ in range(args.steps)]
    clk = clocks.stop()
    R = np.array(rows)
    (ms,) = rk.max([float(R[:, 0].sum())])
    (n_all,) = rk.sum([N])
    iters = int(R[0, 4])
    line = {"metric": "implicit 3D convection-diffusion unknowns/s (kNN + weights + combination + assembly "
                      "+ ILU(0) + BiCGSTAB)",
            "value": throughput(n_all, ms, args.steps), "unit": "unknowns/s", "n_gpus": rk.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": CONVDIFF["workload"], "N": N, "h": ns.h},
            "breakdown_ms": {"knn_weights_combination": float(R[:, 1].mean()),
                             "assemble_and_ilu0": float(R[:, 2].mean()), "bicgstab": float(R[:, 3].mean())},
            "iterations": iters, "relative_residual": float(R[0, 5]),
            "ms_per_iteration": float(R[:, 3].mean()) / max(iters, 1),
            "max_error": float(np.abs(x.cpu().numpy() - u).max()), "clocks": clk}
    ctx.close()
    return line


# ------------------------------------------------------------ reference arm
def run_reference(args):
    """The CPU oracle as the reference arm: each step a bounded sample of
    the disk workload (exhaustive kNN + FP64 weights of 256 interior nodes)
    on all host cores; rank 0 only."""
    rk_rank = int(os.environ.get("RANK", "0"))
    if rk_rank != 0:
        return 0
    from oracle import oracle as O
    ns, rp = make_disk(0, args.n_target or DISK["N_target"])
    threads = O.nthreads_default()
    rng = np.random.default_rng(1)
    vals = []
    (ib, ie) = ns.classes["interior"]
    for _ in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        qi = np.sort(rng.choice(np.arange(ib, ie), 256, replace=False))
        idx, _ = O.knn(ns.pts, 25, queries=qi, nthreads=threads)
        order = np.concatenate([qi, np.setdiff1d(np.unique(idx), qi)])
        remap = np.full(ns.N, -1, dtype=np.int64)
        remap[order] = np.arange(len(order))
        lcol = remap[idx].astype(np.int32).ravel()
        lrp = np.arange(len(qi) + 1, dtype=np.int64) * 25
        O.weights(ns.pts[order], lrp, lcol, 5, 4, 7, rows=(0, len(qi)), nthreads=threads)
        vals.append(len(qi) / (time.perf_counter() - t0))
    v = float(np.median(vals[args.warmup:]))
    line = {"metric": METRIC, "value": v, "unit": "nodes/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 256 / v * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": DISK["workload"],
                       "sample_per_step": "256 interior nodes: exhaustive kNN + FP64 weights (lap, dx, dy)"},
            "cpu_baseline": {"value": v, "unit": "nodes/s", "cores": threads, "kind": "oracle",
                             "sample": "256 interior nodes per step"},
            "e2e": {"value": v, "unit": "nodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- main
def main(argv=None):
    args = parse(argv)
    if args.impl == "reference":
        return run_reference(args)
    import torch
    rk = Ranks("nccl")
    torch.cuda.set_device(rk.local)
    from paper_1912_13282_gb300 import _build
    if rk.local == 0:
        _build.build()
    rk.barrier()
    run = {"disk": run_disk, "ball": run_ball, "batch": run_batch, "surrogate": run_surrogate,
           "wls": run_wls, "poisson": run_poisson, "square": run_square, "balanced": run_balanced,
           "convdiff": run_convdiff}[args.workload]
    line = run(args, rk)
    if rk.rank == 0:
        print(json.dumps(line), flush=True)
    rk.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
