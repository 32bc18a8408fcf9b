"""Benchmark: RBF-FD stencil-weight throughput (nodes/s) on the 1,000,000-node
2D disk-with-5-holes workload (interior: 25 nearest nodes, r^5 + degree-4
monomials, Laplacian and gradient; boundary: 30 nearest nodes, d/dn).

One step = the whole hot path over the node set: grid binning + kNN stencils
(two classes), weights for both classes in the chosen precision (FP32 LU with
FP64 refinement, FP64 fallback), and one application of each assembled
operator to a field.  The plain FP64 GPU path is timed the same way beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).  Under torchrun each rank runs its own
independent node set (seed = rank): weak scaling, no data-path collective.
"""
from __future__ import annotations

import argparse
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

WORKLOAD = {
    "workload": "disk minus 5 holes, 1e6 nodes: interior n=25 PHS r^5 + deg-4 monomials "
                "(lap, dx, dy); boundary n=30 d/dn",
    "N_target": 1_000_000,
    "interior": {"n": 25, "k": 5, "m": 4, "ops": ["lap", "dx", "dy"]},
    "boundary": {"n": 30, "k": 5, "m": 4, "ops": ["dn"]},
}
METRIC = "stencil weights nodes/s at stated error vs FP64 oracle; chosen form vs plain FP64 GPU"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-target", type=int, default=WORKLOAD["N_target"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-error", action="store_true")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons in the background."""

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


# ---------------------------------------------------------------- workload
def make_workload(seed: int, n_target: int):
    import nodesets as NS
    ns = NS.disk_holes(n_target, seed=seed)
    (ib, ie), (bb, be) = ns.classes["interior"], ns.classes["boundary"]
    ni, nb = WORKLOAD["interior"]["n"], WORKLOAD["boundary"]["n"]
    sizes = np.concatenate([np.full(ie - ib, ni), np.full(be - bb, nb)])
    rp = np.zeros(ns.N + 1, dtype=np.int64)
    np.cumsum(sizes, out=rp[1:])
    return ns, rp


class Pipeline:
    """Device buffers and the calls of one step."""

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
        self.op = torch.zeros(self.nnz, dtype=torch.float64, device=dv)   # lap rows + dn rows
        self.dx = torch.zeros(self.nnz, dtype=torch.float64, device=dv)
        self.dy = torch.zeros(self.nnz, dtype=torch.float64, device=dv)
        self.status = torch.empty(self.N, dtype=torch.int32, device=dv)
        self.u = torch.from_numpy(np.sin(np.pi * ns.pts[:, 0]) * np.sin(np.pi * ns.pts[:, 1])).to(dv)
        self.y = torch.empty(self.N, dtype=torch.float64, device=dv)
        self.gy = torch.empty(self.N, dtype=torch.float64, device=dv)
        ni = WORKLOAD["interior"]["n"]
        nb = WORKLOAD["boundary"]["n"]
        self.ranges = [(self.ib, self.ie, ni, self.col[: (self.ie - self.ib) * ni]),
                       (self.bb, self.be, nb, self.col[int(rp[self.bb]):])]

    def knn(self):
        self.ctx.knn_stencils(self.pts, self.ranges, method=self.P.KNN_GRID)

    def weights(self, precision):
        P, W = self.P, WORKLOAD
        wi, wb = W["interior"], W["boundary"]
        self.ctx.rbffd_weights(P.LAP | P.DX | P.DY, wi["k"], wi["m"], self.pts, self.rp, self.col,
                               [self.op, self.dx, self.dy], row_begin=self.ib, row_end=self.ie,
                               n_max=wi["n"], precision=precision, normals=self.nrm,
                               status=self.status)
        self.ctx.rbffd_weights(P.DN, wb["k"], wb["m"], self.pts, self.rp, self.col, [self.op],
                               row_begin=self.bb, row_end=self.be, n_max=wb["n"],
                               precision=precision, normals=self.nrm, status=self.status)

    def apply(self):
        self.ctx.apply_operator(self.rp, self.col, self.op, self.u, self.y)
        self.ctx.apply_operator(self.rp, self.col, self.dx, self.u, self.gy)
        self.ctx.apply_operator(self.rp, self.col, self.dy, self.u, self.gy, beta=1.0)

    def step(self, precision):
        self.knn()
        self.weights(precision)
        self.apply()

    launches_per_step = 9 + 2 + 2 * 2 + 3   # kNN build + 2 queries, 2 classes x (solve + fallback), 3 SpMV


def flush_l2(buf):
    buf.add_(1.0)


def time_steps(pipe, precision, steps, stream, flush, sub=None):
    """CUDA-event time of each step (L2 flushed between steps); optional
    sub-timing of the weights call."""
    import torch
    tot, wts = [], []
    for _ in range(steps):
        flush_l2(flush)
        e0, e1, e2, e3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        e0.record(stream)
        pipe.knn()
        e1.record(stream)
        pipe.weights(precision)
        e2.record(stream)
        pipe.apply()
        e3.record(stream)
        e3.synchronize()
        tot.append(e0.elapsed_time(e3))
        wts.append(e1.elapsed_time(e2))
    return np.array(tot), np.array(wts)


def sampled_error(pipe, rows_per_class=200, seed=0):
    """Max relative weight error (per node and operator) and monomial
    reproduction residual on sampled rows, against the oracle."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle import oracle as O
    from _helpers import monomial_residual, rel_err_rows
    ns = pipe.ns
    rp = pipe.rp_h
    col = pipe.col.cpu().numpy()
    got = {"lap": pipe.op.cpu().numpy(), "dx": pipe.dx.cpu().numpy(),
           "dy": pipe.dy.cpu().numpy(), "dn": pipe.op.cpu().numpy()}
    rng = np.random.default_rng(seed)
    out = {}
    for (b, e), spec, names in (((pipe.ib, pipe.ie), WORKLOAD["interior"], ["lap", "dx", "dy"]),
                                ((pipe.bb, pipe.be), WORKLOAD["boundary"], ["dn"])):
        rows = np.sort(rng.choice(np.arange(b, e), min(rows_per_class, e - b), replace=False))
        # oracle on a local renumbering: rows first
        sts = [col[rp[i]:rp[i + 1]] for i in rows]
        others = np.setdiff1d(np.unique(np.concatenate(sts)), rows)
        order = np.concatenate([rows, others])
        remap = np.full(ns.N, -1, dtype=np.int64)
        remap[order] = np.arange(len(order))
        lcol = np.concatenate([remap[s] for s in sts]).astype(np.int32)
        lrp = np.zeros(len(rows) + 1, dtype=np.int64)
        np.cumsum([len(s) for s in sts], out=lrp[1:])
        ops = sum({"lap": 1, "dx": 2, "dy": 4, "dn": 16}[nm] for nm in names)
        vals, st, _ = O.weights(ns.pts[order], lrp, lcol, spec["k"], spec["m"], ops,
                                normals=ns.normals[order], rows=(0, len(rows)), nthreads=8)
        for oi, nm in enumerate(names):
            w_ref = np.zeros_like(got[nm])
            for t, i in enumerate(rows):
                w_ref[rp[i]:rp[i + 1]] = vals[oi, lrp[t]:lrp[t + 1]]
            err = rel_err_rows(got[nm], w_ref, rp, rows)
            mono = monomial_residual(ns.pts, ns.normals, rp, col, got[nm], nm, spec["m"], rows)
            out[nm] = {"max_rel_err": float(err.max()), "median_rel_err": float(np.median(err)),
                       "monomial_residual": float(mono), "rows": int(len(rows))}
    return out


# ----------------------------------------------------------- CPU baseline
def cpu_baseline(ns, rp, col_h, seconds=15.0, seed=0):
    """The oracle timed on the host cores on a bounded sample of the same
    workload: brute-force kNN for S_k queries and weights for S_w rows, all
    cores.  Returns nodes/s of kNN + weights per node."""
    from oracle import oracle as O
    threads = O.nthreads_default()
    rng = np.random.default_rng(seed)
    (ib, ie), (bb, be) = ns.classes["interior"], ns.classes["boundary"]
    frac_b = (be - bb) / ns.N
    # kNN: calibrate on a few queries, then size the sample to ~1/3 of the budget
    q = rng.choice(np.arange(ib, ie), 64, replace=False)
    t0 = time.perf_counter()
    O.knn(ns.pts, 25, queries=q, nthreads=threads)
    per = (time.perf_counter() - t0) / 64
    sk = int(max(64, min(20000, seconds / 3 / max(per, 1e-9))))
    qi = rng.choice(np.arange(ib, ie), sk, replace=False)
    t0 = time.perf_counter()
    O.knn(ns.pts, 25, queries=qi, nthreads=threads)
    t_knn = (time.perf_counter() - t0) / sk
    # weights: interior rows and boundary rows in their proportion
    sw = 20000
    t_w = 0.0
    for (b, e), n, ops, share in (((ib, ie), 25, 1 | 2 | 4, 1 - frac_b), ((bb, be), 30, 16, frac_b)):
        rows = np.sort(rng.choice(np.arange(b, e), max(1, int(sw * share)), replace=False))
        sts = [col_h[rp[i]:rp[i + 1]] for i in rows]
        others = np.setdiff1d(np.unique(np.concatenate(sts)), rows)
        order = np.concatenate([rows, others])
        remap = np.full(ns.N, -1, dtype=np.int64)
        remap[order] = np.arange(len(order))
        lcol = np.concatenate([remap[s] for s in sts]).astype(np.int32)
        lrp = np.arange(len(rows) + 1, dtype=np.int64) * n
        t0 = time.perf_counter()
        O.weights(ns.pts[order], lrp, lcol, 5, 4, ops, normals=ns.normals[order],
                  rows=(0, len(rows)), nthreads=threads)
        t_w += (time.perf_counter() - t0) / len(rows) * share
    return {"value": 1.0 / (t_knn + t_w), "unit": "nodes/s", "cores": threads, "kind": "oracle",
            "sample": f"{sk} brute-force kNN queries over all {ns.N} nodes + {sw} weight rows "
                      f"(interior/boundary in proportion), all host cores",
            "knn_s_per_node": t_knn, "weights_s_per_node": t_w}


# ------------------------------------------------------------ reference arm
def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    ns, rp = make_workload(0, args.n_target)
    # stencils for the weight sample come from the oracle itself (exhaustive kNN)
    from oracle import oracle as O
    threads = O.nthreads_default()
    rng = np.random.default_rng(1)
    vals = []
    for _ in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        (ib, ie), (bb, be) = ns.classes["interior"], ns.classes["boundary"]
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
            "config": {"workload": WORKLOAD["workload"], "sample_per_step": "256 interior nodes: "
                       "exhaustive kNN + FP64 weights (lap, dx, dy)"},
            "cpu_baseline": {"value": v, "unit": "nodes/s", "cores": threads, "kind": "oracle",
                             "sample": "256 interior nodes per step"},
            "e2e": {"value": v, "unit": "nodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- main
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    rank, world, local = dist_info()
    device = local
    torch.cuda.set_device(device)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{device}"))
    from paper_1912_13282_gb300 import _build
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    import paper_1912_13282_gb300 as P
    stream = torch.cuda.current_stream(device)
    ctx = P.Context(device, stream)
    ns, rp = make_workload(rank, args.n_target)
    pipe = Pipeline(P, ctx, ns, rp, device)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=f"cuda:{device}")
    peaks = {"fp64_flops": ctx.measure_fma_peak(0), "fp32_flops": ctx.measure_fma_peak(1)}

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up (also grows the library workspace before timing)
    for _ in range(max(3, args.warmup)):
        pipe.step(P.FP64)
        pipe.step(P.FP32_IR)
    torch.cuda.synchronize()

    clocks = ClockSampler(device)
    clocks.start()
    barrier()
    tot64, w64 = time_steps(pipe, P.FP64, args.steps, stream, flush)
    barrier()
    tot, wts = time_steps(pipe, P.FP32_IR, args.steps, stream, flush)
    barrier()
    clk = clocks.stop()
    ms = float(tot.sum())
    if world > 1:
        t = torch.tensor([ms, float(tot64.sum())], device=f"cuda:{device}")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, ms64 = float(t[0]), float(t[1])
    else:
        ms64 = float(tot64.sum())
    status = pipe.status.cpu().numpy()
    fallback = float((status == P.binding.ST_FALLBACK).mean())
    value = world * ns.N * args.steps / (ms * 1e-3)

    # end to end: host (pinned) inputs in, weights out, inside the timed region
    e2e = None
    if not args.no_e2e:
        h_pts = torch.from_numpy(ns.pts).pin_memory()
        h_nrm = torch.from_numpy(ns.normals).pin_memory()
        h_out = [torch.empty(pipe.nnz, dtype=torch.float64).pin_memory() for _ in range(3)]
        e_ms = []
        for it in range(args.steps):
            flush_l2(flush)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pipe.pts.copy_(h_pts, non_blocking=True)
            pipe.nrm.copy_(h_nrm, non_blocking=True)
            pipe.step(P.FP32_IR)
            for h, d in zip(h_out, (pipe.op, pipe.dx, pipe.dy)):
                h.copy_(d, non_blocking=True)
            b.record(stream)
            b.synchronize()
            e_ms.append(a.elapsed_time(b))
        e2e = {"value": world * ns.N / (float(np.mean(e_ms)) * 1e-3), "unit": "nodes/s",
               "h2d_bytes_per_step": int(h_pts.numel() * 8 + h_nrm.numel() * 8),
               "d2h_bytes_per_step": int(sum(h.numel() * 8 for h in h_out))}

    # roofline of the dominant kernel (the refined-FP32 weights solve)
    M_i = 25 + 15
    M_b = 30 + 15
    Ni, Nb = pipe.ie - pipe.ib, pipe.be - pipe.bb
    # algorithmic FP64 work of the mixed path: one full residual and one
    # constraint-row residual per stencil (2 flop per multiply-add)
    f64 = Ni * (2 * 3 * (25 * M_i + 15 * 25) + 2 * 3 * 25 * 15) + \
        Nb * (2 * 1 * (30 * M_b + 15 * 30) + 2 * 1 * 30 * 15)
    w_ms = float(np.mean(wts))
    achieved = f64 / (w_ms * 1e-3)
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peaks["fp64_flops"] / 1e12,
            "unit": "TFLOP/s", "frac": achieved / peaks["fp64_flops"], "traffic": None,
            "kernel": "k_weights_mixed (FP64 residual flops)",
            "peak_source": "measured FP64 FMA loop on this GPU (mm_measure_fma_peak)"}

    err = None
    if not args.no_error and rank == 0:
        err = sampled_error(pipe)
    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        cpu = cpu_baseline(ns, rp, pipe.col.cpu().numpy())

    line = {"metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD["workload"], "N": ns.N, "precision": "fp32 LU + fp64 IR",
                       "l2": "256 MiB buffer written between timed steps",
                       "step": "grid kNN + weights (2 classes) + 3 operator applications"},
            "fp64_plain": {"value": world * ns.N * args.steps / (ms64 * 1e-3), "unit": "nodes/s",
                           "ms_per_step": ms64 / args.steps,
                           "weights_ms": float(np.mean(w64))},
            "speedup_vs_fp64_plain": ms64 / ms,
            "weights_ms": w_ms, "fallback_fraction": fallback,
            "error": err, "roofline": roof, "peaks_measured": peaks, "cpu_baseline": cpu,
            "e2e": e2e, "clocks": clk, "gpu_launches": Pipeline.launches_per_step * args.steps}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
