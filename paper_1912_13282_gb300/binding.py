"""Thin ctypes binding of libmm (include/mm.h).

Only argument marshalling lives here: torch tensors are used for device
memory and streams, every step of the pipeline runs in libmm's kernels.  If
libmm.so has not been built (``paper_1912_13282_gb300._build.build()``) the
first call raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import _build

MM_OK, MM_EBADARG, MM_ENOMEM, MM_ECUDA, MM_EUNSUPPORTED, MM_ENOCONV, MM_ESINGULAR = 0, -1, -2, -3, -4, -5, -6
ST_OK, ST_SINGULAR, ST_NONCONVERGED, ST_FALLBACK, ST_BADARG, ST_DUPLICATE, ST_ACCEPTED = range(7)
LAP, DX, DY, DZ, DN = 1, 2, 4, 8, 16
DXX, DXY, DYY, DXZ, DYZ, DZZ = 32, 64, 128, 256, 512, 1024
FP64, FP32_IR = 0, 1
KNN_AUTO, KNN_BRUTE, KNN_GRID = 0, 1, 2
OPT_IR_TOL, OPT_IR_MAX_STEPS, OPT_KAPPA_MAX, OPT_WIDE, OPT_MLP_INFER, OPT_GJ = 1, 2, 3, 4, 5, 6
WIDE_FF, WIDE_FP64 = 0, 1
MLP_FUSED, MLP_LAYERED = 0, 1
GJ_AUTO, GJ_SHARED = 0, 1
SCALE_FARTHEST, SCALE_NEAREST = 0, 1
ROW_INTERNAL, ROW_DIRICHLET, ROW_NEUMANN = 0, 1, 2

EXPORTS = ["mm_ctx_create", "mm_ctx_destroy", "mm_ctx_set_stream", "mm_ctx_set_option",
           "mm_last_error", "mm_ctx_workspace_bytes", "mm_knn_stencils", "mm_rbffd_weights", "mm_apply_operator",
           "mm_diffuse", "mm_measure_fma_peak", "mm_rbffd_weights_ir_noalloc",
           "mm_rbffd_weights_batched", "mm_autotune_batched", "mm_tile_table_save",
           "mm_tile_table_load", "mm_mlp_create", "mm_mlp_destroy", "mm_mlp_num_params",
           "mm_mlp_set_params", "mm_mlp_get_params", "mm_mlp_set_output_scaling",
           "mm_mlp_forward", "mm_mlp_train_step", "mm_mlp_grad", "mm_mlp_save", "mm_mlp_load",
           "mm_stencil_features", "mm_rbffd_weights_surrogate", "mm_wls_weights", "mm_diffuse_bc",
           "mm_combine_operators", "mm_implicit_assemble", "mm_ilu0", "mm_ilu0_solve", "mm_bicgstab",
           "mm_partition_morton", "mm_partition_halo", "mm_balanced_stencils",
           "mm_mlp_fit_output_scaling", "mm_surrogate_targets"]


class KnnRange(C.Structure):
    _fields_ = [("q_begin", C.c_int64), ("q_end", C.c_int64), ("n", C.c_int32),
                ("d_idx", C.c_void_p)]


class CsrPattern(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("nnz", C.c_int64), ("d_row_ptr", C.c_void_p),
                ("d_col", C.c_void_p)]


class WeightsClass(C.Structure):
    _fields_ = [("ops", C.c_uint), ("k", C.c_int), ("m", C.c_int), ("dim", C.c_int),
                ("N", C.c_int64), ("d_pts", C.c_void_p), ("d_normals", C.c_void_p),
                ("stencils", CsrPattern), ("row_begin", C.c_int64), ("row_end", C.c_int64),
                ("n_max", C.c_int), ("d_vals", C.c_void_p * 5), ("d_status", C.c_void_p)]


class LaunchConfig(C.Structure):
    _fields_ = [("warps_per_block", C.c_int), ("blocks_per_sm", C.c_int), ("chunk_rows", C.c_int)]


class MMError(RuntimeError):
    pass


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libmm.so (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            raise MMError(f"{_build.LIB} is missing: build it with "
                          "paper_1912_13282_gb300._build.build() (needs nvcc)")
        lib = C.CDLL(_build.LIB)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        lib.mm_ctx_create.argtypes = [C.POINTER(vp), C.c_int, vp]
        lib.mm_ctx_destroy.argtypes = [vp]
        lib.mm_ctx_destroy.restype = None
        lib.mm_ctx_set_stream.argtypes = [vp, vp]
        lib.mm_ctx_set_option.argtypes = [vp, C.c_int, dbl]
        lib.mm_last_error.argtypes = [vp]
        lib.mm_last_error.restype = C.c_char_p
        lib.mm_ctx_workspace_bytes.argtypes = [vp]
        lib.mm_knn_stencils.argtypes = [vp, C.c_int, i64, vp, C.c_int, C.POINTER(KnnRange),
                                        C.c_int, vp]
        lib.mm_balanced_stencils.argtypes = [vp, C.c_int, i64, vp, C.c_int, C.POINTER(KnnRange), C.c_int,
                                             C.c_int, vp]
        lib.mm_rbffd_weights.argtypes = [vp, C.c_uint, C.c_int, C.c_int, C.c_int, i64, vp, vp,
                                         C.POINTER(CsrPattern), i64, i64, C.c_int, C.c_int,
                                         C.POINTER(vp), vp]
        lib.mm_rbffd_weights_ir_noalloc.argtypes = [vp, C.c_uint, C.c_int, C.c_int, C.c_int, i64,
                                                    vp, vp, C.POINTER(CsrPattern), i64, i64,
                                                    C.c_int, C.POINTER(vp), vp]
        lib.mm_rbffd_weights_batched.argtypes = [vp, C.c_int, C.POINTER(WeightsClass), C.c_int,
                                                 C.POINTER(LaunchConfig)]
        lib.mm_wls_weights.argtypes = [vp, C.c_uint, C.c_int, dbl, C.c_int, C.c_int, i64, vp, vp,
                                       C.POINTER(CsrPattern), i64, i64, C.c_int, C.POINTER(vp), vp]
        lib.mm_autotune_batched.argtypes = [vp, C.c_int, C.POINTER(WeightsClass), C.c_int, i64,
                                            C.POINTER(LaunchConfig), C.POINTER(dbl)]
        lib.mm_tile_table_save.argtypes = [vp, C.c_char_p]
        lib.mm_tile_table_load.argtypes = [vp, C.c_char_p]
        lib.mm_mlp_create.argtypes = [vp, C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64]
        lib.mm_mlp_destroy.argtypes = [vp]
        lib.mm_mlp_destroy.restype = None
        lib.mm_mlp_num_params.argtypes = [vp]
        lib.mm_mlp_set_params.argtypes = [vp, vp, vp]
        lib.mm_mlp_get_params.argtypes = [vp, vp, vp]
        lib.mm_mlp_set_output_scaling.argtypes = [vp, vp, vp, vp]
        lib.mm_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
        lib.mm_mlp_fit_output_scaling.argtypes = [vp, vp, i64, vp]
        lib.mm_surrogate_targets.argtypes = [vp, C.POINTER(CsrPattern), i64, i64, C.c_int, vp, vp, C.c_int, vp]
        lib.mm_mlp_train_step.argtypes = [vp, vp, i64, vp, vp, C.c_float, vp]
        lib.mm_mlp_grad.argtypes = [vp, vp, i64, vp, vp, vp, vp]
        lib.mm_mlp_save.argtypes = [vp, vp, C.c_char_p]
        lib.mm_mlp_load.argtypes = [vp, vp, C.c_char_p]
        lib.mm_stencil_features.argtypes = [vp, C.c_int, i64, vp, C.POINTER(CsrPattern), i64, i64,
                                            C.c_int, C.c_int, vp, vp]
        lib.mm_rbffd_weights_surrogate.argtypes = [vp, vp, C.c_int, C.c_int, C.c_int, i64, vp,
                                                   C.POINTER(CsrPattern), i64, i64, C.c_int, dbl,
                                                   C.c_int, vp, vp, vp]
        lib.mm_apply_operator.argtypes = [vp, C.POINTER(CsrPattern), vp, vp, dbl, dbl, vp]
        lib.mm_diffuse.argtypes = [vp, C.POINTER(CsrPattern), vp, vp, dbl, C.c_int, vp, vp]
        lib.mm_diffuse_bc.argtypes = [vp, C.POINTER(CsrPattern), vp, vp, vp, dbl, C.c_int, vp, vp]
        lib.mm_combine_operators.argtypes = [vp, C.POINTER(CsrPattern), i64, i64, C.c_int, C.POINTER(vp),
                                             C.POINTER(vp), vp]
        lib.mm_implicit_assemble.argtypes = [vp, C.POINTER(CsrPattern), vp, vp, vp, vp]
        lib.mm_ilu0.argtypes = [vp, C.POINTER(CsrPattern), vp, vp, vp]
        lib.mm_ilu0_solve.argtypes = [vp, C.POINTER(CsrPattern), vp, vp, vp, vp]
        lib.mm_bicgstab.argtypes = [vp, C.POINTER(CsrPattern), vp, vp, vp, vp, vp, dbl, C.c_int,
                                    C.POINTER(C.c_int), C.POINTER(dbl)]
        lib.mm_partition_morton.argtypes = [C.c_int, i64, vp, C.c_int, vp, vp]
        lib.mm_partition_halo.argtypes = [C.c_int, i64, vp, vp, i64, i64, dbl, vp, i64, C.POINTER(i64)]
        lib.mm_measure_fma_peak.argtypes = [vp, C.c_int, C.POINTER(dbl)]
        for name in EXPORTS:
            if name not in ("mm_ctx_destroy", "mm_last_error", "mm_mlp_destroy",
                            "mm_mlp_num_params", "mm_ctx_workspace_bytes"):
                getattr(lib, name).restype = C.c_int
        lib.mm_mlp_num_params.restype = i64
        lib.mm_ctx_workspace_bytes.restype = i64
        _lib = lib
        return lib


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _dev(t, name, dtype):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise MMError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise MMError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise MMError(f"{name} must be contiguous")
    return t


class Context:
    """An mm_ctx bound to a device and a torch stream (default: current)."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self._lib = load()
        self.device = device
        s = stream if stream is not None else torch.cuda.current_stream(device)
        self.stream = s
        h = C.c_void_p()
        rc = self._lib.mm_ctx_create(C.byref(h), device, C.c_void_p(s.cuda_stream))
        if rc != MM_OK:
            raise MMError(f"mm_ctx_create failed ({rc})")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.mm_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != MM_OK:
            msg = self._lib.mm_last_error(self._h).decode(errors="replace")
            raise MMError(f"libmm error {rc}: {msg}")

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        self._check(self._lib.mm_ctx_set_stream(self._h, C.c_void_p(stream.cuda_stream)))

    def workspace_bytes(self) -> int:
        """Device workspace the context holds (mm_ctx_workspace_bytes)."""
        return int(self._lib.mm_ctx_workspace_bytes(self._h))

    def set_option(self, key: int, value: float):
        self._check(self._lib.mm_ctx_set_option(self._h, key, float(value)))

    # ------------------------------------------------------------ stencils
    def knn_stencils(self, pts: torch.Tensor, ranges, method: int = KNN_AUTO,
                     status: torch.Tensor | None = None):
        """ranges: list of (q_begin, q_end, n, out_idx int32 [(q_end-q_begin), n])."""
        _dev(pts, "pts", torch.float64)
        N, dim = pts.shape
        arr = (KnnRange * max(1, len(ranges)))()
        for i, (qb, qe, n, out) in enumerate(ranges):
            _dev(out, "idx", torch.int32)
            if out.numel() < (qe - qb) * n:
                raise MMError("idx tensor too small")
            arr[i] = KnnRange(qb, qe, n, out.data_ptr())
        if status is not None:
            _dev(status, "status", torch.int32)
        self._check(self._lib.mm_knn_stencils(self._h, dim, N, _ptr(pts), len(ranges), arr,
                                              method, _ptr(status)))

    def balanced_stencils(self, pts: torch.Tensor, ranges, K: int, method: int = KNN_AUTO,
                          status: torch.Tensor | None = None):
        """mm_balanced_stencils; ranges as knn_stencils, K candidates per query."""
        _dev(pts, "pts", torch.float64)
        N, dim = pts.shape
        arr = (KnnRange * max(1, len(ranges)))()
        for i, (qb, qe, n, out) in enumerate(ranges):
            _dev(out, "idx", torch.int32)
            if out.numel() < (qe - qb) * n:
                raise MMError("idx tensor too small")
            arr[i] = KnnRange(qb, qe, n, out.data_ptr())
        if status is not None:
            _dev(status, "status", torch.int32)
        self._check(self._lib.mm_balanced_stencils(self._h, dim, N, _ptr(pts), len(ranges), arr, int(K),
                                                   method, _ptr(status)))

    # ------------------------------------------------------------- weights
    def rbffd_weights(self, ops: int, k: int, m: int, pts: torch.Tensor, row_ptr: torch.Tensor,
                      col: torch.Tensor, vals, row_begin: int = 0, row_end: int | None = None,
                      n_max: int | None = None, precision: int = FP64,
                      normals: torch.Tensor | None = None, status: torch.Tensor | None = None):
        """vals: list of float64 [nnz] tensors, one per set bit of ops (bit order)."""
        _dev(pts, "pts", torch.float64)
        _dev(row_ptr, "row_ptr", torch.int64)
        _dev(col, "col", torch.int32)
        N, dim = pts.shape
        nrows = row_ptr.numel() - 1
        if row_end is None:
            row_end = nrows
        if n_max is None:
            raise MMError("n_max (largest stencil size in the row range) is required")
        nbits = bin(ops).count("1")
        if len(vals) != nbits:
            raise MMError(f"{nbits} value arrays expected")
        for v in vals:
            _dev(v, "vals", torch.float64)
        if normals is not None:
            _dev(normals, "normals", torch.float64)
        if status is not None:
            _dev(status, "status", torch.int32)
        pat = CsrPattern(nrows, col.numel(), row_ptr.data_ptr(), col.data_ptr())
        vp = (C.c_void_p * max(1, nbits))(*[v.data_ptr() for v in vals])
        self._check(self._lib.mm_rbffd_weights(self._h, ops, k, m, dim, N, _ptr(pts),
                                               _ptr(normals), C.byref(pat), row_begin, row_end,
                                               n_max, precision, vp, _ptr(status)))

    def wls_weights(self, ops: int, m: int, sigma: float, scale: int, pts: torch.Tensor,
                    row_ptr: torch.Tensor, col: torch.Tensor, vals, row_begin: int = 0,
                    row_end: int | None = None, n_max: int | None = None,
                    normals: torch.Tensor | None = None, status: torch.Tensor | None = None):
        """GWLS weights (mm_wls_weights); vals as for rbffd_weights."""
        _dev(pts, "pts", torch.float64)
        _dev(row_ptr, "row_ptr", torch.int64)
        _dev(col, "col", torch.int32)
        N, dim = pts.shape
        nrows = row_ptr.numel() - 1
        if row_end is None:
            row_end = nrows
        if n_max is None:
            raise MMError("n_max (largest stencil size in the row range) is required")
        nbits = bin(ops).count("1")
        if len(vals) != nbits:
            raise MMError(f"{nbits} value arrays expected")
        for v in vals:
            _dev(v, "vals", torch.float64)
        if normals is not None:
            _dev(normals, "normals", torch.float64)
        if status is not None:
            _dev(status, "status", torch.int32)
        pat = CsrPattern(nrows, col.numel(), row_ptr.data_ptr(), col.data_ptr())
        vp = (C.c_void_p * max(1, nbits))(*[v.data_ptr() for v in vals])
        self._check(self._lib.mm_wls_weights(self._h, ops, m, float(sigma), scale, dim, N, _ptr(pts),
                                             _ptr(normals), C.byref(pat), row_begin, row_end, n_max,
                                             vp, _ptr(status)))

    def rbffd_weights_ir_noalloc(self, ops: int, k: int, m: int, pts, row_ptr, col, vals,
                                 row_begin: int = 0, row_end: int | None = None,
                                 n_max: int | None = None, normals=None, status=None):
        """mm_rbffd_weights_ir_noalloc: FP32 + FP64 refinement without any
        device allocation (at most 2^20 rows per call; see include/mm.h)."""
        _dev(pts, "pts", torch.float64)
        _dev(row_ptr, "row_ptr", torch.int64)
        _dev(col, "col", torch.int32)
        N, dim = pts.shape
        nrows = row_ptr.numel() - 1
        row_end = nrows if row_end is None else row_end
        if n_max is None:
            raise MMError("n_max is required")
        for v in vals:
            _dev(v, "vals", torch.float64)
        pat = CsrPattern(nrows, col.numel(), row_ptr.data_ptr(), col.data_ptr())
        vp = (C.c_void_p * max(1, len(vals)))(*[v.data_ptr() for v in vals])
        self._check(self._lib.mm_rbffd_weights_ir_noalloc(
            self._h, ops, k, m, dim, N, _ptr(pts), _ptr(normals), C.byref(pat), row_begin,
            row_end, n_max, vp, _ptr(status)))

    @staticmethod
    def weights_class(ops, k, m, pts, row_ptr, col, vals, row_begin=0, row_end=None, n_max=None,
                      normals=None, status=None):
        """Describe one stencil class for rbffd_weights_batched (tensors must
        stay alive until the call has run)."""
        _dev(pts, "pts", torch.float64)
        _dev(row_ptr, "row_ptr", torch.int64)
        _dev(col, "col", torch.int32)
        N, dim = pts.shape
        nrows = row_ptr.numel() - 1
        nbits = bin(ops).count("1")
        if len(vals) != nbits:
            raise MMError(f"{nbits} value arrays expected")
        if n_max is None:
            raise MMError("n_max is required")
        wc = WeightsClass()
        wc.ops, wc.k, wc.m, wc.dim, wc.N = ops, k, m, dim, N
        wc.d_pts = pts.data_ptr()
        wc.d_normals = normals.data_ptr() if normals is not None else None
        wc.stencils = CsrPattern(nrows, col.numel(), row_ptr.data_ptr(), col.data_ptr())
        wc.row_begin = row_begin
        wc.row_end = nrows if row_end is None else row_end
        wc.n_max = n_max
        for i, v in enumerate(vals):
            _dev(v, "vals", torch.float64)
            wc.d_vals[i] = v.data_ptr()
        wc.d_status = status.data_ptr() if status is not None else None
        return wc

    def rbffd_weights_batched(self, classes, precision=FP64, config=None):
        """mm_rbffd_weights_batched: all classes in one persistent launch.
        config: (warps_per_block, blocks_per_sm, chunk_rows) or None."""
        arr = (WeightsClass * len(classes))(*classes)
        cfg = None if config is None else C.byref(LaunchConfig(*config))
        self._check(self._lib.mm_rbffd_weights_batched(self._h, len(classes), arr, precision, cfg))

    def autotune_batched(self, classes, precision=FP64, sample_rows=0):
        """mm_autotune_batched; returns ((warps_per_block, blocks_per_sm, chunk_rows), ms)."""
        arr = (WeightsClass * len(classes))(*classes)
        best = LaunchConfig()
        ms = C.c_double()
        self._check(self._lib.mm_autotune_batched(self._h, len(classes), arr, precision,
                                                  int(sample_rows), C.byref(best), C.byref(ms)))
        return (best.warps_per_block, best.blocks_per_sm, best.chunk_rows), ms.value

    def tile_table_save(self, path):
        self._check(self._lib.mm_tile_table_save(self._h, str(path).encode()))

    def tile_table_load(self, path):
        self._check(self._lib.mm_tile_table_load(self._h, str(path).encode()))

    # ------------------------------------------------- operator application
    def apply_operator(self, row_ptr, col, vals, u, y, alpha=1.0, beta=0.0):
        _dev(row_ptr, "row_ptr", torch.int64)
        _dev(col, "col", torch.int32)
        _dev(vals, "vals", torch.float64)
        _dev(u, "u", torch.float64)
        _dev(y, "y", torch.float64)
        pat = CsrPattern(row_ptr.numel() - 1, col.numel(), row_ptr.data_ptr(), col.data_ptr())
        self._check(self._lib.mm_apply_operator(self._h, C.byref(pat), _ptr(vals), _ptr(u),
                                                float(alpha), float(beta), _ptr(y)))

    def diffuse(self, row_ptr, col, vals, fixed, dt, steps, u, work):
        _dev(row_ptr, "row_ptr", torch.int64)
        _dev(col, "col", torch.int32)
        _dev(vals, "vals", torch.float64)
        _dev(fixed, "fixed", torch.uint8)
        _dev(u, "u", torch.float64)
        _dev(work, "work", torch.float64)
        pat = CsrPattern(row_ptr.numel() - 1, col.numel(), row_ptr.data_ptr(), col.data_ptr())
        self._check(self._lib.mm_diffuse(self._h, C.byref(pat), _ptr(vals), _ptr(fixed),
                                         float(dt), int(steps), _ptr(u), _ptr(work)))

    def diffuse_bc(self, row_ptr, col, vals, kind, g, dt, steps, u, work):
        """mm_diffuse_bc: kind [nrows] uint8 (ROW_INTERNAL / ROW_DIRICHLET /
        ROW_NEUMANN), g [nrows] float64 Neumann data or None."""
        _dev(row_ptr, "row_ptr", torch.int64)
        _dev(col, "col", torch.int32)
        _dev(vals, "vals", torch.float64)
        _dev(kind, "kind", torch.uint8)
        if g is not None:
            _dev(g, "g", torch.float64)
        _dev(u, "u", torch.float64)
        _dev(work, "work", torch.float64)
        pat = CsrPattern(row_ptr.numel() - 1, col.numel(), row_ptr.data_ptr(), col.data_ptr())
        self._check(self._lib.mm_diffuse_bc(self._h, C.byref(pat), _ptr(vals), _ptr(kind), _ptr(g),
                                            float(dt), int(steps), _ptr(u), _ptr(work)))

    def combine_operators(self, row_ptr, col, terms, coefs, out, row_begin: int = 0,
                          row_end: int | None = None):
        """mm_combine_operators: out = sum_t coefs[t][row] * terms[t] (coefs[t]
        None means 1; coefs None means all 1)."""
        _dev(row_ptr, "row_ptr", torch.int64)
        _dev(col, "col", torch.int32)
        _dev(out, "out", torch.float64)
        for t in terms:
            _dev(t, "terms", torch.float64)
        if coefs is not None:
            if len(coefs) != len(terms):
                raise MMError("one coefficient array (or None) per term expected")
            for a in coefs:
                if a is not None:
                    _dev(a, "coefs", torch.float64)
        nrows = row_ptr.numel() - 1
        if row_end is None:
            row_end = nrows
        pat = CsrPattern(nrows, col.numel(), row_ptr.data_ptr(), col.data_ptr())
        tp = (C.c_void_p * max(1, len(terms)))(*[t.data_ptr() for t in terms])
        cp = None if coefs is None else (C.c_void_p * len(coefs))(
            *[None if a is None else a.data_ptr() for a in coefs])
        self._check(self._lib.mm_combine_operators(self._h, C.byref(pat), row_begin, row_end, len(terms),
                                                   tp, cp, _ptr(out)))

    # ------------------------------------------------------- implicit solve
    def implicit_assemble(self, row_ptr, col, vals, kind, col_out, vals_out):
        """mm_implicit_assemble: rows sorted by column, Dirichlet rows (kind
        == ROW_DIRICHLET, uint8 [nrows] or None) replaced by the identity."""
        _dev(row_ptr, "row_ptr", torch.int64)
        _dev(col, "col", torch.int32)
        _dev(vals, "vals", torch.float64)
        _dev(col_out, "col_out", torch.int32)
        _dev(vals_out, "vals_out", torch.float64)
        if kind is not None:
            _dev(kind, "kind", torch.uint8)
        pat = CsrPattern(row_ptr.numel() - 1, col.numel(), row_ptr.data_ptr(), col.data_ptr())
        self._check(self._lib.mm_implicit_assemble(self._h, C.byref(pat), _ptr(vals), _ptr(kind),
                                                   _ptr(col_out), _ptr(vals_out)))

    def ilu0(self, row_ptr, col, vals, factors, diag):
        """mm_ilu0 on a sorted CSR matrix; factors float64 [nnz] (may be vals),
        diag int64 [nrows]."""
        _dev(row_ptr, "row_ptr", torch.int64)
        _dev(col, "col", torch.int32)
        _dev(vals, "vals", torch.float64)
        _dev(factors, "factors", torch.float64)
        _dev(diag, "diag", torch.int64)
        pat = CsrPattern(row_ptr.numel() - 1, col.numel(), row_ptr.data_ptr(), col.data_ptr())
        self._check(self._lib.mm_ilu0(self._h, C.byref(pat), _ptr(vals), _ptr(factors), _ptr(diag)))

    def ilu0_solve(self, row_ptr, col, factors, diag, b, x):
        pat = CsrPattern(row_ptr.numel() - 1, col.numel(), row_ptr.data_ptr(), col.data_ptr())
        for t, nm, dt in ((row_ptr, "row_ptr", torch.int64), (col, "col", torch.int32),
                          (factors, "factors", torch.float64), (diag, "diag", torch.int64),
                          (b, "b", torch.float64), (x, "x", torch.float64)):
            _dev(t, nm, dt)
        self._check(self._lib.mm_ilu0_solve(self._h, C.byref(pat), _ptr(factors), _ptr(diag), _ptr(b),
                                            _ptr(x)))

    def bicgstab(self, row_ptr, col, vals, b, x, factors=None, diag=None, tol=1e-10, maxit=1000,
                 check=True):
        """mm_bicgstab; returns (return code, iterations, relative residual).
        With check=True a code other than MM_OK or MM_ENOCONV raises."""
        pat = CsrPattern(row_ptr.numel() - 1, col.numel(), row_ptr.data_ptr(), col.data_ptr())
        for t, nm, dt in ((row_ptr, "row_ptr", torch.int64), (col, "col", torch.int32),
                          (vals, "vals", torch.float64), (b, "b", torch.float64), (x, "x", torch.float64)):
            _dev(t, nm, dt)
        it, res = C.c_int(0), C.c_double(0.0)
        rc = self._lib.mm_bicgstab(self._h, C.byref(pat), _ptr(vals), _ptr(factors), _ptr(diag), _ptr(b),
                                   _ptr(x), float(tol), int(maxit), C.byref(it), C.byref(res))
        if check and rc not in (MM_OK, MM_ENOCONV):
            self._check(rc)
        return rc, it.value, res.value

    def measure_fma_peak(self, which: int) -> float:
        out = C.c_double()
        self._check(self._lib.mm_measure_fma_peak(self._h, which, C.byref(out)))
        return out.value


def partition_morton(pts, nparts: int):
    """mm_partition_morton on host points (numpy [N, dim]): (perm, starts)."""
    import numpy as np
    lib = load()
    p = np.ascontiguousarray(pts, dtype=np.float64)
    N, dim = p.shape
    perm = np.empty(N, dtype=np.int64)
    starts = np.empty(nparts + 1, dtype=np.int64)
    rc = lib.mm_partition_morton(dim, N, p.ctypes.data_as(C.c_void_p), nparts, perm.ctypes.data_as(C.c_void_p),
                                 starts.ctypes.data_as(C.c_void_p))
    if rc != MM_OK:
        raise MMError(f"mm_partition_morton failed ({rc})")
    return perm, starts


def partition_halo(pts, perm, begin: int, end: int, radius: float):
    """mm_partition_halo: indices of the nodes outside perm[begin:end] within
    `radius` of one of its nodes (increasing)."""
    import numpy as np
    lib = load()
    p = np.ascontiguousarray(pts, dtype=np.float64)
    pm = np.ascontiguousarray(perm, dtype=np.int64)
    N, dim = p.shape
    cap = max(1024, 2 * (end - begin))
    while True:
        halo = np.empty(cap, dtype=np.int64)
        cnt = C.c_int64(0)
        rc = lib.mm_partition_halo(dim, N, p.ctypes.data_as(C.c_void_p), pm.ctypes.data_as(C.c_void_p), begin, end,
                                   float(radius), halo.ctypes.data_as(C.c_void_p), cap, C.byref(cnt))
        if rc == MM_OK:
            return halo[:cnt.value].copy()
        if rc != MM_EUNSUPPORTED:
            raise MMError(f"mm_partition_halo failed ({rc})")
        cap = int(cnt.value)


class MLP:
    """The surrogate network (mm_mlp_*): 2D stencil features -> scaled
    Laplacian weights."""

    def __init__(self, ctx: Context, n_in: int, n_out: int, seed: int = 0):
        self.ctx = ctx
        self._lib = ctx._lib
        h = C.c_void_p()
        ctx._check(self._lib.mm_mlp_create(ctx._h, C.byref(h), n_in, 256, 3, n_out, seed))
        self._h = h
        self.n_in, self.n_out = n_in, n_out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.mm_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self) -> int:
        return int(self._lib.mm_mlp_num_params(self._h))

    def set_params(self, params):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        self.ctx._check(self._lib.mm_mlp_set_params(self.ctx._h, self._h, a.ctypes.data_as(C.c_void_p)))

    def get_params(self):
        import numpy as np
        a = np.empty(self.num_params, dtype=np.float32)
        self.ctx._check(self._lib.mm_mlp_get_params(self.ctx._h, self._h, a.ctypes.data_as(C.c_void_p)))
        return a

    def set_output_scaling(self, mean, std):
        import numpy as np
        m = np.ascontiguousarray(mean, dtype=np.float32)
        s = np.ascontiguousarray(std, dtype=np.float32)
        self.ctx._check(self._lib.mm_mlp_set_output_scaling(self.ctx._h, self._h,
                                                             m.ctypes.data_as(C.c_void_p),
                                                             s.ctypes.data_as(C.c_void_p)))

    def fit_output_scaling(self, t: torch.Tensor):
        """mm_mlp_fit_output_scaling from training targets t [B, n_out] (device)."""
        _dev(t, "t", torch.float32)
        self.ctx._check(self._lib.mm_mlp_fit_output_scaling(self.ctx._h, self._h, t.shape[0], _ptr(t)))

    def forward(self, x: torch.Tensor, y: torch.Tensor):
        _dev(x, "x", torch.float32)
        _dev(y, "y", torch.float32)
        self.ctx._check(self._lib.mm_mlp_forward(self.ctx._h, self._h, x.shape[0], _ptr(x), _ptr(y)))

    def train_step(self, x: torch.Tensor, t: torch.Tensor, lr: float, loss: torch.Tensor | None = None):
        _dev(x, "x", torch.float32)
        _dev(t, "t", torch.float32)
        self.ctx._check(self._lib.mm_mlp_train_step(self.ctx._h, self._h, x.shape[0], _ptr(x), _ptr(t),
                                                    float(lr), _ptr(loss)))

    def grad(self, x: torch.Tensor, t: torch.Tensor):
        import numpy as np
        _dev(x, "x", torch.float32)
        _dev(t, "t", torch.float32)
        g = np.empty(self.num_params, dtype=np.float32)
        loss = C.c_float()
        self.ctx._check(self._lib.mm_mlp_grad(self.ctx._h, self._h, x.shape[0], _ptr(x), _ptr(t),
                                              g.ctypes.data_as(C.c_void_p), C.byref(loss)))
        return float(loss.value), g

    def save(self, path):
        self.ctx._check(self._lib.mm_mlp_save(self.ctx._h, self._h, str(path).encode()))

    def load(self, path):
        self.ctx._check(self._lib.mm_mlp_load(self.ctx._h, self._h, str(path).encode()))


def stencil_features(ctx: Context, pts, row_ptr, col, row_begin, row_end, n, x, scale=None,
                     orient=True):
    _dev(pts, "pts", torch.float64)
    pat = CsrPattern(row_ptr.numel() - 1, col.numel(), row_ptr.data_ptr(), col.data_ptr())
    ctx._check(ctx._lib.mm_stencil_features(ctx._h, pts.shape[1], pts.shape[0], _ptr(pts),
                                            C.byref(pat), row_begin, row_end, n, int(orient),
                                            _ptr(x), _ptr(scale)))


def surrogate_targets(ctx: Context, row_ptr, row_begin, row_end, n, vals, scale, q, out):
    """mm_surrogate_targets: out [(row_end - row_begin), n] FP32 = vals * scale^q."""
    _dev(vals, "vals", torch.float64)
    _dev(scale, "scale", torch.float64)
    _dev(out, "out", torch.float32)
    pat = CsrPattern(row_ptr.numel() - 1, vals.numel(), row_ptr.data_ptr(), 0)
    ctx._check(ctx._lib.mm_surrogate_targets(ctx._h, C.byref(pat), row_begin, row_end, n, _ptr(vals),
                                             _ptr(scale), q, _ptr(out)))


def rbffd_weights_surrogate(ctx: Context, net: MLP, k, m, pts, row_ptr, col, row_begin, row_end, n,
                            tau, lap_vals, status=None, rho=None, fallback=FP64):
    _dev(pts, "pts", torch.float64)
    _dev(lap_vals, "lap_vals", torch.float64)
    pat = CsrPattern(row_ptr.numel() - 1, col.numel(), row_ptr.data_ptr(), col.data_ptr())
    ctx._check(ctx._lib.mm_rbffd_weights_surrogate(ctx._h, net._h, k, m, pts.shape[1], pts.shape[0],
                                                   _ptr(pts), C.byref(pat), row_begin, row_end, n,
                                                   float(tau), int(fallback), _ptr(lap_vals),
                                                   _ptr(status), _ptr(rho)))
