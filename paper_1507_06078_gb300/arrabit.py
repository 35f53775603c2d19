"""Thin ctypes binding of the C ABI declared in include/arrabit.h.

Every function here only marshals arguments (tensor pointers, leading dimensions, host
arrays) and calls the library of the same name; all arithmetic runs in the library's CUDA
kernels.  PyTorch supplies device memory and the stream: a Context runs its kernels on
the torch stream that was current when it was created.

The library must have been built (``paper_1507_06078_gb300.build.build()``); loading
fails loudly otherwise - there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import weakref
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "lib", "libarrabit.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "arrabit.h")

ARB_OK, ARB_NOT_CONVERGED, ARB_INVALID_ARG, ARB_OUT_OF_MEMORY = 0, 1, -1, -2
ARB_NOT_SYMMETRIC, ARB_BREAKDOWN, ARB_CUDA_ERROR, ARB_TIMEOUT, ARB_REJECTED = -3, -4, -5, -6, -7
ARB_LARGEST, ARB_SMALLEST = 0, 1
ARB_FP64, ARB_MIXED, ARB_MIXED_DF = 0, 1, 2
ARB_FILTER_CHEBINTERP, ARB_FILTER_CHEBYSHEV = 0, 1
ARB_INNER_MPM, ARB_INNER_GN = 0, 1
ARB_ADAPT_Q, ARB_ADAPT_DEGREE = 1, 2
ARB_BATCH_GRAPHS, ARB_BATCH_AUTOTUNE = 1, 2
STOP_REASONS = {0: "converged", 1: "near_tol", 2: "stalled", 3: "maxit", 4: "all_locked"}


class ArbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"arrabit status {status}: {msg}")
        self.status = status


class arb_options(C.Structure):
    _fields_ = [("p", C.c_int32), ("q", C.c_int32), ("degree", C.c_int32), ("maxit", C.c_int32),
                ("maxit1", C.c_int32), ("maxit2", C.c_int32), ("inner_fixed", C.c_int32),
                ("filter", C.c_int32), ("precision", C.c_int32), ("b_update", C.c_int32),
                ("tol1", C.c_double), ("shift_sigma", C.c_double), ("tol_switch", C.c_double),
                ("seed", C.c_uint64), ("inner", C.c_int32), ("adapt", C.c_int32), ("q_max", C.c_int32),
                ("d_max", C.c_int32)]


class arb_filter_job(C.Structure):
    _fields_ = [("mat", C.c_void_p), ("op_scale", C.c_double), ("op_shift", C.c_double), ("a", C.c_double),
                ("b", C.c_double), ("degree", C.c_int32), ("fp32", C.c_int32), ("coef", C.c_void_p),
                ("X", C.c_void_p), ("ldx", C.c_int64), ("ncols", C.c_int32), ("reserved0", C.c_int32),
                ("xscale", C.c_void_p), ("Y", C.c_void_p), ("ldy", C.c_int64), ("colss", C.c_void_p)]


class arb_batch_stats(C.Structure):
    _fields_ = [("rounds", C.c_int64), ("batched_launches", C.c_int64), ("graph_launches", C.c_int64),
                ("graphs_captured", C.c_int64), ("single_steps", C.c_int64), ("t_total", C.c_double),
                ("t_batched", C.c_double), ("t_single", C.c_double), ("t_checks", C.c_double),
                ("t_batch_kernel", C.c_double), ("t_prepare", C.c_double), ("batched_jobs", C.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class arb_info(C.Structure):
    _fields_ = [("maxres", C.c_double), ("a", C.c_double), ("b0", C.c_double), ("b_final", C.c_double),
                ("sigma", C.c_double), ("t_total", C.c_double), ("t_filter", C.c_double),
                ("t_arr", C.c_double), ("spmm_cols", C.c_int64), ("outer_iters", C.c_int32),
                ("n_filters", C.c_int32), ("n_locked", C.c_int32), ("stop_reason", C.c_int32),
                ("last_rank", C.c_int32), ("outer_iters_fp32", C.c_int32), ("max_locked", C.c_int32),
                ("final_q", C.c_int32), ("final_d", C.c_int32), ("reserved0", C.c_int32)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if not f.startswith("reserved")}
        d["stop_reason"] = STOP_REASONS.get(self.stop_reason, str(self.stop_reason))
        return d


_lib = None
_vp, _i32, _i64, _dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
_PROTOS = {
    "arb_ctx_set_dense_df": (_i32, [_vp, C.c_int]),
    "arb_ctx_create": (_i32, [C.POINTER(_vp), C.c_int, _vp]),
    "arb_ctx_destroy": (_i32, [_vp]),
    "arb_last_error": (C.c_char_p, [_vp]),
    "arb_status_string": (C.c_char_p, [_i32]),
    "arb_kernel_launches": (_i64, [_vp]),
    "arb_options_default": (None, [C.POINTER(arb_options), _i32]),
    "arb_matrix_create_csr": (_i32, [_vp, _i64, _i64, _vp, _vp, _vp, C.c_int, C.POINTER(_vp)]),
    "arb_matrix_create_csr_f32": (_i32, [_vp, _i64, _i64, _vp, _vp, _vp, C.c_int, C.POINTER(_vp)]),
    "arb_csr_check_symmetric": (_i32, [_i64, _i64, _vp, _vp, _vp, _dbl]),
    "arb_matrix_destroy": (_i32, [_vp]),
    "arb_sell_layout": (_i32, [_i64, _vp, _i32, _i32, _vp, _vp, _vp, _vp, _i64, C.POINTER(_i64)]),
    "arb_matrix_set_sell": (_i32, [_vp, _vp, _i32, _i32]),
    "arb_matrix_sell_info": (_i32, [_vp, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i64)]),
    "arb_matrix_gershgorin": (_i32, [_vp, _vp, C.POINTER(_dbl), C.POINTER(_dbl)]),
    "arb_solve": (_i32, [_vp, _vp, _i32, _i32, _dbl, C.POINTER(arb_options), _vp, C.c_int, _vp, _vp, _i64,
                         C.c_int, C.POINTER(arb_info)]),
    "arb_gaussian_block": (_i32, [_vp, _i64, _i32, C.c_uint64, _vp, _i64]),
    "arb_filter": (_i32, [_vp, _vp, _dbl, _dbl, _dbl, _dbl, _i32, _vp, _vp, _i64, _i32, _vp, _vp, _i64, _vp]),
    "arb_filter_f32": (_i32, [_vp, _vp, _dbl, _dbl, _dbl, _dbl, _i32, _vp, _vp, _i64, _i32, _vp, _vp, _i64,
                              _vp]),
    "arb_filter_df": (_i32, [_vp, _vp, _dbl, _dbl, _dbl, _dbl, _i32, _vp, _vp, _i64, _i32, _vp, _vp, _i64, _vp]),
    "arb_filter_coefficients": (_i32, [_i32, _i32, _vp]),
    "arb_filter_batched": (_i32, [_vp, _i32, _vp]),
    "arb_spmm": (_i32, [_vp, _vp, _dbl, _dbl, _vp, _i64, _i32, _vp, _i64]),
    "arb_gram": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i64]),
    "arb_gram_f32": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i64]),
    "arb_gram_noalloc": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i64]),
    "arb_gemm_tall_f32": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _dbl, _dbl, _vp, _i64]),
    "arb_server_footprint": (_i64, [_i64, _i64, _i32, _i32, _i32]),
    "arb_server_create": (_i32, [C.c_int, C.c_size_t, _i32, C.POINTER(_vp)]),
    "arb_submit": (_i32, [_vp, _vp, _i32, _i32, _dbl, C.POINTER(arb_options), _vp, C.c_int, C.POINTER(_i64)]),
    "arb_wait": (_i32, [_vp, _i64, _i32, _vp, _vp, _i64, C.POINTER(arb_info), C.POINTER(_dbl)]),
    "arb_server_destroy": (_i32, [_vp]),
    "arb_solve_batched": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32]),
    "arb_solve_lockstep": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32,
                                  C.POINTER(arb_batch_stats)]),
    "arb_matrix_autotune": (_i32, [_vp, _vp, _i32, _vp, C.POINTER(_dbl)]),
    "arb_syevj": (_i32, [_vp, _i32, _vp, _i64, _vp, _vp, _i64, C.POINTER(_i32)]),
    "arb_rcond_gram": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, C.POINTER(_dbl)]),
    "arb_orth": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, C.POINTER(_i32)]),
    "arb_rayleigh_ritz": (_i32, [_vp, _vp, _dbl, _dbl, _i64, _vp, _i64, _i32, _vp, _i64, _vp, C.POINTER(_i32)]),
    "arb_arr": (_i32, [_vp, _vp, _dbl, _dbl, _i64, _vp, _i64, _i32, _i32, _i32, _vp, _i64, _vp, C.POINTER(_i32)]),
}


def header_functions() -> list[str]:
    """Names of the functions include/arrabit.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(arb_\w+)\s*\(", txt)))


def load():
    """Load the built library (raises if it is missing: no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIBPATH):
        raise RuntimeError(f"CUDA library not built: {LIBPATH} missing "
                           "(run paper_1507_06078_gb300.build.build())")
    lib = C.CDLL(LIBPATH)
    for name, (res, args) in _PROTOS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(ctx, st: int, what: str):
    if st not in (ARB_OK, ARB_NOT_CONVERGED):
        msg = load().arb_last_error(ctx.handle if ctx is not None else None)
        raise ArbError(st, f"{what}: {load().arb_status_string(st).decode()} ({msg.decode() if msg else ''})")
    return st


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _dev2d(t, name: str):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.dim() == 2
            and t.stride(1) == 1):
        raise ValueError(f"{name}: expected a row-major 2D float64 CUDA tensor")
    return t.stride(0)


class Context:
    """A library context bound to a CUDA device and the current torch stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        lib = load()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.device = device
        h = _vp()
        st = lib.arb_ctx_create(C.byref(h), device, _vp(stream.cuda_stream))
        if st != ARB_OK:
            raise ArbError(st, "arb_ctx_create failed")
        self.handle = h
        self._mats = weakref.WeakSet()

    def close(self):
        if self.handle:
            for m in list(self._mats):
                m.close()
            load().arb_ctx_destroy(self.handle)
            self.handle = None

    def launches(self) -> int:
        return int(load().arb_kernel_launches(self.handle))

    def set_dense_df(self, enable: bool):
        """FP64 Gram / tall-skinny products of this context in double-float arithmetic."""
        _check(self, load().arb_ctx_set_dense_df(self.handle, 1 if enable else 0), "arb_ctx_set_dense_df")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Matrix:
    """A CSR matrix copied into library-owned device memory."""

    def __init__(self, ctx: Context, n: int, rowptr, col, val):
        """val: float64 values, or float32 (arb_matrix_create_csr_f32)."""
        lib = load()
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        f32 = np.asarray(val).dtype == np.float32
        val = np.ascontiguousarray(val, dtype=np.float32 if f32 else np.float64)
        h = _vp()
        fn = lib.arb_matrix_create_csr_f32 if f32 else lib.arb_matrix_create_csr
        st = fn(ctx.handle, n, col.shape[0], rowptr.ctypes.data, col.ctypes.data, val.ctypes.data, 0, C.byref(h))
        _check(ctx, st, "arb_matrix_create_csr_f32" if f32 else "arb_matrix_create_csr")
        self.ctx, self.handle, self.n, self.nnz = ctx, h, n, col.shape[0]
        ctx._mats.add(self)

    @classmethod
    def from_csr(cls, ctx: Context, A) -> "Matrix":
        return cls(ctx, A.n, A.rowptr, A.col, A.val)

    def set_sell(self, chunk: int = 32, sigma: int = 1024):
        """Give the matrix a SELL-C-sigma copy (chunk = 0: back to CSR only)."""
        _check(self.ctx, load().arb_matrix_set_sell(self.ctx.handle, self.handle, chunk, sigma),
               "arb_matrix_set_sell")

    def sell_info(self) -> tuple[int, int, int]:
        c, s, slots = _i32(), _i32(), _i64()
        st = load().arb_matrix_sell_info(self.handle, C.byref(c), C.byref(s), C.byref(slots))
        if st != ARB_OK:
            raise ArbError(st, "arb_matrix_sell_info")
        return c.value, s.value, slots.value

    def close(self):
        if self.handle:
            load().arb_matrix_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def arb_sell_layout(rowptr, chunk: int, sigma: int):
    """Host SELL-C-sigma layout of a CSR pattern: (perm, len, cptr, src) as numpy arrays."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    n = rowptr.shape[0] - 1
    perm = np.zeros(max(n, 1), dtype=np.int32)
    ln = np.zeros(max(n, 1), dtype=np.int32)
    cptr = np.zeros((n + chunk - 1) // max(chunk, 1) + 1 if chunk > 0 else 1, dtype=np.int64)
    slots = _i64()
    lib = load()
    st = lib.arb_sell_layout(n, rowptr.ctypes.data, chunk, sigma, perm.ctypes.data, ln.ctypes.data,
                             cptr.ctypes.data, None, 0, C.byref(slots))
    if st != ARB_OK:
        raise ArbError(st, "arb_sell_layout")
    src = np.zeros(max(slots.value, 1), dtype=np.int64)
    st = lib.arb_sell_layout(n, rowptr.ctypes.data, chunk, sigma, perm.ctypes.data, ln.ctypes.data,
                             cptr.ctypes.data, src.ctypes.data, src.shape[0], C.byref(slots))
    if st != ARB_OK:
        raise ArbError(st, "arb_sell_layout")
    return perm[:n], ln[:n], cptr, src[:slots.value]


def arb_options_default(k: int) -> arb_options:
    o = arb_options()
    load().arb_options_default(C.byref(o), k)
    return o


def arb_matrix_gershgorin(ctx: Context, mat: Matrix) -> tuple[float, float]:
    lo, hi = _dbl(), _dbl()
    _check(ctx, load().arb_matrix_gershgorin(ctx.handle, mat.handle, C.byref(lo), C.byref(hi)), "gershgorin")
    return lo.value, hi.value


def arb_filter_coefficients(kind: int, degree: int) -> np.ndarray:
    c = np.zeros(degree + 1, dtype=np.float64)
    st = load().arb_filter_coefficients(kind, degree, c.ctypes.data)
    if st != ARB_OK:
        raise ArbError(st, "arb_filter_coefficients")
    return c


@dataclass
class SolveResult:
    status: int
    evals: np.ndarray
    evecs: object
    info: dict


def arb_solve(ctx: Context, mat: Matrix, k: int, which: int, tol: float, opts: arb_options | None = None,
              x0=None, evecs: str | None = "host") -> SolveResult:
    """Algorithm 8 end to end.  x0: numpy (host) or torch CUDA n x p float64, or None.
    evecs: "host" (numpy, n x k), "device" (torch CUDA tensor holding the column-major
    n x k block as a k x n row-major view), or None."""
    import torch
    lib = load()
    if opts is None:
        opts = arb_options_default(k)
    x0_ptr, x0_dev = 0, 0
    if x0 is not None:
        if isinstance(x0, np.ndarray):
            x0 = np.ascontiguousarray(x0, dtype=np.float64)
            x0_ptr = x0.ctypes.data
        else:
            _dev2d(x0, "x0")
            if x0.stride(0) != x0.shape[1]:
                raise ValueError("x0 must be contiguous")
            x0_ptr, x0_dev = _ptr(x0), 1
    ev = np.zeros(k, dtype=np.float64)
    out, optr, odev = None, 0, 0
    if evecs == "host":
        out = np.zeros((k, mat.n), dtype=np.float64)  # column-major n x k == row-major k x n
        optr = out.ctypes.data
    elif evecs == "device":
        out = torch.empty((k, mat.n), dtype=torch.float64, device=f"cuda:{ctx.device}")
        optr, odev = _ptr(out), 1
    info = arb_info()
    st = lib.arb_solve(ctx.handle, mat.handle, k, which, tol, C.byref(opts), _vp(x0_ptr), x0_dev,
                       ev.ctypes.data, _vp(optr), mat.n, odev, C.byref(info))
    _check(ctx, st, "arb_solve")
    vecs = None
    if out is not None:
        vecs = out.T
    return SolveResult(st, ev, vecs, info.as_dict())


def arb_csr_check_symmetric(n: int, rowptr, col, val, rel_tol: float = 0.0) -> int:
    """ARB_OK or ARB_NOT_SYMMETRIC (host arrays; no context, no device)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    return int(load().arb_csr_check_symmetric(n, col.shape[0], rowptr.ctypes.data, col.ctypes.data,
                                              val.ctypes.data, rel_tol))


def arb_gaussian_block(ctx: Context, n: int, ncols: int, seed: int, X=None):
    """Device start block from the library's Philox stream (same numbering as the input
    generator)."""
    import torch
    if X is None:
        X = torch.empty((n, ncols), dtype=torch.float64, device=f"cuda:{ctx.device}")
    ldx = _dev2d(X, "X")
    _check(ctx, load().arb_gaussian_block(ctx.handle, n, ncols, seed, _vp(_ptr(X)), ldx), "arb_gaussian_block")
    return X


def arb_filter(ctx: Context, mat: Matrix, op_scale: float, op_shift: float, a: float, b: float,
               coef: np.ndarray, X, xscale=None, Y=None, colss=None):
    """Y = psi_d(S) X diag(xscale); returns Y (torch, n x ncols)."""
    import torch
    ldx = _dev2d(X, "X")
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    if Y is None:
        Y = torch.empty_like(X)
    ldy = _dev2d(Y, "Y")
    st = load().arb_filter(ctx.handle, mat.handle, op_scale, op_shift, a, b, len(coef) - 1, coef.ctypes.data,
                           _vp(_ptr(X)), ldx, X.shape[1], _vp(_ptr(xscale)), _vp(_ptr(Y)), ldy,
                           _vp(_ptr(colss)))
    _check(ctx, st, "arb_filter")
    return Y


def arb_filter_df(ctx: Context, mat: Matrix, op_scale: float, op_shift: float, a: float, b: float,
                  coef: np.ndarray, X, xscale=None, Y=None, colss=None):
    """arb_filter computed in double-float arithmetic (X, Y: FP64 CUDA tensors)."""
    import torch
    ldx = _dev2d(X, "X")
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    if Y is None:
        Y = torch.empty_like(X)
    ldy = _dev2d(Y, "Y")
    st = load().arb_filter_df(ctx.handle, mat.handle, op_scale, op_shift, a, b, len(coef) - 1, coef.ctypes.data,
                              _vp(_ptr(X)), ldx, X.shape[1], _vp(_ptr(xscale)), _vp(_ptr(Y)), ldy,
                              _vp(_ptr(colss)))
    _check(ctx, st, "arb_filter_df")
    return Y


def arb_filter_f32(ctx: Context, mat: Matrix, op_scale: float, op_shift: float, a: float, b: float,
                   coef: np.ndarray, X, xscale=None, Y=None, colss=None):
    """FP32 variant of arb_filter (X, Y: row-major 2D float32 CUDA tensors)."""
    import torch
    if not (X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.stride(1) == 1):
        raise ValueError("X: expected a row-major 2D float32 CUDA tensor")
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    if Y is None:
        Y = torch.empty_like(X)
    st = load().arb_filter_f32(ctx.handle, mat.handle, op_scale, op_shift, a, b, len(coef) - 1, coef.ctypes.data,
                               _vp(_ptr(X)), X.stride(0), X.shape[1], _vp(_ptr(xscale)), _vp(_ptr(Y)), Y.stride(0),
                               _vp(_ptr(colss)))
    _check(ctx, st, "arb_filter_f32")
    return Y


def arb_spmm(ctx: Context, mat: Matrix, op_scale: float, op_shift: float, X, Y=None):
    import torch
    ldx = _dev2d(X, "X")
    if Y is None:
        Y = torch.empty_like(X)
    ldy = _dev2d(Y, "Y")
    _check(ctx, load().arb_spmm(ctx.handle, mat.handle, op_scale, op_shift, _vp(_ptr(X)), ldx, X.shape[1],
                                _vp(_ptr(Y)), ldy), "arb_spmm")
    return Y


def _gram_shapes(X, Y, C_out):
    """X^T Y needs X and Y with the same row count and, when given, C_out of shape
    (X columns, Y columns); checked before any pointer reaches the library, whose
    arguments carry no row count for Y and no row count for C."""
    if X.dim() != 2 or Y.dim() != 2:
        raise ValueError("X and Y must be 2D")
    if Y.shape[0] != X.shape[0]:
        raise ValueError(f"Y has {Y.shape[0]} rows, X has {X.shape[0]}")
    if C_out is not None and tuple(C_out.shape) != (X.shape[1], Y.shape[1]):
        raise ValueError(f"C_out must be {X.shape[1]} x {Y.shape[1]}, got {tuple(C_out.shape)}")


def arb_gram(ctx: Context, X, Y, C_out=None):
    import torch
    _gram_shapes(X, Y, C_out)
    ldx = _dev2d(X, "X")
    ldy = _dev2d(Y, "Y")
    if C_out is None:
        C_out = torch.empty((X.shape[1], Y.shape[1]), dtype=torch.float64, device=X.device)
    ldc = _dev2d(C_out, "C")
    _check(ctx, load().arb_gram(ctx.handle, X.shape[0], _vp(_ptr(X)), ldx, X.shape[1], _vp(_ptr(Y)), ldy,
                                Y.shape[1], _vp(_ptr(C_out)), ldc), "arb_gram")
    return C_out


def arb_gram_f32(ctx: Context, X, Y, C_out=None):
    """C = X^T Y for FP32 CUDA tensors (row-major 2D), FP64 result."""
    import torch
    _gram_shapes(X, Y, C_out)
    for name, T in (("X", X), ("Y", Y)):
        if not (T.is_cuda and T.dtype == torch.float32 and T.dim() == 2 and T.stride(1) == 1):
            raise ValueError(f"{name}: expected a row-major 2D float32 CUDA tensor")
    if C_out is None:
        C_out = torch.empty((X.shape[1], Y.shape[1]), dtype=torch.float64, device=X.device)
    ldc = _dev2d(C_out, "C")
    _check(ctx, load().arb_gram_f32(ctx.handle, X.shape[0], _vp(_ptr(X)), X.stride(0), X.shape[1], _vp(_ptr(Y)),
                                    Y.stride(0), Y.shape[1], _vp(_ptr(C_out)), ldc), "arb_gram_f32")
    return C_out


def arb_gemm_tall_f32(ctx: Context, In, W, alpha=1.0, beta=0.0, Out=None):
    """Out = alpha In W + beta Out: In, Out row-major 2D float32 CUDA tensors, W float64 (na x nb)."""
    import torch
    for name, T in (("In", In),) + ((("Out", Out),) if Out is not None else ()):
        if not (T.is_cuda and T.dtype == torch.float32 and T.dim() == 2 and T.stride(1) == 1):
            raise ValueError(f"{name}: expected a row-major 2D float32 CUDA tensor")
    ldw = _dev2d(W, "W")
    if Out is None:
        Out = torch.empty((In.shape[0], W.shape[1]), dtype=torch.float32, device=In.device)
    _check(ctx, load().arb_gemm_tall_f32(ctx.handle, In.shape[0], _vp(_ptr(In)), In.stride(0), In.shape[1],
                                         _vp(_ptr(W)), ldw, W.shape[1], alpha, beta, _vp(_ptr(Out)),
                                         Out.stride(0)), "arb_gemm_tall_f32")
    return Out


def arb_gram_noalloc(ctx: Context, X, Y, C_out):
    """C = X^T Y without any device allocation by the library (partial sums in its static
    scratch); C_out must be given."""
    if C_out is None:
        raise ValueError("C_out must be given (the call allocates nothing)")
    _gram_shapes(X, Y, C_out)
    ldx = _dev2d(X, "X")
    ldy = _dev2d(Y, "Y")
    ldc = _dev2d(C_out, "C")
    _check(ctx, load().arb_gram_noalloc(ctx.handle, X.shape[0], _vp(_ptr(X)), ldx, X.shape[1], _vp(_ptr(Y)), ldy,
                                        Y.shape[1], _vp(_ptr(C_out)), ldc), "arb_gram_noalloc")
    return C_out


def arb_syevj(ctx: Context, H):
    import torch
    ldh = _dev2d(H, "H")
    m = H.shape[0]
    w = torch.empty(m, dtype=torch.float64, device=H.device)
    V = torch.empty((m, m), dtype=torch.float64, device=H.device)
    sweeps = _i32()
    _check(ctx, load().arb_syevj(ctx.handle, m, _vp(_ptr(H)), ldh, _vp(_ptr(w)), _vp(_ptr(V)), m,
                                 C.byref(sweeps)), "arb_syevj")
    return w, V, sweeps.value


def arb_rcond_gram(ctx: Context, X, xscale=None) -> float:
    ldx = _dev2d(X, "X")
    rc = _dbl()
    _check(ctx, load().arb_rcond_gram(ctx.handle, X.shape[0], _vp(_ptr(X)), ldx, X.shape[1],
                                      _vp(_ptr(xscale)), C.byref(rc)), "arb_rcond_gram")
    return rc.value


def arb_orth(ctx: Context, Z):
    import torch
    ldz = _dev2d(Z, "Z")
    U = torch.empty_like(Z)
    r = _i32()
    _check(ctx, load().arb_orth(ctx.handle, Z.shape[0], _vp(_ptr(Z)), ldz, Z.shape[1], _vp(_ptr(U)),
                                U.stride(0), C.byref(r)), "arb_orth")
    return U[:, :r.value]


def arb_rayleigh_ritz(ctx: Context, mat: Matrix, op_scale: float, op_shift: float, Z):
    import torch
    ldz = _dev2d(Z, "Z")
    Y = torch.empty_like(Z)
    w = torch.empty(Z.shape[1], dtype=torch.float64, device=Z.device)
    r = _i32()
    _check(ctx, load().arb_rayleigh_ritz(ctx.handle, mat.handle, op_scale, op_shift, Z.shape[0], _vp(_ptr(Z)),
                                         ldz, Z.shape[1], _vp(_ptr(Y)), Y.stride(0), _vp(_ptr(w)), C.byref(r)),
           "arb_rayleigh_ritz")
    return Y[:, :r.value], w[:r.value]


def arb_arr(ctx: Context, mat: Matrix, op_scale: float, op_shift: float, X, q: int, npairs: int | None = None):
    import torch
    ldx = _dev2d(X, "X")
    npairs = X.shape[1] if npairs is None else npairs
    Y = torch.empty((X.shape[0], npairs), dtype=torch.float64, device=X.device)
    w = torch.empty(npairs, dtype=torch.float64, device=X.device)
    r = _i32()
    _check(ctx, load().arb_arr(ctx.handle, mat.handle, op_scale, op_shift, X.shape[0], _vp(_ptr(X)), ldx,
                               X.shape[1], q, npairs, _vp(_ptr(Y)), Y.stride(0), _vp(_ptr(w)), C.byref(r)),
           "arb_arr")
    return Y, w, r.value


def arb_server_footprint(n: int, nnz: int, p: int, q: int, precision: int = ARB_FP64) -> int:
    return int(load().arb_server_footprint(n, nnz, p, q, precision))


class Server:
    """Continuous-batching solve server (arb_server_*): submit() returns a ticket,
    wait() the result.  Matrices must outlive their requests."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 8 << 30, max_slots: int = 4):
        h = _vp()
        st = load().arb_server_create(device, hbm_budget_bytes, max_slots, C.byref(h))
        if st != ARB_OK:
            raise ArbError(st, "arb_server_create failed")
        self.handle = h
        self._meta = {}

    def submit(self, mat: Matrix, k: int, which: int, tol: float, opts: arb_options | None = None, x0=None,
               want_evecs: bool = True) -> int:
        if opts is None:
            opts = arb_options_default(k)
        ptr = 0
        if x0 is not None:
            x0 = np.ascontiguousarray(x0, dtype=np.float64)
            ptr = x0.ctypes.data
        t = _i64()
        st = load().arb_submit(self.handle, mat.handle, k, which, tol, C.byref(opts), _vp(ptr), int(want_evecs),
                               C.byref(t))
        if st != ARB_OK:
            raise ArbError(st, "arb_submit: " + load().arb_status_string(st).decode())
        self._meta[t.value] = (mat.n, k, want_evecs)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        n, k, want = self._meta[ticket]
        ev = np.zeros(k)
        vecs = np.zeros((k, n)) if want else None
        info = arb_info()
        lat = _dbl()
        st = load().arb_wait(self.handle, ticket, timeout_ms, ev.ctypes.data, _vp(vecs.ctypes.data if want else 0), n,
                             C.byref(info), C.byref(lat))
        if st == ARB_TIMEOUT:
            return None
        del self._meta[ticket]
        if st not in (ARB_OK, ARB_NOT_CONVERGED):
            raise ArbError(st, "arb_wait: " + load().arb_status_string(st).decode())
        return SolveResult(st, ev, vecs.T if want else None, dict(info.as_dict(), latency_s=lat.value))

    def close(self):
        if self.handle:
            load().arb_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def arb_filter_batched(ctx: Context, jobs: list[dict]):
    """Filter several instances in one launch.  Each job: dict(mat, op_scale, op_shift, a, b,
    coef (numpy), X (torch CUDA float32/float64, row-major, any leading dimension),
    xscale=None, colss=None, Y=None (preallocated output of X's shape)); returns the list
    of outputs Y."""
    import torch
    arr = (arb_filter_job * len(jobs))()
    keep, outs = [], []
    for i, j in enumerate(jobs):
        X = j["X"]
        if not (X.is_cuda and X.dim() == 2 and X.stride(1) == 1 and X.dtype in (torch.float32, torch.float64)):
            raise ValueError("X: row-major 2D float32/float64 CUDA tensor expected")
        coef = np.ascontiguousarray(j["coef"], dtype=np.float64)
        Y = j.get("Y")
        if Y is None:
            Y = torch.empty_like(X)
        elif not (Y.is_cuda and Y.dim() == 2 and Y.stride(1) == 1 and Y.dtype == X.dtype and Y.shape == X.shape):
            raise ValueError("Y: row-major 2D CUDA tensor of X's shape and type expected")
        keep += [coef, X, Y]
        outs.append(Y)
        arr[i] = arb_filter_job(j["mat"].handle, j["op_scale"], j["op_shift"], j["a"], j["b"], len(coef) - 1,
                                1 if X.dtype == torch.float32 else 0, coef.ctypes.data, X.data_ptr(), X.stride(0),
                                X.shape[1], 0, _ptr(j.get("xscale")), Y.data_ptr(), Y.stride(0), _ptr(j.get("colss")))
    _check(ctx, load().arb_filter_batched(ctx.handle, len(jobs), C.cast(arr, _vp)), "arb_filter_batched")
    return outs


def arb_solve_batched(ctx: Context, problems: list[dict], max_concurrent: int = 8, evecs: bool = True):
    """problems: dicts with mat, k, which, tol, opts (arb_options) and optional x0 (numpy).
    Returns (status, [SolveResult])."""
    nb = len(problems)
    mats = (_vp * nb)(*[p["mat"].handle.value for p in problems])
    ks = (_i32 * nb)(*[p["k"] for p in problems])
    wh = (_i32 * nb)(*[p["which"] for p in problems])
    tl = (_dbl * nb)(*[p["tol"] for p in problems])
    opts = (arb_options * nb)(*[p.get("opts") or arb_options_default(p["k"]) for p in problems])
    keep = []
    x0s = (_vp * nb)()
    for i, p in enumerate(problems):
        if p.get("x0") is not None:
            x = np.ascontiguousarray(p["x0"], dtype=np.float64)
            keep.append(x)
            x0s[i] = x.ctypes.data
    evs = [np.zeros(p["k"]) for p in problems]
    vecs = [np.zeros((p["k"], p["mat"].n)) for p in problems] if evecs else None
    evp = (_vp * nb)(*[e.ctypes.data for e in evs])
    vcp = (_vp * nb)(*[v.ctypes.data for v in vecs]) if evecs else None
    infos = (arb_info * nb)()
    st = load().arb_solve_batched(ctx.handle, nb, C.cast(mats, _vp), C.cast(ks, _vp), C.cast(wh, _vp),
                                  C.cast(tl, _vp), C.cast(opts, _vp), C.cast(x0s, _vp), C.cast(evp, _vp),
                                  C.cast(vcp, _vp) if evecs else None, None, C.cast(infos, _vp), max_concurrent)
    _check(ctx, st, "arb_solve_batched")
    return st, [SolveResult(ARB_OK, evs[i], vecs[i].T if evecs else None, infos[i].as_dict()) for i in range(nb)]


def _batch_args(problems, evecs):
    nb = len(problems)
    mats = (_vp * nb)(*[p["mat"].handle.value for p in problems])
    ks = (_i32 * nb)(*[p["k"] for p in problems])
    wh = (_i32 * nb)(*[p["which"] for p in problems])
    tl = (_dbl * nb)(*[p["tol"] for p in problems])
    opts = (arb_options * nb)(*[p.get("opts") or arb_options_default(p["k"]) for p in problems])
    keep = []
    x0s = (_vp * nb)()
    for i, p in enumerate(problems):
        if p.get("x0") is not None:
            x = np.ascontiguousarray(p["x0"], dtype=np.float64)
            keep.append(x)
            x0s[i] = x.ctypes.data
    evs = [np.zeros(p["k"]) for p in problems]
    vecs = [np.zeros((p["k"], p["mat"].n)) for p in problems] if evecs else None
    evp = (_vp * nb)(*[e.ctypes.data for e in evs])
    vcp = (_vp * nb)(*[v.ctypes.data for v in vecs]) if evecs else None
    return nb, mats, ks, wh, tl, opts, keep, x0s, evs, vecs, evp, vcp


def arb_solve_lockstep(ctx: Context, problems: list[dict], flags: int = ARB_BATCH_GRAPHS, evecs: bool = True):
    """Lock-step batched solve: problems as for arb_solve_batched.  Returns (status,
    [SolveResult], stats dict)."""
    nb, mats, ks, wh, tl, opts, keep, x0s, evs, vecs, evp, vcp = _batch_args(problems, evecs)
    infos = (arb_info * nb)()
    stats = arb_batch_stats()
    st = load().arb_solve_lockstep(ctx.handle, nb, C.cast(mats, _vp), C.cast(ks, _vp), C.cast(wh, _vp),
                                   C.cast(tl, _vp), C.cast(opts, _vp), C.cast(x0s, _vp), C.cast(evp, _vp),
                                   C.cast(vcp, _vp) if evecs else None, None, C.cast(infos, _vp), flags,
                                   C.byref(stats))
    _check(ctx, st, "arb_solve_lockstep")
    del keep
    return st, [SolveResult(ARB_OK, evs[i], vecs[i].T if evecs else None, infos[i].as_dict()) for i in range(nb)], \
        stats.as_dict()


def arb_matrix_autotune(ctx: Context, mat: Matrix, ncols: int) -> dict:
    """Time the fused SpMM layouts and widths on this matrix and keep the fastest:
    {"sell_C": C (0 = CSR), "vec": width, "ms": time per pass}."""
    choice = (_i32 * 2)()
    ms = _dbl()
    _check(ctx, load().arb_matrix_autotune(ctx.handle, mat.handle, ncols, C.cast(choice, _vp), C.byref(ms)),
           "arb_matrix_autotune")
    return {"sell_C": choice[0], "vec": choice[1], "ms": ms.value}
