"""Thin Python binding of liblt (include/lt.h): same names as the C ABI, argument
marshalling only.  Every computation runs in liblt's CUDA kernels; there is no fallback
of any kind -- if liblt.so is missing or fails to load, every call raises.

Tensors are torch CUDA tensors in the library layout: a contiguous tensor of shape
(IK, ..., I3, I2, I1) holds the column-major I1 x I2 x I3 x ... x IK tensor, so
I1 = t.shape[-1] and I2 = t.shape[-2].  Dtype float64 for LT_FP64 contexts, float32
for LT_FP32 / LT_MIXED.  Masks are uint8 tensors of the same shape.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblt.so")

LT_OK = 0
STATUS = {0: "LT_OK", -1: "LT_ERR_ARG", -2: "LT_ERR_SHAPE", -3: "LT_ERR_SINGULAR",
          -4: "LT_ERR_NOCONV", -5: "LT_ERR_TIMEOUT", -6: "LT_ERR_NONFINITE",
          -7: "LT_ERR_CUDA", -8: "LT_ERR_WORKSPACE", -9: "LT_ERR_UNSUPPORTED"}
STATUS_CODE = {name: code for code, name in STATUS.items()}
LT_DEV_NOCONV, LT_DEV_NONFINITE, LT_DEV_TIMEOUT = 1, 2, 4
LT_FP64, LT_FP32, LT_MIXED = 0, 1, 2
(LT_OP_TRANSFORM, LT_OP_INVERSE, LT_OP_PRODUCT, LT_OP_SVD, LT_OP_SVT, LT_OP_PGA, LT_OP_TRUNCATE,
 LT_OP_NORMS) = range(8)
(LT_OPT_MAX_SWEEPS, LT_OPT_JACOBI_TOL, LT_OPT_OBJECTIVE, LT_OPT_PROFILE, LT_OPT_JACOBI_GROUP,
 LT_OPT_JACOBI_BLOCK, LT_OPT_TC_MODE_MIN, LT_OPT_TC_TILE_N, LT_OPT_MU0, LT_OPT_NU,
 LT_OPT_JACOBI_CLUSTER, LT_OPT_TC_WAIT_US, LT_OPT_TC_TEST_NO_LOADS, LT_OPT_WARM_START,
 LT_OPT_AUTOTUNE, LT_OPT_TRANSFORM_TMA) = range(16)
LT_K_TRANSFORM, LT_K_JACOBI, LT_K_GEMM, LT_K_AUX = 0, 1, 2, 3
KERNEL_FAMILIES = ("transform", "jacobi", "gemm", "aux")

# Every entry point of include/lt.h: name -> (restype, argtypes)
_vp, _i64, _dbl, _sz = C.c_void_p, C.c_int64, C.c_double, C.c_size_t


class lt_pga_state(C.Structure):
    _fields_ = [("X_prev", C.c_void_p), ("t_prev", C.c_double), ("t", C.c_double),
                ("k", C.c_int64)]


class lt_pga_report(C.Structure):
    _fields_ = [("iters_done", C.c_int64), ("rel_residual", C.c_double),
                ("objective", C.c_double), ("max_sweeps_used", C.c_int32),
                ("device_status", C.c_int32)]


class lt_kernel_stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("ms", C.c_double), ("flops", C.c_double),
                ("bytes", C.c_double)]


class lt_tune_report(C.Structure):
    _fields_ = [("jacobi_group", C.c_int32), ("jacobi_block", C.c_int32),
                ("tc_tile_n", C.c_int32), ("candidates", C.c_int32),
                ("best_ms", C.c_double), ("default_ms", C.c_double)]


class lt_stats(C.Structure):
    _fields_ = [("k", lt_kernel_stats * 4), ("jacobi_phase_cycles", C.c_double * 10),
                ("tc_launches", C.c_int64)]


SIGNATURES = {
    "lt_make_dct": (C.c_int, [_i64, C.POINTER(C.c_double)]),
    "lt_make_cproduct": (C.c_int, [_i64, C.POINTER(C.c_double)]),
    "lt_ctx_create": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.POINTER(C.c_double)),
                                C.c_int, C.POINTER(C.c_void_p)]),
    "lt_ctx_create_fourier": (C.c_int, [C.c_int, C.POINTER(C.c_int64),
                                        C.POINTER(C.POINTER(C.c_double)), C.c_int,
                                        C.POINTER(C.c_void_p)]),
    "lt_ctx_destroy": (C.c_int, [_vp]),
    "lt_ctx_set_option": (C.c_int, [_vp, C.c_int, _dbl]),
    "lt_workspace_size": (C.c_int, [_vp, C.c_int, _i64, _i64, _i64, C.POINTER(C.c_size_t)]),
    "lt_transform": (C.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _sz, _vp]),
    "lt_inverse": (C.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _sz, _vp]),
    "lt_product": (C.c_int, [_vp, _i64, _i64, _i64, _vp, _vp, _vp, _vp, _sz, _vp]),
    "lt_svd": (C.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "lt_svt": (C.c_int, [_vp, _i64, _i64, _vp, _dbl, _vp, _vp, _sz, _vp]),
    "lt_pga_complete": (C.c_int, [_vp, _i64, _i64, _vp, _vp, _dbl, _dbl, _i64, _dbl, _vp,
                                  C.POINTER(lt_pga_state), C.POINTER(lt_pga_report), _vp, _sz,
                                  _vp]),
    "lt_workspace_size_batched": (C.c_int, [C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                            C.POINTER(C.c_int64), C.POINTER(C.c_size_t)]),
    "lt_pga_complete_batched": (C.c_int, [C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                          C.POINTER(C.c_int64), C.POINTER(C.c_void_p),
                                          C.POINTER(C.c_void_p), C.POINTER(C.c_double),
                                          C.POINTER(C.c_double), _i64, C.POINTER(C.c_void_p),
                                          C.POINTER(lt_pga_report), _vp, _sz, _vp]),
    "lt_product_noalloc": (C.c_int, [_vp, _i64, _i64, _i64, _vp, _vp, _vp, _vp]),
    "lt_truncate": (C.c_int, [_vp, _i64, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "lt_autotune_svt": (C.c_int, [_vp, _i64, _i64, _vp, _dbl, _vp, _vp, _sz, _vp,
                                  C.POINTER(lt_tune_report)]),
    "lt_autotune_product": (C.c_int, [_vp, _i64, _i64, _i64, _vp, _vp, _vp, _vp, _sz, _vp,
                                      C.POINTER(lt_tune_report)]),
    "lt_norms": (C.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _sz, _vp]),
    "lt_ctx_get_stats": (C.c_int, [_vp, C.POINTER(lt_stats), C.c_int]),
    "lt_last_device_status": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
    "lt_status_string": (C.c_char_p, [C.c_int]),
    "lt_measure_fma_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double), _vp]),
}

_lib: Optional[C.CDLL] = None


class LtError(RuntimeError):
    def __init__(self, fn, status):
        super().__init__(f"{fn} failed: {STATUS.get(status, status)}")
        self.status = status


def lib() -> C.CDLL:
    """Load liblt.so (built in-tree by paper_2202_02870_gb300.build).  Raises when the
    library is absent: nothing in this package runs without it."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"liblt.so not found at {LIB_PATH}; build it with "
                               "`python -m paper_2202_02870_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(fn, status):
    if status != LT_OK:
        raise LtError(fn, status)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- transform matrices
def lt_make_dct(n: int) -> np.ndarray:
    M = np.empty((n, n), dtype=np.float64)
    _check("lt_make_dct", lib().lt_make_dct(n, M.ctypes.data_as(C.POINTER(C.c_double))))
    return M


def lt_make_cproduct(n: int) -> np.ndarray:
    M = np.empty((n, n), dtype=np.float64)
    _check("lt_make_cproduct", lib().lt_make_cproduct(n, M.ctypes.data_as(C.POINTER(C.c_double))))
    return M


# ---------------------------------------------------------------- context
class Context:
    """Owns an lt_ctx (the operator L with matrices M_3..M_K)."""

    def __init__(self, mode_sizes: Sequence[int], matrices: Sequence[np.ndarray],
                 precision: int = LT_FP64, fourier: bool = False):
        """fourier=True: M_3 = F_{I3} (lt_ctx_create_fourier) and `matrices` holds
        M_4..M_K only."""
        sizes = (C.c_int64 * len(mode_sizes))(*[int(s) for s in mode_sizes])
        self._mats = [np.ascontiguousarray(m, dtype=np.float64) for m in matrices]
        ptrs = (C.POINTER(C.c_double) * max(1, len(self._mats)))(
            *[m.ctypes.data_as(C.POINTER(C.c_double)) for m in self._mats])
        h = C.c_void_p()
        if fourier:
            _check("lt_ctx_create_fourier", lib().lt_ctx_create_fourier(
                len(mode_sizes) + 2, sizes, ptrs if self._mats else None, int(precision),
                C.byref(h)))
        else:
            _check("lt_ctx_create", lib().lt_ctx_create(len(mode_sizes) + 2, sizes, ptrs,
                                                        int(precision), C.byref(h)))
        self.handle = h
        self.fourier = bool(fourier)
        self.mode_sizes = tuple(int(s) for s in mode_sizes)
        self.precision = int(precision)
        self.P = int(np.prod(self.mode_sizes))

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == LT_FP64 else torch.float32

    def close(self):
        if self.handle:
            lib().lt_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lt_ctx_create(mode_sizes, matrices, precision=LT_FP64) -> Context:
    return Context(mode_sizes, matrices, precision)


def lt_ctx_create_fourier(mode_sizes, matrices_rest=(), precision=LT_FP64) -> Context:
    """Context of the Fourier operator: M_3 = F_{I3}, M_4.. = matrices_rest."""
    return Context(mode_sizes, matrices_rest, precision, fourier=True)


def lt_ctx_destroy(ctx: Context):
    ctx.close()


def lt_ctx_set_option(ctx: Context, opt: int, value: float):
    _check("lt_ctx_set_option", lib().lt_ctx_set_option(ctx.handle, int(opt), float(value)))


def lt_workspace_size(ctx: Context, op: int, I1: int, I2: int, I2b: int = 0) -> int:
    out = C.c_size_t()
    _check("lt_workspace_size", lib().lt_workspace_size(ctx.handle, int(op), I1, I2, I2b,
                                                        C.byref(out)))
    return int(out.value)


def _workspace(ctx, nbytes, device, ws):
    if nbytes == 0:
        return ws, 0
    if ws is None:
        import torch
        ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
    return ws, int(ws.numel() * ws.element_size())


def _dims(t):
    return int(t.shape[-1]), int(t.shape[-2])


def _require(t, ctx, what):
    if not t.is_cuda or not t.is_contiguous() or t.dtype != ctx.dtype:
        raise ValueError(f"{what}: expected a contiguous CUDA {ctx.dtype} tensor")


# ---------------------------------------------------------------- operations
def lt_transform(ctx, X, X_hat, ws=None, stream=None):
    _require(X, ctx, "X"); _require(X_hat, ctx, "X_hat")
    I1, I2 = _dims(X)
    _check("lt_transform", lib().lt_transform(ctx.handle, I1, I2, _ptr(X), _ptr(X_hat),
                                              None, 0, _stream(stream)))
    return X_hat


def lt_inverse(ctx, X_hat, X, ws=None, stream=None):
    _require(X, ctx, "X"); _require(X_hat, ctx, "X_hat")
    I1, I2 = _dims(X)
    _check("lt_inverse", lib().lt_inverse(ctx.handle, I1, I2, _ptr(X_hat), _ptr(X),
                                          None, 0, _stream(stream)))
    return X


def lt_product(ctx, A, B, Cout, ws=None, stream=None):
    for t, n in ((A, "A"), (B, "B"), (Cout, "C")):
        _require(t, ctx, n)
    I1, l = _dims(A)
    l2, I2 = _dims(B)
    if l2 != l:
        raise ValueError("inner sizes of A and B differ")
    need = lt_workspace_size(ctx, LT_OP_PRODUCT, I1, l, I2)
    ws, nb = _workspace(ctx, need, A.device, ws)
    _check("lt_product", lib().lt_product(ctx.handle, I1, l, I2, _ptr(A), _ptr(B), _ptr(Cout),
                                          _ptr(ws), nb, _stream(stream)))
    return Cout


LT_NOALLOC_SCRATCH_BYTES = 32 << 20


def lt_product_noalloc(ctx, A, B, Cout, stream=None):
    """lt_product for callers that cannot allocate: no workspace argument; the library
    uses its fixed LT_NOALLOC_SCRATCH_BYTES device array (see include/lt.h)."""
    for t, n in ((A, "A"), (B, "B"), (Cout, "C")):
        _require(t, ctx, n)
    I1, l = _dims(A)
    l2, I2 = _dims(B)
    if l2 != l:
        raise ValueError("inner sizes of A and B differ")
    _check("lt_product_noalloc", lib().lt_product_noalloc(ctx.handle, I1, l, I2, _ptr(A), _ptr(B),
                                                          _ptr(Cout), _stream(stream)))
    return Cout


def lt_svd(ctx, A, U, S, V, sigma=None, ws=None, stream=None):
    for t, n in ((A, "A"), (U, "U"), (S, "S"), (V, "V")):
        _require(t, ctx, n)
    I1, I2 = _dims(A)
    need = lt_workspace_size(ctx, LT_OP_SVD, I1, I2)
    ws, nb = _workspace(ctx, need, A.device, ws)
    _check("lt_svd", lib().lt_svd(ctx.handle, I1, I2, _ptr(A), _ptr(U), _ptr(S), _ptr(V),
                                  _ptr(sigma), _ptr(ws), nb, _stream(stream)))
    return U, S, V


def lt_svt(ctx, A, tau, D, ws=None, stream=None):
    _require(A, ctx, "A"); _require(D, ctx, "D")
    I1, I2 = _dims(A)
    need = lt_workspace_size(ctx, LT_OP_SVT, I1, I2)
    ws, nb = _workspace(ctx, need, A.device, ws)
    _check("lt_svt", lib().lt_svt(ctx.handle, I1, I2, _ptr(A), float(tau), _ptr(D),
                                  _ptr(ws), nb, _stream(stream)))
    return D


def lt_truncate(ctx, A, k, A_k, ws=None, stream=None):
    _require(A, ctx, "A"); _require(A_k, ctx, "A_k")
    I1, I2 = _dims(A)
    need = lt_workspace_size(ctx, LT_OP_TRUNCATE, I1, I2)
    ws, nb = _workspace(ctx, need, A.device, ws)
    _check("lt_truncate", lib().lt_truncate(ctx.handle, I1, I2, _ptr(A), int(k), _ptr(A_k),
                                            _ptr(ws), nb, _stream(stream)))
    return A_k


def lt_norms(ctx, A, out, multirank=None, ws=None, stream=None):
    """out: CUDA float64 tensor of 4 (nuclear sum, spectral, tubal rank, average rank);
    multirank: CUDA int32 tensor of P or None."""
    _require(A, ctx, "A")
    import torch
    if not out.is_cuda or out.dtype != torch.float64 or out.numel() < 4:
        raise ValueError("out: expected a CUDA float64 tensor of 4 elements")
    if multirank is not None and (not multirank.is_cuda or multirank.dtype != torch.int32):
        raise ValueError("multirank: expected a CUDA int32 tensor")
    I1, I2 = _dims(A)
    need = lt_workspace_size(ctx, LT_OP_NORMS, I1, I2)
    ws, nb = _workspace(ctx, need, A.device, ws)
    _check("lt_norms", lib().lt_norms(ctx.handle, I1, I2, _ptr(A), _ptr(out), _ptr(multirank),
                                      _ptr(ws), nb, _stream(stream)))
    return out


def lt_pga_complete(ctx, mask, obs, tau, step, iters, X, tol=0.0, state=None, report=None,
                    ws=None, stream=None):
    """X: in = start (zeros for a cold start), out = the last iterate.  `state` and
    `report` are lt_pga_state / lt_pga_report ctypes structures (or None); they are
    filled once the stream reaches the end of the call's work."""
    _require(obs, ctx, "obs"); _require(X, ctx, "X")
    if mask.dtype.itemsize != 1 or not mask.is_cuda or not mask.is_contiguous():
        raise ValueError("mask: expected a contiguous CUDA uint8 tensor")
    I1, I2 = _dims(X)
    need = lt_workspace_size(ctx, LT_OP_PGA, I1, I2)
    ws, nb = _workspace(ctx, need, X.device, ws)
    _check("lt_pga_complete", lib().lt_pga_complete(
        ctx.handle, I1, I2, _ptr(mask), _ptr(obs), float(tau), float(step), int(iters),
        float(tol), _ptr(X), C.byref(state) if state is not None else None,
        C.byref(report) if report is not None else None, _ptr(ws), nb, _stream(stream)))
    return X


def lt_workspace_size_batched(ctxs, I1s, I2s) -> int:
    n = len(ctxs)
    out = C.c_size_t()
    _check("lt_workspace_size_batched", lib().lt_workspace_size_batched(
        n, (C.c_void_p * n)(*[c.handle.value for c in ctxs]), (C.c_int64 * n)(*I1s),
        (C.c_int64 * n)(*I2s), C.byref(out)))
    return int(out.value)


def lt_pga_complete_batched(ctxs, masks, obss, taus, steps, iters, Xs, reports=None,
                            ws=None, stream=None):
    n = len(ctxs)
    I1s = [int(x.shape[-1]) for x in Xs]
    I2s = [int(x.shape[-2]) for x in Xs]
    need = lt_workspace_size_batched(ctxs, I1s, I2s)
    ws, nb = _workspace(ctxs[0], need, Xs[0].device, ws)
    rep_arr = (lt_pga_report * n)() if reports is not None else None
    _check("lt_pga_complete_batched", lib().lt_pga_complete_batched(
        n, (C.c_void_p * n)(*[c.handle.value for c in ctxs]), (C.c_int64 * n)(*I1s),
        (C.c_int64 * n)(*I2s), (C.c_void_p * n)(*[m.data_ptr() for m in masks]),
        (C.c_void_p * n)(*[o.data_ptr() for o in obss]), (C.c_double * n)(*taus),
        (C.c_double * n)(*steps), int(iters), (C.c_void_p * n)(*[x.data_ptr() for x in Xs]),
        rep_arr, _ptr(ws), nb, _stream(stream)))
    if reports is not None:
        reports.append(rep_arr)
    return Xs


def lt_autotune_svt(ctx, A, tau, D, ws=None, stream=None) -> lt_tune_report:
    """Times the SVT kernel forms on A and sets the fastest on the context."""
    _require(A, ctx, "A"); _require(D, ctx, "D")
    I1, I2 = _dims(A)
    need = lt_workspace_size(ctx, LT_OP_SVT, I1, I2)
    ws, nb = _workspace(ctx, need, A.device, ws)
    rep = lt_tune_report()
    _check("lt_autotune_svt", lib().lt_autotune_svt(ctx.handle, I1, I2, _ptr(A), float(tau), _ptr(D),
                                                    _ptr(ws), nb, _stream(stream), C.byref(rep)))
    return rep


def lt_autotune_product(ctx, A, B, Cout, ws=None, stream=None) -> lt_tune_report:
    """Times the tensor-core tile widths of lt_product on A, B and sets the fastest."""
    for t, n in ((A, "A"), (B, "B"), (Cout, "C")):
        _require(t, ctx, n)
    I1, l = _dims(A)
    _, I2 = _dims(B)
    need = lt_workspace_size(ctx, LT_OP_PRODUCT, I1, l, I2)
    ws, nb = _workspace(ctx, need, A.device, ws)
    rep = lt_tune_report()
    _check("lt_autotune_product", lib().lt_autotune_product(
        ctx.handle, I1, l, I2, _ptr(A), _ptr(B), _ptr(Cout), _ptr(ws), nb, _stream(stream),
        C.byref(rep)))
    return rep


def lt_ctx_get_stats(ctx, reset: bool = False) -> dict:
    """Per kernel family: launches, summed event ms (LT_OPT_PROFILE), algorithmic flops
    and bytes."""
    st = lt_stats()
    _check("lt_ctx_get_stats", lib().lt_ctx_get_stats(ctx.handle, C.byref(st), int(bool(reset))))
    out = {name: {"launches": int(st.k[i].launches), "ms": float(st.k[i].ms),
                  "flops": float(st.k[i].flops), "bytes": float(st.k[i].bytes)}
           for i, name in enumerate(KERNEL_FAMILIES)}
    out["jacobi_phase_cycles"] = dict(zip(("load", "qr", "sweeps", "select", "coefficients",
                                           "rows", "qr_pivot", "qr_swap", "qr_householder",
                                           "qr_update"),
                                          [float(v) for v in st.jacobi_phase_cycles]))
    out["tc_launches"] = int(st.tc_launches)
    return out


def lt_last_device_status(ctx) -> int:
    out = C.c_int32()
    _check("lt_last_device_status", lib().lt_last_device_status(ctx.handle, C.byref(out)))
    return int(out.value)


def lt_status_string(s: int) -> str:
    return lib().lt_status_string(int(s)).decode()


def lt_measure_fma_peak(precision: int, stream=None) -> float:
    """FMA throughput of the current GPU in GFLOP/s (LT_FP64 or LT_FP32)."""
    out = C.c_double()
    _check("lt_measure_fma_peak", lib().lt_measure_fma_peak(int(precision), C.byref(out),
                                                            _stream(stream)))
    return float(out.value)
