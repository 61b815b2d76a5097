"""ctypes binding of ``libgb300rbt.so`` (argument marshalling only).

Every function here has the name of the C entry point it calls (see
``include/rbt.h``) and converts torch CUDA tensors to device pointers,
leading dimensions and the current CUDA stream.  All arithmetic happens in the
library's kernels; if the library cannot be loaded, every call raises.

Matrix convention: a matrix argument is a 2-D CUDA tensor in column-major
layout, i.e. ``t.stride(0) == 1`` and leading dimension ``t.stride(1)`` (a
Fortran-ordered view such as ``torch.empty(cols, ld).T[:rows]``); a vector is
a 1-D contiguous tensor (one column, leading dimension = its length).
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _build

RBT_OK = 0
RBT_ERR_ARG = -1
RBT_ERR_CUDA = -2
RBT_ERR_WORKSPACE = -3
RBT_ERR_TIMEOUT = -4
RBT_ERR_UNSUPPORTED = -5
RBT_ZERO_PIVOT = 1
RBT_NONFINITE = 2
RBT_NOT_CONVERGED = 3

PREC = {"f64": 0, "f32": 1, "tf32": 2, "bf16": 3, "df64": 4, "df64tc": 5, "df64tc7": 6}
# storage dtype of a working matrix per precision (df64: float pairs held as float64-sized slots,
# exposed to Python as a float32 tensor of twice the rows, hi then lo of each element)
PREC_DTYPE = {0: torch.float64, 1: torch.float32, 2: torch.float32, 3: torch.float32, 4: torch.float64, 5: torch.float64,
              6: torch.float64}


class RbtError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__("%s failed: %s (%d)" % (fn, msg, code))
        self.code = code


class rbt_opts(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("seed", ctypes.c_uint64), ("prec", ctypes.c_int32),
                ("refine_max", ctypes.c_int32), ("tol", ctypes.c_double), ("fallback", ctypes.c_int32),
                ("nb", ctypes.c_int32), ("align", ctypes.c_int64), ("refine_mode", ctypes.c_int32),
                ("restart", ctypes.c_int32), ("kind", ctypes.c_int32), ("grid_p", ctypes.c_int32),
                ("grid_q", ctypes.c_int32)]


class rbt_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("zero_pivot", ctypes.c_int64), ("iters", ctypes.c_int32),
                ("fell_back", ctypes.c_int32), ("berr_unrefined", ctypes.c_double), ("berr", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
LIB_PATH = _build.LIB

_I64, _I32, _U64, _P, _SZ, _D = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p,
                                 ctypes.c_size_t, ctypes.c_double)
_SIGS = {
    "rbt_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rbt_reference_size": (_I64, [_I64, _I32, _I64, _I32, _I32]),
    "rbt_generate": (_I32, [_I64, _I32, _U64, _P, _P, _I64, _P]),
    "rbt_apply_2sided": (_I32, [_I64, _I32, _P, _P, _I64, _P, _I64, _P, _I64, _P]),
    "rbt_apply_2sided_wp": (_I32, [_I64, _I32, _P, _P, _I64, _P, _I64, _P, _I64, _I32, _P]),
    "rbt_apply_2sided_layered": (_I32, [_I64, _I32, _P, _P, _I64, _P, _I64, _P]),
    "rbt_apply_vec": (_I32, [_I64, _I32, _P, _I64, _I32, _P, _I64, _I64, _P]),
    "rbt_apply_2sided_tiled": (_I32, [_I64, _I32, _I64, _P, _P, _I64, _P, _I64, _P, _I64, _P]),
    "rbt_apply_vec_tiled": (_I32, [_I64, _I32, _I64, _P, _I64, _I32, _P, _I64, _I64, _P]),
    "rbt_generate_rot": (_I32, [_I64, _I32, _I64, _U64, _P, _P, _I64, _P]),
    "rbt_transform_2sided": (_I32, [_I64, _I32, _I64, _I32, _I32, _P, _P, _I64, _P, _I64, _P, _I64, _P]),
    "rbt_transform_vec": (_I32, [_I64, _I32, _I64, _I32, _P, _I64, _I32, _P, _I64, _I64, _P]),
    "genp_factor_workspace": (_SZ, [_I64, _I32, _I32]),
    "genp_factor": (_I32, [_I64, _I32, _P, _I64, _P, _P, _SZ, _I32, _P]),
    "genp_update_workspace": (_SZ, [_I64, _I64, _I64, _I32]),
    "genp_update": (_I32, [_I32, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _P, _SZ, _P]),
    "genp_solve_workspace": (_SZ, [_I64, _I64, _I32]),
    "genp_solve": (_I32, [_I64, _I64, _I32, _P, _I64, _I32, _P, _I64, _P, _SZ, _P]),
    "genp_solve_wp_workspace": (_SZ, [_I64, _I64]),
    "genp_solve_wp": (_I32, [_I64, _I64, _I32, _P, _I64, _I32, _P, _I64, _P, _SZ, _P]),
    "rbt_residual_workspace": (_SZ, [_I64, _I64]),
    "rbt_residual": (_I32, [_I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _P, _P, _SZ, _P]),
    "rbt_norm_inf": (_I32, [_I64, _P, _I64, _P, _P, _SZ, _P]),
    "rbt_residual_noalloc_max_bytes": (_SZ, []),
    "rbt_residual_noalloc": (_I32, [_I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _P, _P]),
    "rbt_solve_batched_workspace": (_SZ, [ctypes.POINTER(rbt_opts), _I64, _P, _P]),
    "rbt_solve_batched_plan": (_I32, [ctypes.POINTER(rbt_opts), _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ,
                                      _P]),
    "rbt_solve_batched_run": (_I32, [ctypes.POINTER(rbt_opts), _P, _P, _P]),
    "rbt_solve_batched_autotune": (_I32, [ctypes.POINTER(rbt_opts), _P, _P, _P, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_double)]),
    "rbt_solve_batched_variant": (_I32, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "rbt_solve_batched_adjoint": (_I32, [ctypes.POINTER(rbt_opts), _P, _I64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "rbt_solve_adjoint": (_I32, [ctypes.POINTER(rbt_opts), ctypes.POINTER(rbt_info), _I64, _I64, _P, _I64, _P, _I64,
                                 _P, _I64, _P, _SZ, ctypes.POINTER(rbt_info), _P]),
    "rbt_outer": (_I32, [_I64, _I64, _I64, _D, _P, _I64, _P, _I64, _P, _I64, _P]),
    "rbt_kernel_launches": (_U64, []),
    "rbt_debug_wait_limit": (_I64, [_I64]),
    "rbt_debug_stall": (_I32, [_I32]),
    "rbt_debug_oz_products_workspace": (_SZ, [_I64, _I64, _I64]),
    "rbt_debug_oz_products": (_I32, [_I64, _I64, _I64, _P, _P, _P, _P, _SZ, _P]),
    "rbt_prof_enable": (None, [_I32]),
    "rbt_prof_reset": (None, []),
    "rbt_prof_read": (_I32, [_I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    "rbt_solve_workspace": (_SZ, [ctypes.POINTER(rbt_opts), _I64, _I64]),
    "rbt_solve_host_workspace": (_SZ, [ctypes.POINTER(rbt_opts), _I64, _I64]),
    "rbt_solve_host": (_I32, [ctypes.POINTER(rbt_opts), _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _SZ,
                              ctypes.POINTER(rbt_info), _P]),
    "rbt_solve": (_I32, [ctypes.POINTER(rbt_opts), _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _SZ,
                         ctypes.POINTER(rbt_info), _P]),
}


def declared_symbols():
    """Names of the entry points this binding declares."""
    return list(_SIGS)


def load(build: bool = True):
    """Load (building first if needed) the CUDA library; raises if impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libgb300rbt.so is missing (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(fn, code, ok=(RBT_OK,)):
    if code not in ok:
        msg = load().rbt_status_string(code).decode()
        raise RbtError(fn, code, msg)
    return code


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _mat(t, name, dtype=None, host=False):
    """(pointer, ld, rows, cols) of a column-major CUDA matrix or a vector
    (host=True: of a CPU tensor)."""
    if not isinstance(t, torch.Tensor) or t.is_cuda == host:
        raise TypeError("%s must be a %s tensor" % (name, "CPU" if host else "CUDA"))
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    if t.dim() == 1:
        if t.stride(0) != 1 and t.numel() > 1:
            raise ValueError("%s must be contiguous" % name)
        return ctypes.c_void_p(t.data_ptr()), max(1, t.shape[0]), t.shape[0], 1
    if t.dim() != 2:
        raise ValueError("%s must be 1-D or 2-D" % name)
    rows, cols = t.shape
    if cols > 1 and rows > 1 and t.stride(0) != 1:
        raise ValueError("%s must be column-major (stride(0) == 1)" % name)
    ld = t.stride(1) if cols > 1 else max(1, rows)
    if rows > 1 and cols == 1 and t.stride(0) != 1:
        raise ValueError("%s must be column-major (stride(0) == 1)" % name)
    return ctypes.c_void_p(t.data_ptr()), max(ld, 1), rows, cols


def colmajor(rows, cols, dtype=torch.float64, device="cuda", ld=None):
    """Uninitialized column-major CUDA matrix (rows x cols, leading dimension ld)."""
    ld = rows if ld is None else ld
    return torch.empty((cols, max(ld, 1)), dtype=dtype, device=device).T[:rows]


def to_device(a, device="cuda"):
    """Column-major CUDA copy of a numpy array (1-D or 2-D)."""
    import numpy as np
    a = np.asarray(a)
    if a.ndim == 1:
        return torch.from_numpy(np.ascontiguousarray(a)).to(device)
    return torch.from_numpy(np.ascontiguousarray(a.T)).to(device).T


def to_host(t):
    import numpy as np
    a = t.detach().cpu()
    if a.dim() == 1:
        return a.numpy().copy()
    return np.asfortranarray(a.numpy())


# ------------------------------------------------------------------ entry points

def rbt_generate(n, d, seed, U, V, stream=None):
    pu, ldu, _, _ = _mat(U, "U", torch.float64)
    pv, ldv, _, _ = _mat(V, "V", torch.float64)
    if ldu != ldv:
        raise ValueError("U and V must share a leading dimension")
    return _check("rbt_generate", load().rbt_generate(n, d, seed & (2**64 - 1), pu, pv, ldu, _stream(stream)))


def rbt_apply_2sided_wp(n, d, U, V, A_in, A_out, prec, stream=None):
    """Working copy of U^T A V in precision prec.  For "df64" A_out is a float64-typed
    column-major tensor whose 8-byte slots hold the float pair (hi, lo)."""
    prec = PREC.get(prec, prec)
    pu, ldw, _, _ = _mat(U, "U", torch.float64)
    pv, _, _, _ = _mat(V, "V", torch.float64)
    pa, lda, _, _ = _mat(A_in, "A_in", torch.float64)
    po, ldo, _, _ = _mat(A_out, "A_out", PREC_DTYPE[prec])
    return _check("rbt_apply_2sided_wp", load().rbt_apply_2sided_wp(n, d, pu, pv, ldw, pa, lda, po, ldo, prec,
                                                                    _stream(stream)))


def df64_to_double(t):
    """Value of a df64 working matrix (float64-typed slots holding float pairs) as float64."""
    pairs = t.contiguous().view(torch.float32) if t.dim() == 1 else None
    if pairs is None:
        cols = t.T.contiguous()                      # (cols, rows) slots
        f = cols.view(torch.float32).reshape(cols.shape[0], cols.shape[1], 2)
        return (f[..., 0].double() + f[..., 1].double()).T
    f = pairs.reshape(-1, 2)
    return f[:, 0].double() + f[:, 1].double()


def rbt_apply_2sided(n, d, U, V, A_in, A_out=None, stream=None):
    A_out = A_in if A_out is None else A_out
    pu, ldw, _, _ = _mat(U, "U", torch.float64)
    pv, _, _, _ = _mat(V, "V", torch.float64)
    pa, lda, _, _ = _mat(A_in, "A_in", torch.float64)
    if A_out.dtype == torch.float32:
        return rbt_apply_2sided_wp(n, d, U, V, A_in, A_out, "f32", stream)
    po, ldo, _, _ = _mat(A_out, "A_out", torch.float64)
    return _check("rbt_apply_2sided", load().rbt_apply_2sided(n, d, pu, pv, ldw, pa, lda, po, ldo, _stream(stream)))


def rbt_apply_2sided_tiled(n, d, align, U, V, A_in, A_out=None, stream=None):
    """A_out <- U^T A_in V with the tiled reference size (align = tile size n_b)."""
    A_out = A_in if A_out is None else A_out
    pu, ldw, _, _ = _mat(U, "U", torch.float64)
    pv, _, _, _ = _mat(V, "V", torch.float64)
    pa, lda, _, _ = _mat(A_in, "A_in", torch.float64)
    po, ldo, _, _ = _mat(A_out, "A_out", torch.float64)
    return _check("rbt_apply_2sided_tiled", load().rbt_apply_2sided_tiled(n, d, align, pu, pv, ldw, pa, lda, po, ldo,
                                                                          _stream(stream)))


def rbt_apply_vec_tiled(n, d, align, W, trans, B, stream=None):
    pw, ldw, _, _ = _mat(W, "W", torch.float64)
    pb, ldb, _, nrhs = _mat(B, "B", torch.float64)
    return _check("rbt_apply_vec_tiled", load().rbt_apply_vec_tiled(n, d, align, pw, ldw, 1 if trans else 0, pb, ldb,
                                                                    nrhs, _stream(stream)))


def rbt_apply_2sided_layered(n, d, U, V, A, stream=None):
    pu, ldw, _, _ = _mat(U, "U", torch.float64)
    pv, _, _, _ = _mat(V, "V", torch.float64)
    pa, lda, _, _ = _mat(A, "A", torch.float64)
    return _check("rbt_apply_2sided_layered", load().rbt_apply_2sided_layered(n, d, pu, pv, ldw, pa, lda,
                                                                              _stream(stream)))


def rbt_generate_rot(n, d, align, seed, U, V, stream=None):
    """Packed coefficients of the rotation-form butterflies (cos / sin per pair, 1 elsewhere)."""
    pu, ldu, _, _ = _mat(U, "U", torch.float64)
    pv, ldv, _, _ = _mat(V, "V", torch.float64)
    if ldu != ldv:
        raise ValueError("U and V must share a leading dimension")
    return _check("rbt_generate_rot", load().rbt_generate_rot(n, d, align, seed & (2**64 - 1), pu, pv, ldu,
                                                              _stream(stream)))


def rbt_transform_2sided(n, d, align, kind, prec, U, V, A_in, A_out, stream=None):
    """U^T A V for either butterfly kind, written in precision prec."""
    prec = PREC.get(prec, prec)
    pu, ldw, _, _ = _mat(U, "U", torch.float64)
    pv, _, _, _ = _mat(V, "V", torch.float64)
    pa, lda, _, _ = _mat(A_in, "A_in", torch.float64)
    po, ldo, _, _ = _mat(A_out, "A_out", PREC_DTYPE[prec])
    return _check("rbt_transform_2sided", load().rbt_transform_2sided(n, d, align, KIND.get(kind, kind), prec, pu, pv,
                                                                      ldw, pa, lda, po, ldo, _stream(stream)))


def rbt_transform_vec(n, d, align, kind, W, trans, B, stream=None):
    pw, ldw, _, _ = _mat(W, "W", torch.float64)
    pb, ldb, _, nrhs = _mat(B, "B", torch.float64)
    return _check("rbt_transform_vec", load().rbt_transform_vec(n, d, align, KIND.get(kind, kind), pw, ldw,
                                                                1 if trans else 0, pb, ldb, nrhs, _stream(stream)))


def rbt_apply_vec(n, d, W, trans, B, stream=None):
    pw, ldw, _, _ = _mat(W, "W", torch.float64)
    pb, ldb, _, nrhs = _mat(B, "B", torch.float64)
    return _check("rbt_apply_vec", load().rbt_apply_vec(n, d, pw, ldw, 1 if trans else 0, pb, ldb, nrhs,
                                                        _stream(stream)))


def genp_factor_workspace(n, prec, nb=0):
    return int(load().genp_factor_workspace(n, PREC.get(prec, prec), nb))


def genp_factor(n, prec, A, d_info, work=None, nb=0, stream=None):
    prec = PREC.get(prec, prec)
    pa, lda, _, _ = _mat(A, "A", PREC_DTYPE[prec])
    pw = ctypes.c_void_p(work.data_ptr()) if work is not None else ctypes.c_void_p(0)
    nbytes = work.numel() * work.element_size() if work is not None else 0
    return _check("genp_factor", load().genp_factor(n, prec, pa, lda, ctypes.c_void_p(d_info.data_ptr()), pw,
                                                    nbytes, nb, _stream(stream)))


def genp_update_workspace(M, N, K, prec):
    return int(load().genp_update_workspace(M, N, K, PREC.get(prec, prec)))


def genp_update(prec, A, B, C, d_status, work=None, stream=None):
    """C -= A B on the device (float column-major matrices)."""
    prec = PREC.get(prec, prec)
    dt = torch.float64 if prec in (4, 5, 6) else torch.float32   # df64 pairs live in 8-byte slots
    pa, lda, M, K = _mat(A, "A", dt)
    pb, ldb, K2, N = _mat(B, "B", dt)
    pc, ldc, _, _ = _mat(C, "C", dt)
    if K2 != K:
        raise ValueError("inner dimensions differ")
    pw = ctypes.c_void_p(work.data_ptr()) if work is not None else ctypes.c_void_p(0)
    nbytes = work.numel() * work.element_size() if work is not None else 0
    return _check("genp_update", load().genp_update(prec, M, N, K, pa, lda, pb, ldb, pc, ldc,
                                                    ctypes.c_void_p(d_status.data_ptr()), pw, nbytes,
                                                    _stream(stream)))


def genp_solve_workspace(n, nrhs, prec):
    return int(load().genp_solve_workspace(n, nrhs, PREC.get(prec, prec)))


def genp_solve(n, prec, LU, trans, B, work=None, stream=None):
    prec = PREC.get(prec, prec)
    pl, lda, _, _ = _mat(LU, "LU", PREC_DTYPE[prec])
    pb, ldb, _, nrhs = _mat(B, "B", torch.float64)
    pw = ctypes.c_void_p(work.data_ptr()) if work is not None else ctypes.c_void_p(0)
    nbytes = work.numel() * work.element_size() if work is not None else 0
    return _check("genp_solve", load().genp_solve(n, nrhs, prec, pl, lda, 1 if trans else 0, pb, ldb, pw, nbytes,
                                                  _stream(stream)))


def genp_solve_wp_workspace(n, nrhs):
    return int(load().genp_solve_wp_workspace(n, nrhs))


def genp_solve_wp(n, prec, LU, trans, B, work=None, stream=None):
    prec = PREC.get(prec, prec)
    pl, lda, _, _ = _mat(LU, "LU", PREC_DTYPE[prec])
    pb, ldb, _, nrhs = _mat(B, "B", torch.float64)
    pw = ctypes.c_void_p(work.data_ptr()) if work is not None else ctypes.c_void_p(0)
    nbytes = work.numel() * work.element_size() if work is not None else 0
    return _check("genp_solve_wp", load().genp_solve_wp(n, nrhs, prec, pl, lda, 1 if trans else 0, pb, ldb, pw,
                                                        nbytes, _stream(stream)))


def rbt_residual_workspace(n, nrhs):
    return int(load().rbt_residual_workspace(n, nrhs))


def rbt_residual(n, A, X, B, R, d_berr=None, d_anorm=None, work=None, stream=None):
    pa, lda, _, _ = _mat(A, "A", torch.float64)
    px, ldx, _, nrhs = _mat(X, "X", torch.float64)
    pb, ldb, _, _ = _mat(B, "B", torch.float64)
    pr, ldr, _, _ = _mat(R, "R", torch.float64)
    pberr = ctypes.c_void_p(d_berr.data_ptr()) if d_berr is not None else ctypes.c_void_p(0)
    pan = ctypes.c_void_p(d_anorm.data_ptr()) if d_anorm is not None else ctypes.c_void_p(0)
    pw = ctypes.c_void_p(work.data_ptr()) if work is not None else ctypes.c_void_p(0)
    nbytes = work.numel() * work.element_size() if work is not None else 0
    return _check("rbt_residual", load().rbt_residual(n, nrhs, pa, lda, px, ldx, pb, ldb, pr, ldr, pan, pberr,
                                                      pw, nbytes, _stream(stream)))


def rbt_residual_noalloc_max_bytes():
    return int(load().rbt_residual_noalloc_max_bytes())


def rbt_residual_noalloc(n, A, X, B, R, d_berr=None, d_anorm=None, stream=None):
    """rbt_residual without a workspace: scratch comes from the library's fixed device array."""
    pa, lda, _, _ = _mat(A, "A", torch.float64)
    px, ldx, _, nrhs = _mat(X, "X", torch.float64)
    pb, ldb, _, _ = _mat(B, "B", torch.float64)
    pr, ldr, _, _ = _mat(R, "R", torch.float64)
    pberr = ctypes.c_void_p(d_berr.data_ptr()) if d_berr is not None else ctypes.c_void_p(0)
    pan = ctypes.c_void_p(d_anorm.data_ptr()) if d_anorm is not None else ctypes.c_void_p(0)
    return _check("rbt_residual_noalloc", load().rbt_residual_noalloc(n, nrhs, pa, lda, px, ldx, pb, ldb, pr, ldr,
                                                                      pan, pberr, _stream(stream)))


def rbt_norm_inf(n, A, d_out, work, stream=None):
    pa, lda, _, _ = _mat(A, "A", torch.float64)
    return _check("rbt_norm_inf", load().rbt_norm_inf(n, pa, lda, ctypes.c_void_p(d_out.data_ptr()),
                                                      ctypes.c_void_p(work.data_ptr()),
                                                      work.numel() * work.element_size(), _stream(stream)))


BATCHED_INFO_DTYPE = None


def _info_dtype():
    import numpy as np
    return np.dtype([("status", np.int32), ("iters", np.int32), ("fell_back", np.int32), ("reserved", np.int32),
                     ("zero_pivot", np.int64), ("berr_unrefined", np.float64), ("berr", np.float64)])


class BatchedPlan:
    """Host-side handle of a planned batch: the workspace, the per-system info
    array and the ctypes arrays the plan was built from (kept alive)."""

    def __init__(self, opts, work, infos, keep):
        self.opts, self.work, self.infos, self._keep = opts, work, infos, keep

    def infos_host(self):
        import numpy as np
        raw = self.infos.cpu().numpy().tobytes()
        return np.frombuffer(raw, dtype=_info_dtype())


def _i64_array(vals):
    return (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])


def _ptr_array(tensors):
    return (ctypes.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])


def rbt_solve_batched_plan(opts, As, Bs, Xs, seeds=None, stream=None):
    """Plan a batch: As/Bs/Xs are lists of column-major CUDA float64 tensors
    (B, X: n x nrhs or length-n vectors).  Returns a BatchedPlan."""
    batch = len(As)
    ns, nrhs, lda, ldb, ldx = [], [], [], [], []
    for A, B, X in zip(As, Bs, Xs):
        _, la, n, _ = _mat(A, "A", torch.float64)
        _, lb, _, r = _mat(B, "B", torch.float64)
        _, lx, _, _ = _mat(X, "X", torch.float64)
        ns.append(n)
        nrhs.append(r)
        lda.append(la)
        ldb.append(lb)
        ldx.append(lx)
    keep = dict(n=_i64_array(ns), nrhs=_i64_array(nrhs), lda=_i64_array(lda), ldb=_i64_array(ldb),
                ldx=_i64_array(ldx), A=_ptr_array(As), B=_ptr_array(Bs), X=_ptr_array(Xs),
                seeds=(ctypes.c_uint64 * batch)(*[int(s) & (2**64 - 1) for s in seeds]) if seeds is not None else None,
                tensors=(As, Bs, Xs))
    lib = load()
    ws = int(lib.rbt_solve_batched_workspace(ctypes.byref(opts), batch, keep["n"], keep["nrhs"]))
    dev = As[0].device if batch else torch.device("cuda")
    work = torch.empty(max(ws, 1), dtype=torch.uint8, device=dev)
    infos = torch.zeros(max(batch, 1) * 40, dtype=torch.uint8, device=dev)
    _check("rbt_solve_batched_plan", lib.rbt_solve_batched_plan(
        ctypes.byref(opts), batch, keep["n"], keep["nrhs"], keep["A"], keep["lda"], keep["B"], keep["ldb"],
        keep["X"], keep["ldx"], keep["seeds"], ctypes.c_void_p(work.data_ptr()), ws, _stream(stream)))
    return BatchedPlan(opts, work, infos, keep)


def rbt_solve_batched_run(plan, stream=None):
    return _check("rbt_solve_batched_run", load().rbt_solve_batched_run(
        ctypes.byref(plan.opts), ctypes.c_void_p(plan.work.data_ptr()), ctypes.c_void_p(plan.infos.data_ptr()),
        _stream(stream)))


def rbt_solve_batched_autotune(plan, stream=None):
    v = ctypes.c_int32(-1)
    ms = ctypes.c_double(0)
    _check("rbt_solve_batched_autotune", load().rbt_solve_batched_autotune(
        ctypes.byref(plan.opts), ctypes.c_void_p(plan.work.data_ptr()), ctypes.c_void_p(plan.infos.data_ptr()),
        _stream(stream), ctypes.byref(v), ctypes.byref(ms)))
    return v.value, ms.value


def rbt_solve_batched_variant(plan):
    t = ctypes.c_int32(0)
    nb = ctypes.c_int32(0)
    v = load().rbt_solve_batched_variant(ctypes.c_void_p(plan.work.data_ptr()), ctypes.byref(t), ctypes.byref(nb))
    return v, t.value, nb.value


def rbt_kernel_launches():
    return int(load().rbt_kernel_launches())


STALL = {"none": 0, "chain": 1, "oz_copy": 2}


def rbt_debug_wait_limit(ns):
    """Set the limit of every bounded device wait (ns <= 0: the default, one second); returns the previous."""
    return int(load().rbt_debug_wait_limit(int(ns)))


def rbt_debug_stall(which):
    """Make one kind of bounded wait run out on purpose (testing); returns the previous setting."""
    return int(load().rbt_debug_stall(STALL.get(which, which)))


def rbt_debug_oz_products(da, db, stream=None):
    """Raw accumulators of the sliced update for int8 digit tensors da (8 x M x K)
    and db (8 x N x K) on the device; returns a float32 tensor of 8 x M x N."""
    if da.dtype != torch.int8 or db.dtype != torch.int8 or not da.is_cuda or not db.is_cuda:
        raise TypeError("da and db must be int8 CUDA tensors")
    da, db = da.contiguous(), db.contiguous()
    S, M, K = da.shape
    _, N, K2 = db.shape
    if K2 != K or S != 8 or db.shape[0] != 8:
        raise ValueError("digit shapes differ")
    acc = torch.empty((8, M, N), dtype=torch.float32, device=da.device)
    ws = int(load().rbt_debug_oz_products_workspace(M, N, K))
    work = torch.empty(max(ws, 1), dtype=torch.uint8, device=da.device)
    _check("rbt_debug_oz_products", load().rbt_debug_oz_products(
        M, N, K, ctypes.c_void_p(da.data_ptr()), ctypes.c_void_p(db.data_ptr()), ctypes.c_void_p(acc.data_ptr()),
        ctypes.c_void_p(work.data_ptr()), ws, _stream(stream)))
    return acc


PROF_CLASSES = {"update": 0, "transform": 1, "panel": 2, "solve": 3, "residual": 4, "slice": 5}


def rbt_prof_enable(on=True):
    load().rbt_prof_enable(1 if on else 0)


def rbt_prof_reset():
    load().rbt_prof_reset()


def rbt_prof_read(cls):
    ms = ctypes.c_double(0)
    nl = ctypes.c_int64(0)
    _check("rbt_prof_read", load().rbt_prof_read(PROF_CLASSES.get(cls, cls), ctypes.byref(ms), ctypes.byref(nl)))
    return ms.value, nl.value


REFINE = {"stationary": 0, "gmres": 1}
KIND = {"scaled": 0, "rotation": 1}


def rbt_reference_size(n, d, align=1, grid=(1, 1)):
    """Reference size m of the butterflies (host query): non-tiled, tiled (align = n_b)
    or communication-free on a p x q process grid (grid = (p, q))."""
    return int(load().rbt_reference_size(n, d, align, int(grid[0]), int(grid[1])))


def make_opts(depth=2, seed=1, prec="f64", refine_max=30, tol=1e-13, fallback=True, nb=0, align=1,
              refine="stationary", restart=0, kind="scaled", grid=(1, 1)):
    o = rbt_opts()
    o.depth = depth
    o.seed = seed & (2**64 - 1)
    o.prec = PREC.get(prec, prec)
    o.refine_max = refine_max
    o.tol = tol
    o.fallback = 1 if fallback else 0
    o.nb = nb
    o.align = align
    o.refine_mode = REFINE.get(refine, refine)
    o.restart = restart
    o.kind = KIND.get(kind, kind)
    o.grid_p, o.grid_q = int(grid[0]), int(grid[1])
    return o


def rbt_solve_workspace(opts, n, nrhs):
    return int(load().rbt_solve_workspace(ctypes.byref(opts), n, nrhs))


def rbt_solve_host_workspace(opts, n, nrhs):
    return int(load().rbt_solve_host_workspace(ctypes.byref(opts), n, nrhs))


def rbt_solve_host(opts, n, A, B, X, work, stream=None, ok=(RBT_OK, RBT_NOT_CONVERGED, RBT_ZERO_PIVOT, RBT_NONFINITE)):
    """rbt_solve with A, B, X as column-major float64 CPU tensors (pinned for
    the SM-driven copies) and a device work buffer; returns (status, info dict)."""
    pa, lda, _, _ = _mat(A, "A", torch.float64, host=True)
    pb, ldb, _, nrhs = _mat(B, "B", torch.float64, host=True)
    px, ldx, _, _ = _mat(X, "X", torch.float64, host=True)
    info = rbt_info()
    code = load().rbt_solve_host(ctypes.byref(opts), n, nrhs, pa, lda, pb, ldb, px, ldx,
                                 ctypes.c_void_p(work.data_ptr()), work.numel() * work.element_size(),
                                 ctypes.byref(info), _stream(stream))
    _check("rbt_solve_host", code, ok)
    return code, info.as_dict()


def rbt_solve(opts, n, A, B, X, work, stream=None, ok=(RBT_OK, RBT_NOT_CONVERGED, RBT_ZERO_PIVOT, RBT_NONFINITE)):
    """Returns (status, info dict)."""
    pa, lda, _, _ = _mat(A, "A", torch.float64)
    pb, ldb, _, nrhs = _mat(B, "B", torch.float64)
    px, ldx, _, _ = _mat(X, "X", torch.float64)
    info = rbt_info()
    code = load().rbt_solve(ctypes.byref(opts), n, nrhs, pa, lda, pb, ldb, px, ldx,
                            ctypes.c_void_p(work.data_ptr()), work.numel() * work.element_size(),
                            ctypes.byref(info), _stream(stream))
    _check("rbt_solve", code, ok)
    return code, info.as_dict()
