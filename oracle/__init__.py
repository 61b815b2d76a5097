"""Plain FP64 CPU oracle for the generalized RBT + GENP solver (arXiv 2312.09376).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path in ``paper_2312_09376_gb300``; the two meet only through the
seeded inputs of ``paper_2312_09376_gb300.inputs``.

The arithmetic lives in ``rbt_oracle.c`` (plain C, double precision, literal
loops).  This module compiles it with gcc on first use and wraps it with ctypes
over numpy arrays (column-major, i.e. Fortran order).

Every function below follows the passage cited in the C source:
  * sizes and layers: Sec. 3, Eq. (O-matrix-definition), Eq. (rbt-depth-d),
    Eq. (butterfly-alignment), Algorithm 1's reference size;
  * random coefficients: Sec. 6 (exp(r/20), r uniform on [-1, 1]);
  * GENP and its solves: Sec. 1 and Sec. 4 (elimination without pivoting);
  * backward error: Eq. (inf-norm-backerr);
  * full solve: Eq. (precond) with the refinement of Sec. 5.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rbt_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build/liboracle.so`` (plain -O2, no fast-math)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    hdr = os.path.join(_HERE, "rbt_oracle.h")
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC), os.path.getmtime(hdr)))
    if force or stale:
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_BLOCKED_SRC = os.path.join(_HERE, "rbt_cpu_blocked.c")
_BLOCKED_PATH = os.path.join(_BUILD_DIR, "libcpu_blocked.so")
_blocked = None


def build_blocked(force: bool = False) -> str:
    """Compile the timed CPU baseline (tier b: cache-blocked, OpenMP) into
    ``oracle/_build/libcpu_blocked.so``: its own file at -O3 with OpenMP, the
    oracle's generator linked in from rbt_oracle.c built as for liboracle."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    hdr = os.path.join(_HERE, "rbt_oracle.h")
    srcs = [_BLOCKED_SRC, _SRC, hdr]
    stale = (not os.path.exists(_BLOCKED_PATH)
             or os.path.getmtime(_BLOCKED_PATH) < max(os.path.getmtime(p) for p in srcs))
    if force or stale:
        pid = os.getpid()
        o1 = os.path.join(_BUILD_DIR, "cpu_blocked.%d.o" % pid)
        o2 = os.path.join(_BUILD_DIR, "oracle_gen.%d.o" % pid)
        tmp = _BLOCKED_PATH + ".%d.tmp" % pid
        subprocess.run(["gcc", "-O3", "-std=c11", "-fPIC", "-fopenmp", "-fno-fast-math", "-c", _BLOCKED_SRC,
                        "-o", o1], check=True)
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-fno-fast-math", "-ffp-contract=off", "-c", _SRC,
                        "-o", o2], check=True)
        subprocess.run(["gcc", "-shared", "-fopenmp", "-o", tmp, o1, o2, "-lm"], check=True)
        os.replace(tmp, _BLOCKED_PATH)
        for o in (o1, o2):
            os.unlink(o)
    return _BLOCKED_PATH


def _load_blocked():
    global _blocked
    with _lock:
        if _blocked is not None:
            return _blocked
        lib = ctypes.CDLL(build_blocked())
        i64, i32, u64, dbl, P = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
        for name, res, args in (("cpu_threads", i32, []),
                                ("cpu_set_threads", i32, [i32]),
                                ("cpu_genp", i64, [i64, P, i64, i32]),
                                ("cpu_rbt_solve", i64, [i64, i64, i32, u64, P, i64, P, i64, P, i64, i32, dbl, i32,
                                                        P])):
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _blocked = lib
        return lib


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
        P = ctypes.c_void_p
        sig = {
            "orc_ceil_log2": (i32, [i64]),
            "orc_depth_eff": (i32, [i64, i32]),
            "orc_ref_size": (i64, [i64, i32]),
            "orc_ref_size_tiled": (i64, [i64, i32, i64]),
            "orc_lcm": (i64, [i64, i64]),
            "orc_ref_size_comm_free": (i64, [i64, i32, i64, i64, i64]),
            "orc_splitmix64": (u64, [u64]),
            "orc_coef": (dbl, [u64, i32, i32, i64]),
            "orc_generate": (None, [i64, i32, u64, P, P, i64]),
            "orc_layer_rows": (None, [i64, i32, i32, P, i64, i64]),
            "orc_layer_cols": (None, [i64, i32, i32, P, i64, i64]),
            "orc_layer_rows_tiled": (None, [i64, i32, i64, i32, P, i64, i64]),
            "orc_layer_cols_tiled": (None, [i64, i32, i64, i32, P, i64, i64]),
            "orc_transform_2sided_tiled": (None, [i64, i32, i64, P, i64, P, i64, P, i64]),
            "orc_transform_vec_tiled": (None, [i64, i32, i64, P, i64, i32, P, i64, i64]),
            "orc_rbt_solve_tiled": (i64, [i64, i64, i32, i64, u64, P, i64, P, i64, P, i64, i32, dbl, P]),
            "orc_gmres_ir": (None, [i64, i32, i64, P, P, P, P, i64, P, P, i32, i32, dbl, P, P]),
            "orc_rot_u": (dbl, [u64, i32, i32, i64]),
            "orc_generate_rot": (None, [i64, i32, i64, u64, P, P, i64]),
            "orc_layer_rows_rot": (None, [i64, i32, i64, i32, P, i64, P, i64, i64]),
            "orc_layer_cols_rot": (None, [i64, i32, i64, i32, P, i64, P, i64, i64]),
            "orc_transform_2sided_rot": (None, [i64, i32, i64, P, i64, P, i64, P, i64]),
            "orc_transform_vec_rot": (None, [i64, i32, i64, P, i64, i32, P, i64, i64]),
            "orc_rbt_solve_kind": (i64, [i64, i64, i32, i64, i32, u64, P, i64, P, i64, P, i64, i32, dbl, P]),
            "orc_transform_2sided": (None, [i64, i32, P, i64, P, i64, P, i64]),
            "orc_transform_vec": (None, [i64, i32, P, i64, i32, P, i64, i64]),
            "orc_genp": (i64, [i64, P, i64]),
            "orc_genp_solve": (None, [i64, i64, P, i64, i32, P, i64]),
            "orc_residual": (None, [i64, i64, P, i64, P, i64, P, i64, P, i64]),
            "orc_norm_inf_mat": (dbl, [i64, P, i64]),
            "orc_backward_error": (dbl, [i64, i64, P, i64, P, i64, P, i64]),
            "orc_rbt_solve": (i64, [i64, i64, i32, u64, P, i64, P, i64, P, i64, i32, dbl, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _f64(a, copy=True):
    """A Fortran-ordered float64 array (copied unless told otherwise)."""
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a.reshape(-1, 1)
    return np.array(a, dtype=np.float64, order="F", copy=True) if copy else np.asfortranarray(a)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _ld(a):
    return max(1, a.shape[0])


# ---------------------------------------------------------------- sizes

def ceil_log2(n: int) -> int:
    return int(_load().orc_ceil_log2(n))


def depth_eff(n: int, d: int) -> int:
    return int(_load().orc_depth_eff(n, d))


def ref_size(n: int, d: int, align: int = 1) -> int:
    """Reference size m of Sec. 3: non-tiled for align = 1, tiled for align = n_b."""
    if align == 1:
        return int(_load().orc_ref_size(n, d))
    return int(_load().orc_ref_size_tiled(n, d, align))


def lcm(p: int, q: int) -> int:
    return int(_load().orc_lcm(p, q))


def ref_size_comm_free(n: int, d: int, nb: int, p: int, q: int) -> int:
    """Reference size of Eq. (comm-free-rbt-size): twice the top half of the first
    layer, lcm(p, q) 2^(d-1) ceil(n_t 2^-d / lcm(p, q)) tiles of n_b rows."""
    return int(_load().orc_ref_size_comm_free(n, d, nb, p, q))


# ------------------------------------------------------------ generator

def splitmix64(key: int) -> int:
    return int(_load().orc_splitmix64(ctypes.c_uint64(key & (2**64 - 1))))


def coef(seed: int, side: int, layer: int, i: int) -> float:
    return float(_load().orc_coef(seed, side, layer, i))


def generate(n: int, d: int, seed: int):
    """Packed U, V (n x d each, column k-1 = diagonal of R_k)."""
    U = np.zeros((n, d), order="F")
    V = np.zeros((n, d), order="F")
    if n > 0 and d > 0:
        _load().orc_generate(n, d, seed, _ptr(U), _ptr(V), n)
    return U, V


# ------------------------------------------------------------ transforms

def layer_rows(n, d, k, X, align: int = 1):
    X = _f64(X)
    if align == 1:
        _load().orc_layer_rows(n, d, k, _ptr(X), _ld(X), X.shape[1])
    else:
        _load().orc_layer_rows_tiled(n, d, align, k, _ptr(X), _ld(X), X.shape[1])
    return X


def layer_cols(n, d, k, X, align: int = 1):
    X = _f64(X)
    if align == 1:
        _load().orc_layer_cols(n, d, k, _ptr(X), _ld(X), X.shape[0])
    else:
        _load().orc_layer_cols_tiled(n, d, align, k, _ptr(X), _ld(X), X.shape[0])
    return X


def transform_2sided(A, U, V, d: int, align: int = 1):
    """Return U^T A V (A is not modified); align = n_b selects the tiled reference size."""
    A = _f64(A)
    n = A.shape[0]
    U = _f64(U)
    V = _f64(V)
    if n > 0:
        if align == 1:
            _load().orc_transform_2sided(n, d, _ptr(U), _ld(U), _ptr(V), _ld(V), _ptr(A), _ld(A))
        else:
            _load().orc_transform_2sided_tiled(n, d, align, _ptr(U), _ld(U), _ptr(V), _ld(V), _ptr(A), _ld(A))
    return A


def transform_vec(B, W, d: int, trans: bool, align: int = 1):
    """Return W^T B (trans) or W B (not trans)."""
    squeeze = np.asarray(B).ndim == 1
    B = _f64(B)
    W = _f64(W)
    n, nrhs = B.shape
    if n > 0 and nrhs > 0:
        if align == 1:
            _load().orc_transform_vec(n, d, _ptr(W), _ld(W), 1 if trans else 0, _ptr(B), _ld(B), nrhs)
        else:
            _load().orc_transform_vec_tiled(n, d, align, _ptr(W), _ld(W), 1 if trans else 0, _ptr(B), _ld(B),
                                            nrhs)
    return B[:, 0] if squeeze else B


# ------------------------------------------------- rotation butterflies

def rot_u(seed: int, side: int, layer: int, i: int) -> float:
    """The uniform u on [0, 1) whose angle 2 pi u rotates the pair with top row i."""
    return float(_load().orc_rot_u(seed, side, layer, i))


def generate_rot(n: int, d: int, seed: int, align: int = 1):
    """Packed rotation coefficients (n x d each): cos at each pair's top row,
    sin at its bottom row, 1 at nu rows and in layers past the effective depth."""
    U = np.zeros((n, d), order="F")
    V = np.zeros((n, d), order="F")
    if n > 0 and d > 0:
        _load().orc_generate_rot(n, d, align, seed, _ptr(U), _ptr(V), n)
    return U, V


def layer_rows_rot(n, d, k, W, X, align: int = 1):
    X = _f64(X)
    W = _f64(W)
    _load().orc_layer_rows_rot(n, d, align, k, _ptr(W), _ld(W), _ptr(X), _ld(X), X.shape[1])
    return X


def layer_cols_rot(n, d, k, W, X, align: int = 1):
    X = _f64(X)
    W = _f64(W)
    _load().orc_layer_cols_rot(n, d, align, k, _ptr(W), _ld(W), _ptr(X), _ld(X), X.shape[0])
    return X


def transform_2sided_rot(A, U, V, d: int, align: int = 1):
    """Return U^T A V for rotation butterflies (A is not modified)."""
    A = _f64(A)
    n = A.shape[0]
    U = _f64(U)
    V = _f64(V)
    if n > 0:
        _load().orc_transform_2sided_rot(n, d, align, _ptr(U), _ld(U), _ptr(V), _ld(V), _ptr(A), _ld(A))
    return A


def transform_vec_rot(B, W, d: int, trans: bool, align: int = 1):
    """Return W^T B (trans) or W B for rotation butterflies."""
    squeeze = np.asarray(B).ndim == 1
    B = _f64(B)
    W = _f64(W)
    n, nrhs = B.shape
    if n > 0 and nrhs > 0:
        _load().orc_transform_vec_rot(n, d, align, _ptr(W), _ld(W), 1 if trans else 0, _ptr(B), _ld(B), nrhs)
    return B[:, 0] if squeeze else B


# ------------------------------------------------------------------ GENP

def genp(A):
    """Return (LU, status): status -1 on success else the first bad pivot index."""
    A = _f64(A)
    n = A.shape[0]
    st = int(_load().orc_genp(n, _ptr(A), _ld(A))) if n > 0 else -1
    return A, st


def genp_solve(LU, B, trans: bool = False):
    squeeze = np.asarray(B).ndim == 1
    LU = _f64(LU, copy=False)
    B = _f64(B)
    n, nrhs = B.shape
    if n > 0 and nrhs > 0:
        _load().orc_genp_solve(n, nrhs, _ptr(LU), _ld(LU), 1 if trans else 0, _ptr(B), _ld(B))
    return B[:, 0] if squeeze else B


def residual(A, X, B):
    squeeze = np.asarray(B).ndim == 1
    A = _f64(A, copy=False)
    X = _f64(X, copy=False)
    B = _f64(B, copy=False)
    n, nrhs = B.shape
    R = np.zeros((n, nrhs), order="F")
    _load().orc_residual(n, nrhs, _ptr(A), _ld(A), _ptr(X), _ld(X), _ptr(B), _ld(B), _ptr(R), _ld(R))
    return R[:, 0] if squeeze else R


def norm_inf_mat(A) -> float:
    A = _f64(A, copy=False)
    return float(_load().orc_norm_inf_mat(A.shape[0], _ptr(A), _ld(A)))


def backward_error(A, X, B) -> float:
    A = _f64(A, copy=False)
    X = _f64(X, copy=False)
    B = _f64(B, copy=False)
    n, nrhs = B.shape
    return float(_load().orc_backward_error(n, nrhs, _ptr(A), _ld(A), _ptr(X), _ld(X), _ptr(B), _ld(B)))


def rbt_solve(A, B, d: int, seed: int, refine_max: int = 30, tol: float = 1e-13, align: int = 1,
              kind: str = "scaled"):
    """Full RBT solve with the scaled butterflies of Eq. (rbt-depth-d)
    (kind "scaled") or the rotation form (kind "rotation").
    Returns (X, status, berr_unrefined, berr, iters)."""
    squeeze = np.asarray(B).ndim == 1
    A = _f64(A, copy=False)
    B = _f64(B, copy=False)
    n, nrhs = B.shape
    X = np.zeros((n, nrhs), order="F")
    out = np.zeros(3)
    if kind not in ("scaled", "rotation"):
        raise ValueError(kind)
    if kind == "rotation":
        st = int(_load().orc_rbt_solve_kind(n, nrhs, d, align, 1, seed, _ptr(A), _ld(A), _ptr(B), _ld(B),
                                            _ptr(X), _ld(X), refine_max, tol, _ptr(out)))
    elif align == 1:
        st = int(_load().orc_rbt_solve(n, nrhs, d, seed, _ptr(A), _ld(A), _ptr(B), _ld(B),
                                       _ptr(X), _ld(X), refine_max, tol, _ptr(out)))
    else:
        st = int(_load().orc_rbt_solve_tiled(n, nrhs, d, align, seed, _ptr(A), _ld(A), _ptr(B), _ld(B),
                                             _ptr(X), _ld(X), refine_max, tol, _ptr(out)))
    return (X[:, 0] if squeeze else X), st, float(out[0]), float(out[1]), int(out[2])


# ------------------------------------------- timed CPU baseline (tier b)

def cpu_threads() -> int:
    """Threads the blocked baseline runs on (OpenMP; OMP_NUM_THREADS or all cores)."""
    return int(_load_blocked().cpu_threads())


def cpu_set_threads(n: int) -> int:
    """Use n threads in the blocked baseline (n <= 0: unchanged); returns the count in effect."""
    return int(_load_blocked().cpu_set_threads(n))


def cpu_genp(A, nb: int = 128):
    """Blocked GENP of the tier-b baseline; returns (LU, status) as genp()."""
    A = _f64(A)
    n = A.shape[0]
    st = int(_load_blocked().cpu_genp(n, _ptr(A), _ld(A), nb)) if n > 0 else -1
    return A, st


def cpu_rbt_solve(A, B, d: int, seed: int, refine_max: int = 30, tol: float = 1e-13, nb: int = 128):
    """The tier-b solve (same method as rbt_solve, non-tiled size).  Returns
    (X, status, berr_unrefined, berr, iters, seconds_factor, seconds_total)."""
    squeeze = np.asarray(B).ndim == 1
    A = _f64(A, copy=False)
    B = _f64(B, copy=False)
    n, nrhs = B.shape
    X = np.zeros((n, nrhs), order="F")
    out = np.zeros(5)
    st = int(_load_blocked().cpu_rbt_solve(n, nrhs, d, seed, _ptr(A), _ld(A), _ptr(B), _ld(B), _ptr(X), _ld(X),
                                           refine_max, tol, nb, _ptr(out)))
    return (X[:, 0] if squeeze else X), st, float(out[0]), float(out[1]), int(out[2]), float(out[3]), float(out[4])


# ------------------------------------------------------------- GMRES-IR

def gmres_ir(A, b, U, V, d: int, LU, x0, restart: int = 30, max_iter: int = 200, tol: float = 1e-13,
             align: int = 1):
    """Refinement of x0 by restarted GMRES right preconditioned with
    V (LU)^{-1} U^T.  Returns (x, berr_in, berr, products, cycles, history)."""
    A = _f64(A, copy=False)
    n = A.shape[0]
    b = _f64(np.asarray(b).reshape(-1))
    x = _f64(np.asarray(x0).reshape(-1))
    U = _f64(U)
    V = _f64(V)
    LU = _f64(LU)
    out = np.zeros(4)
    hist = np.zeros(max(max_iter, 1))
    _load().orc_gmres_ir(n, d, align, _ptr(U), _ptr(V), _ptr(LU), _ptr(A), _ld(A), _ptr(b), _ptr(x), restart,
                         max_iter, tol, _ptr(out), _ptr(hist))
    used = int(out[2])
    return x[:, 0], float(out[0]), float(out[1]), used, int(out[3]), hist[:used]
