"""Host-side packing of double-float operands for the GPU tests: a double-float
element is an unevaluated pair (hi, lo) of floats in one 8-byte slot."""
import numpy as np
import torch

from paper_2312_09376_gb300 import _lib


def to_df64(a):
    """Column-major device tensor of 8-byte slots holding (hi, lo) float pairs
    of a, and the value those pairs represent (hi + lo, exactly, as float64)."""
    a = np.asarray(a, dtype=np.float64)
    hi = a.astype(np.float32)
    lo = (a - hi.astype(np.float64)).astype(np.float32)
    rows, cols = a.shape
    buf = np.empty((cols, rows, 2), dtype=np.float32)    # column-major order of pairs
    buf[..., 0] = hi.T
    buf[..., 1] = lo.T
    slots = torch.from_numpy(buf.reshape(-1)).view(torch.float64).reshape(cols, rows)
    return slots.cuda().T, hi.astype(np.float64) + lo.astype(np.float64)


def from_df64(t):
    return _lib.to_host(_lib.df64_to_double(t))
