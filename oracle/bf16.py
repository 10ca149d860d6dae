"""bfloat16 rounding of FP64 values, written from the format's definition.

bfloat16 keeps the sign, the 8-bit exponent of IEEE binary32 and 8 significant
bits (7 stored).  A finite FP64 value in the normal binary32 range is rounded
to the nearest number with 8 significant bits, ties to even.  Used by the
oracle to build the mixed-precision preconditioner's coefficient set (the
stored stencil entries are rounded to bfloat16, arithmetic stays FP64 here).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def round_bf16(x):
    """Round each real FP64 value to the nearest bfloat16 value (ties to even).
    Values are assumed to be zero or within the binary32 normal range."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                 # x = m * 2^e, 0.5 <= |m| < 1
    q = np.rint(m * 256.0)             # 8 significant bits, round half to even
    return np.ldexp(q, e - 8)


def round_complex_bf16(z):
    z = np.asarray(z)
    return round_bf16(z.real) + 1j * round_bf16(z.imag)


def round_matrix_bf16(A):
    """Copy of sparse matrix A with every stored entry rounded to bfloat16
    (real and imaginary parts separately)."""
    A = sp.csr_matrix(A, copy=True)
    A.data = round_complex_bf16(A.data) if np.iscomplexobj(A.data) else round_bf16(A.data)
    return A
