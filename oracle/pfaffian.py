"""Pfaffian of a complex antisymmetric matrix (Sec. 3, eq. power1/4: pf[M]^2 = det M).

``pfaffian_brute``: expansion along the first row over perfect matchings,
  pf(A) = sum_{j>0} (-1)^(j+1) A[0, j] pf(A without rows/cols 0 and j);
  exponential cost, only for n <= 10; it is the textbook definition.
``pfaffian``: Parlett-Reid elimination with partial pivoting (Wimmer, ACM TOMS 38,
  30 (2012), section on Gaussian elimination), written from that description.
  Each step takes the 2x2 pivot block [[0, a], [-a, 0]] with a = A[k, k+1] and
  replaces the trailing block by its Schur complement
      A'' = A' + (c b^T - b c^T) / a,   b = A[k, k+2:], c = A[k+1, k+2:],
  so that pf(A) = a * pf(A'').  Row/column swaps flip the sign.  The result is
  returned as (log|pf|, phase) so that n = 6144 neither over- nor underflows.
``pfaffian_c``: the same elimination in plain C (oracle/pfaffian_c.c) for large n.

Pinned by tests/test_oracle_pfaffian.py: brute force, pf^2 = det,
pf(B^T A B) = det(B) pf(A), block-diagonal closed form.
"""
import ctypes
import os

import numpy as np


def pfaffian_brute(A):
    A = np.asarray(A)
    n = A.shape[0]
    if n == 0:
        return 1.0 + 0j
    if n % 2:
        return 0.0 + 0j
    total = 0.0 + 0j
    for j in range(1, n):
        keep = [i for i in range(n) if i not in (0, j)]
        total += (-1) ** (j + 1) * A[0, j] * pfaffian_brute(A[np.ix_(keep, keep)])
    return total


def pfaffian(A):
    """(log|pf A|, phase of pf A) by Parlett-Reid elimination with pivoting."""
    A = np.array(A, dtype=np.complex128, copy=True)
    n = A.shape[0]
    if n % 2:
        return -np.inf, 0.0 + 0j
    logabs, phase = 0.0, 1.0 + 0j
    for k in range(0, n - 1, 2):
        p = k + 1 + int(np.argmax(np.abs(A[k, k + 1:])))
        if p != k + 1:
            A[[k + 1, p], :] = A[[p, k + 1], :]
            A[:, [k + 1, p]] = A[:, [p, k + 1]]
            phase = -phase
        a = A[k, k + 1]
        if a == 0:
            return -np.inf, 0.0 + 0j
        logabs += np.log(abs(a))
        phase *= a / abs(a)
        if k + 2 < n:
            b = A[k, k + 2:].copy()
            c = A[k + 1, k + 2:].copy()
            A[k + 2:, k + 2:] += (np.outer(c, b) - np.outer(b, c)) / a
    return logabs, phase


def pfaffian_value(A):
    la, ph = pfaffian(A)
    return 0.0 if la == -np.inf else np.exp(la) * ph


_here = os.path.dirname(os.path.abspath(__file__))
_lib = None


def build_c(force=False):
    """Compile oracle/pfaffian_c.c into oracle/_build/libpforacle.so (gcc, OpenMP)."""
    import subprocess
    out_dir = os.path.join(_here, "_build")
    so = os.path.join(out_dir, "libpforacle.so")
    src = os.path.join(_here, "pfaffian_c.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        os.makedirs(out_dir, exist_ok=True)
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               src, "-o", so, "-lm"])
    return so


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_c())
        _lib.pf_parlett_reid.restype = ctypes.c_int
        _lib.pf_parlett_reid.argtypes = [ctypes.c_long, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]
    return _lib


def pfaffian_c(A):
    """Same as ``pfaffian`` but in C; A is copied (row-major complex128)."""
    lib = _load()
    M = np.array(A, dtype=np.complex128, order="C", copy=True)
    n = M.shape[0]
    la, pr, pi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib.pf_parlett_reid(n, M.ctypes.data, ctypes.byref(la), ctypes.byref(pr), ctypes.byref(pi))
    return la.value, complex(pr.value, pi.value)
