"""Eigenvalues of Q = gamma_5 D closest to zero (Sec. 3: lambda_bar = min_n |lambda_n|).

``modes_dense``: all eigenvalues of the dense Hermitian Q(m0) (LAPACK zheevd via
numpy), returned sorted by |lambda|, k of them, with zero residuals.
``modes_sparse``: the k eigenvalues of the sparse Q(m0) nearest zero by
shift-invert Lanczos (scipy ARPACK, sigma = 0), with true residual norms
||Q v - lambda v|| of the returned unit vectors.
Both are library routines used as one step.  Pins (tests/test_oracle_sign.py,
tests/test_oracle_dirac.py): modes_dense reproduces the free-field closed-form
spectrum with C* momenta; modes_sparse reproduces the same closed form on a free
2^3 x 6 field and agrees with modes_dense on a rough 2^3 x 4 field.
"""
import numpy as np
import scipy.sparse.linalg as spla


def modes_dense(op, m0, k=None):
    w = np.linalg.eigvalsh(op.dense_Q(m0))
    w = w[np.argsort(np.abs(w), kind="stable")]
    if k is not None:
        w = w[:k]
    return w, np.zeros_like(w)


def modes_sparse(op, m0, k, tol=1e-12):
    Q = op.sparse_Q(m0).tocsc()
    w, v = spla.eigsh(Q, k=k, sigma=0.0, which="LM", tol=tol)
    r = np.linalg.norm(Q @ v - v * w[None, :], axis=0)
    order = np.argsort(np.abs(w), kind="stable")
    return w[order], r[order]
