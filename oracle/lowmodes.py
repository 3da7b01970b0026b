"""Eigenvalues of Q = gamma_5 D closest to zero (Sec. 3: lambda_bar = min_n |lambda_n|).

``modes_dense``: all eigenvalues of the dense Hermitian Q(m0) (LAPACK zheevd via
numpy), returned sorted by |lambda|, k of them, with zero residuals.
``modes_sparse``: the k eigenvalues of the sparse Q(m0) nearest zero: shift-invert
Lanczos (scipy ARPACK, sigma = 0), the found vectors completed with their C* partners
C T gamma_5 v^* (Q commutes with that antiunitary map, Sec. 3, so every eigenvalue is at
least doubly degenerate and a single-vector Krylov method finds the second copy only
through rounding), then Lanczos on Q^-1 restricted to the complement of what was found,
repeated until the value nearest zero left there lies beyond the k-th found; finally a
Rayleigh-Ritz with Q on all vectors, with true residual norms ||Q v - lambda v||.
modes_dense is a library routine used as one step.  Pins (tests/test_oracle_sign.py,
tests/test_oracle_dirac.py): modes_dense reproduces the free-field closed-form
spectrum with C* momenta; modes_sparse reproduces the same closed form on a free
2^3 x 6 field and agrees with modes_dense on a rough 2^3 x 4 field.
"""
import contextlib

import numpy as np
import scipy.sparse.linalg as spla

try:   # many tiny BLAS calls in the Lanczos loops: threads only add overhead there
    from threadpoolctl import threadpool_limits as _blas_threads
except ImportError:
    def _blas_threads(limits):
        return contextlib.nullcontext()


def modes_dense(op, m0, k=None):
    w = np.linalg.eigvalsh(op.dense_Q(m0))
    w = w[np.argsort(np.abs(w), kind="stable")]
    if k is not None:
        w = w[:k]
    return w, np.zeros_like(w)


def modes_sparse(op, m0, k, tol=1e-12, seed=0):
    with _blas_threads(1):
        return _modes_sparse(op, m0, k, tol, seed)


def _modes_sparse(op, m0, k, tol, seed):
    Q = op.sparse_Q(m0).tocsc()
    n = Q.shape[0]
    rng = np.random.default_rng(seed)
    _, X = spla.eigsh(Q, k=k, sigma=0.0, which="LM", tol=tol, v0=rng.normal(size=n) + 0j)
    # every eigenspace of Q is closed under the antiunitary P v = C T gamma_5 v^* (Sec. 3)
    CT = op.CT_matrix()
    g5 = np.where(np.arange(n) % 12 >= 6, -1.0, 1.0)
    V = _orth(np.hstack([X, CT @ (g5[:, None] * X.conj())]))
    lu = None
    while V.shape[1] + 8 < n:
        # a degenerate value can have further copies outside span(V); a copy nearer zero
        # than the k-th value found is the dominant eigenvector of the deflated Q^-1
        if lu is None:
            lu = spla.splu(Q)
        Vh = np.ascontiguousarray(V.conj().T)
        B = spla.LinearOperator((n, n), matvec=lambda x: _deflate(V, Vh, lu.solve(_deflate(V, Vh, x))),
                                dtype=complex)
        mu, Y = spla.eigsh(B, k=2, ncv=20, which="LM", tol=1e-6, v0=rng.normal(size=n) + 0j)
        kth = np.sort(np.abs(np.linalg.eigvalsh(V.conj().T @ (Q @ V))))[k - 1]
        if 1.0 / np.max(np.abs(mu)) > kth * (1 + 1e-4):
            break
        # found one: refine it with a tight solve of the deflated operator, with partners
        _, Y = spla.eigsh(B, k=2, which="LM", tol=tol, v0=Y[:, np.argmax(np.abs(mu))])
        V = _orth(np.hstack([V, Y, CT @ (g5[:, None] * Y.conj())]))
    H = V.conj().T @ (Q @ V)
    w, y = np.linalg.eigh(0.5 * (H + H.conj().T))
    order = np.argsort(np.abs(w), kind="stable")[:k]
    w, X = w[order], V @ y[:, order]
    r = np.linalg.norm(Q @ X - X * w[None, :], axis=0)
    return w, r


def _deflate(V, Vh, x):
    """x minus its projection on the orthonormal columns of V (Vh = V^H)."""
    return x - V @ (Vh @ x)


def _orth(A):
    """Orthonormal basis of span(A), dropping directions below 1e-10 of the largest."""
    U, sv, _ = np.linalg.svd(A, full_matrices=False)
    return U[:, sv > 1e-10 * sv[0]]
