"""Pins of oracle/pfaffian.py against the definition and algebraic identities."""
import numpy as np
import pytest

from oracle.pfaffian import pfaffian, pfaffian_brute, pfaffian_c, pfaffian_value


def rand_antisym(rng, n):
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return X - X.T


@pytest.mark.parametrize("n", [2, 4, 6, 8, 10])
def test_brute_force(n):
    rng = np.random.default_rng(n)
    A = rand_antisym(rng, n)
    ref = pfaffian_brute(A)
    assert np.isclose(pfaffian_value(A), ref, rtol=1e-11)
    la, ph = pfaffian_c(A)
    assert np.isclose(np.exp(la) * ph, ref, rtol=1e-11)


def test_4x4_closed_form():
    rng = np.random.default_rng(7)
    A = rand_antisym(rng, 4)
    ref = A[0, 1] * A[2, 3] - A[0, 2] * A[1, 3] + A[0, 3] * A[1, 2]
    assert np.isclose(pfaffian_value(A), ref, rtol=1e-13)


@pytest.mark.parametrize("n", [20, 64])
def test_square_is_det(n):
    rng = np.random.default_rng(n)
    A = rand_antisym(rng, n)
    la, ph = pfaffian(A)
    sd, ld = np.linalg.slogdet(A)
    assert np.isclose(2 * la, ld, rtol=0, atol=1e-9)
    assert np.isclose(ph * ph, sd, atol=1e-9)


def test_congruence():
    # pf(B^T A B) = det(B) pf(A)
    rng = np.random.default_rng(3)
    n = 12
    A = rand_antisym(rng, n)
    B = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    lhs = pfaffian_value(B.T @ A @ B)
    rhs = np.linalg.det(B) * pfaffian_value(A)
    assert np.isclose(lhs, rhs, rtol=1e-9)


def test_block_diagonal_and_permutation():
    a = np.array([1.5, -2.0 + 1j, 0.25j, 3.0])
    n = 2 * len(a)
    A = np.zeros((n, n), dtype=complex)
    for i, v in enumerate(a):
        A[2 * i, 2 * i + 1], A[2 * i + 1, 2 * i] = v, -v
    assert np.isclose(pfaffian_value(A), np.prod(a))
    # an odd permutation of the basis flips the sign
    P = np.eye(n)[[1, 0] + list(range(2, n))]
    assert np.isclose(pfaffian_value(P.T @ A @ P), -np.prod(a))
    la, ph = pfaffian_c(P.T @ A @ P)
    assert np.isclose(np.exp(la) * ph, -np.prod(a))


def test_large_modulus_no_overflow():
    # pf of a block-diagonal matrix with 400 blocks of 1e3: log|pf| = 400 log 1e3
    n = 800
    A = np.zeros((n, n), dtype=complex)
    for i in range(n // 2):
        A[2 * i, 2 * i + 1], A[2 * i + 1, 2 * i] = 1e3, -1e3
    la, ph = pfaffian_c(A)
    assert np.isclose(la, 400 * np.log(1e3)) and np.isclose(ph, 1.0)


def test_singular():
    A = np.zeros((4, 4), dtype=complex)
    A[0, 1], A[1, 0] = 1, -1
    assert pfaffian(A)[0] == -np.inf
