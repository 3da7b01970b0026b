"""Pins of oracle/gamma.py: Clifford algebra and charge conjugation (Sec. 3: C = i g0 g2)."""
import numpy as np

from oracle.gamma import GAMMA, GAMMA5, CMAT, SIGMA


def test_clifford():
    for m in range(4):
        assert np.allclose(GAMMA[m], GAMMA[m].conj().T)
        for n in range(4):
            ac = GAMMA[m] @ GAMMA[n] + GAMMA[n] @ GAMMA[m]
            assert np.allclose(ac, 2.0 * (m == n) * np.eye(4))


def test_gamma5_chiral():
    # chiral basis: gamma_5 diagonal with the upper two components positive
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]))


def test_charge_conjugation():
    Ci = np.linalg.inv(CMAT)
    assert np.allclose(CMAT.T, -CMAT)                       # antisymmetric
    for m in range(4):
        assert np.allclose(CMAT @ GAMMA[m] @ Ci, -GAMMA[m].T)
    assert np.allclose(CMAT @ GAMMA5 @ Ci, GAMMA5.T)


def test_sigma_blocks():
    # sigma_{mu nu} are Hermitian and commute with gamma_5 (block diagonal)
    for m in range(4):
        for n in range(4):
            S = SIGMA[m, n]
            assert np.allclose(S, S.conj().T)
            assert np.allclose(S @ GAMMA5, GAMMA5 @ S)
    # hand-derived values in this basis: sigma_12 = -diag(s3, s3), sigma_01 = diag(s1, -s1)
    s1 = np.array([[0, 1], [1, 0]])
    s3 = np.diag([1, -1])
    z = np.zeros((2, 2))
    assert np.allclose(SIGMA[1, 2], -np.block([[s3, z], [z, s3]]))
    assert np.allclose(SIGMA[0, 1], np.block([[s1, z], [z, -s1]]))
