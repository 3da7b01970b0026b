"""Dirac algebra in the chiral basis (Sec. 3: C = i gamma_0 gamma_2 "in the chiral basis").

Basis: gamma_0 = [[0, -1], [-1, 0]], gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 = diag(1, 1, -1, -1).
sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu].
Direction index: 0 = t, 1 = x, 2 = y, 3 = z.
Pinned by tests/test_oracle_gamma.py (Clifford algebra, C^T = -C,
C gamma_mu C^-1 = -gamma_mu^T, gamma_5 diagonal).
"""
import numpy as np

I2 = np.eye(2, dtype=np.complex128)
Z2 = np.zeros((2, 2), dtype=np.complex128)
PAULI = np.array([[[0, 1], [1, 0]],
                  [[0, -1j], [1j, 0]],
                  [[1, 0], [0, -1]]], dtype=np.complex128)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = np.zeros((4, 4, 4), dtype=np.complex128)
GAMMA[0] = _block(Z2, -I2, -I2, Z2)
for _k in range(3):
    GAMMA[_k + 1] = _block(Z2, -1j * PAULI[_k], 1j * PAULI[_k], Z2)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
CMAT = 1j * GAMMA[0] @ GAMMA[2]
SIGMA = np.zeros((4, 4, 4, 4), dtype=np.complex128)
for _m in range(4):
    for _n in range(4):
        SIGMA[_m, _n] = 0.5j * (GAMMA[_m] @ GAMMA[_n] - GAMMA[_n] @ GAMMA[_m])
ID4 = np.eye(4, dtype=np.complex128)
