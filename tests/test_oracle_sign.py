"""Pins of oracle/sign.py and oracle/lowmodes.py (Sec. 3).

The sign is checked three independent ways on tiny rough configurations that do
have negative Pfaffians: the dense Pfaffian ratio (definition), the negative
eigenvalue count of Q (the theorem pf = prod lambda_n), and the real eigenvalues
mu of D(0): det D(m0) = prod (mu + m0), so sign pf(m0) = prod over real mu (one
per degenerate pair) of sign(mu + m0).  The mass flow must reproduce them.
"""
import numpy as np
import pytest

from synth_inputs import make_config
from oracle.dirac import WilsonDirac
from oracle.lowmodes import modes_dense, modes_sparse
from oracle.sign import (m0_max_default, negative_count, pfaffian_sign_flow, sign_by_eigencount,
                         sign_by_pfaffian)


@pytest.fixture(scope="module")
def rough():
    cfg = make_config(T=4, L=2, eps=2.0, theta_sigma=0.3, csw_su3=1.5, csw_u1=1.0, seed=2)
    op = WilsonDirac(cfg)
    mu = np.linalg.eigvals(op.dense_D(0.0))
    real = np.sort(mu[np.abs(mu.imag) < 1e-9].real)
    assert len(real) % 2 == 0
    pairs = real[0::2]
    assert np.allclose(real[0::2], real[1::2], atol=1e-8)
    return op, pairs


def sign_from_real_eigs(pairs, m0):
    return int(np.prod(np.sign(pairs + m0)))


MASSES = [-2.2, -2.05, -1.85, -1.65, -1.5, -0.5, 0.3]


def test_three_routes_agree(rough):
    op, pairs = rough
    signs = []
    for m in MASSES:
        a, ratio = sign_by_pfaffian(op, m)
        b = sign_by_eigencount(op, m)
        c = sign_from_real_eigs(pairs, m)
        assert abs(ratio.imag) < 1e-8 * abs(ratio)
        assert a == b == c, (m, a, b, c)
        signs.append(a)
    assert -1 in signs and 1 in signs


def test_flow_matches_definition(rough):
    op, pairs = rough
    for m in [-2.05, -1.65, -1.5, 0.3]:
        s, rep = pfaffian_sign_flow(lambda mm: modes_dense(op, mm, 24), m, m0_max_default(op.cfg))
        assert s == sign_from_real_eigs(pairs, m), m
    for m in [-1.65, -1.5]:
        s2, _ = pfaffian_sign_flow(lambda mm: modes_sparse(op, mm, 16), m, m0_max_default(op.cfg))
        assert s2 == sign_from_real_eigs(pairs, m)


def test_large_mass_positive(rough):
    op, _ = rough
    m = m0_max_default(op.cfg) + 1e-9
    w = np.linalg.eigvalsh(op.dense_Q(m))
    assert np.min(np.abs(w)) > 0
    assert negative_count(op, m) == op.n // 2          # Q ~ m0 gamma_5: half negative
    assert sign_by_eigencount(op, m) == 1


def test_feynman_hellmann_bound(rough):
    """|lambda_n(m + d) - lambda_n(m)| <= d for the ordered spectra (eq. derivativebound)."""
    op, _ = rough
    m, d = -1.0, 0.05
    w1 = np.linalg.eigvalsh(op.dense_Q(m))
    w2 = np.linalg.eigvalsh(op.dense_Q(m + d))
    assert np.max(np.abs(w2 - w1)) <= d + 1e-12
    # and d/dm lambda = (v, gamma_5 v) lies in [-1, 1]
    w, V = np.linalg.eigh(op.dense_Q(m))
    g5 = np.tile(np.repeat([1, 1, -1, -1], 3), op.lat.n_sites)
    dl = np.real(np.sum(V.conj() * g5[:, None] * V, axis=0))
    w_eps = np.linalg.eigvalsh(op.dense_Q(m + 1e-6))
    assert np.allclose((w_eps - w) / 1e-6, dl, atol=1e-4)


def test_lowmodes_sparse_vs_dense(rough):
    op, _ = rough
    wd, _ = modes_dense(op, -1.3, 8)
    ws, rs = modes_sparse(op, -1.3, 8)
    assert np.allclose(np.sort(wd), np.sort(ws), atol=1e-10)
    assert np.all(rs < 1e-9)
