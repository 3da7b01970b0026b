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


@pytest.mark.parametrize("retreat", [False, True])
def test_flow_matches_definition(rough, retreat):
    op, pairs = rough
    for m in [-2.05, -1.65, -1.5, 0.3]:
        s, rep = pfaffian_sign_flow(lambda mm: modes_dense(op, mm, 24), m, m0_max_default(op.cfg),
                                    retreat=retreat)
        assert s == sign_from_real_eigs(pairs, m), (m, retreat)
    for m in [-1.65, -1.5]:
        s2, _ = pfaffian_sign_flow(lambda mm: modes_sparse(op, mm, 16), m, m0_max_default(op.cfg),
                                   retreat=retreat)
        assert s2 == sign_from_real_eigs(pairs, m)


def test_flow_step_a_follows_the_enumerated_algorithm(rough):
    """Paper order (Sec. 3): while lambda_bar grows every step-A step is exactly
    c lambda_bar; the first decrease hands over to step B, which starts from a mass
    whose crossing-free interval reaches the next mass visited."""
    op, _ = rough
    c = 1.9
    s, rep = pfaffian_sign_flow(lambda mm: modes_dense(op, mm, 24), -1.65, m0_max_default(op.cfg), c=c)
    m, lb, ph = rep["masses"], rep["lambda_bar"], rep["phase"]
    assert "B" in ph
    i = 0
    while ph[i + 1] == "A":
        assert m[i + 1] > m[i]
        if lb[i + 1] < lb[i]:
            break
        assert np.isclose(m[i + 1] - m[i], c * lb[i], rtol=1e-12)     # step 5
        i += 1
    # the first B mass continues from a certified mass: within lambda_bar of one of the
    # step-A masses before it, above it
    j = ph.index("B")
    starts = [k for k in range(j) if m[k] < m[j] and m[j] - m[k] <= lb[k] + 1e-12]
    assert starts


def test_flow_retreat_option_shortens_uncovered_steps():
    """A window function that makes lambda_bar collapse after the first step: the paper
    order goes to step B from the first mass; the retreat option first tries the edge
    of the crossing-free interval, m0 + 0.95 lambda_bar."""
    def modes(m):      # a pair +-lambda that dips to 1e-3 at m = 1 + 0.95 * 1.002
        lam = abs(0.5 - 0.5253 * (m - 1.0)) + 1e-3
        w = np.array([lam, -lam, 3.0, -3.0, 4.0, -4.0])
        return w, np.zeros(6)
    s0, r0 = pfaffian_sign_flow(modes, 1.0, 3.0, max_steps=50)
    s1, r1 = pfaffian_sign_flow(modes, 1.0, 3.0, max_steps=50, retreat=True)
    assert s0 == s1 == 1
    assert r0["phase"][:3] == ["A", "A", "B"] and r0["masses"][2] > 1.0
    assert r1["phase"][:4] == ["A", "A", "A", "B"]
    assert np.isclose(r1["masses"][2], 1.0 + 0.95 * 0.501)


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


def test_lowmodes_sparse_free_field_closed_form():
    """modes_sparse on a free 2^3 x 6 field (n = 1152): the 12 eigenvalues nearest zero
    equal the closed-form C* spectrum +-sqrt(M(p)^2 + sum sin^2 p) (Sec. 2 operator)."""
    from synth_inputs import GaugeConfig, unit_su3_field
    T, L, m0 = 6, 2, -0.35
    op = WilsonDirac(GaugeConfig(T, L, unit_su3_field(T, L), None, 1.9, 1.0))
    ev = []
    for n1 in range(2 * L):
        p1 = np.pi * n1 / L
        for n2 in range(L):
            for n3 in range(L):
                for n0 in range(T):
                    p = np.array([2 * np.pi * n0 / T, p1, p1 + 2 * np.pi * n2 / L, p1 + 2 * np.pi * n3 / L])
                    M = m0 + np.sum(1 - np.cos(p))
                    e = np.sqrt(M * M + np.sum(np.sin(p) ** 2))
                    ev += [e] * 6 + [-e] * 6
    ev = np.array(ev)
    ref = np.sort(np.abs(ev))[:12]
    ws, rs = modes_sparse(op, m0, 12)
    assert np.allclose(np.sort(np.abs(ws)), ref, atol=1e-10)
    assert np.all(rs < 1e-9)
