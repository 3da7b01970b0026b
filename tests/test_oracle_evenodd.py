"""Pins of oracle/evenodd.py (Sec. 4: D^oo, W_eo, the even-odd Schur complement)."""
import numpy as np
import pytest

from synth_inputs import GaugeConfig, make_config, unit_su3_field
from oracle.dirac import WilsonDirac
from oracle.evenodd import dhat_dense, log_det_oo, parity, schur_det, w_eo


@pytest.fixture(scope="module")
def rough():
    cfg = make_config(T=4, L=2, eps=0.9, theta_sigma=0.4, csw_su3=1.3, csw_u1=0.8, seed=5)
    return WilsonDirac(cfg)


def test_odd_odd_part_is_site_diagonal_and_matches_blocks(rough):
    D = rough.dense_D(-0.4)
    p = np.repeat(parity(rough.lat), 12)
    o = np.nonzero(p == 1)[0]
    Doo = D[np.ix_(o, o)]
    site = o // 12
    off_site = site[:, None] != site[None, :]
    assert np.max(np.abs(Doo[off_site])) == 0.0          # no hopping between odd sites
    assert np.isclose(np.linalg.slogdet(Doo)[1], log_det_oo(rough, -0.4), rtol=1e-12)


def test_schur_identity(rough):
    loo, lhat, ld = schur_det(rough, 0.25)
    assert np.isclose(loo + lhat, ld, rtol=1e-11)
    assert np.isclose(loo, log_det_oo(rough, 0.25), rtol=1e-12)


def test_free_field_closed_form():
    T, L = 4, 2
    op = WilsonDirac(GaugeConfig(T, L, unit_su3_field(T, L), None, 1.9, 1.0))
    n_odd = op.lat.n_sites // 2
    for m0 in (-0.3, 0.7):
        assert np.isclose(log_det_oo(op, m0), 12 * n_odd * np.log(abs(4.0 + m0)), rtol=1e-13)
    assert np.isclose(w_eo(op, -0.3, 0.7), (4.7 / 3.7) ** (6 * n_odd), rtol=1e-12)


def test_dhat_inverts_the_full_solve_on_even_sites(rough):
    # D y = (b_e, 0)  =>  D_hat y_e = b_e  (block elimination of the odd sites)
    m0 = -0.35
    Dhat, e = dhat_dense(rough, m0)
    rng = np.random.default_rng(3)
    n = rough.dense_D(m0).shape[0]
    b = np.zeros(n, complex)
    b[e] = rng.normal(size=e.size) + 1j * rng.normal(size=e.size)
    y = np.linalg.solve(rough.dense_D(m0), b)
    assert np.allclose(Dhat @ y[e], b[e], rtol=0, atol=1e-11 * np.abs(b).max())
    assert np.array_equal(e, np.nonzero(np.repeat(parity(rough.lat), 12) == 0)[0])


def test_qhat_is_hermitian(rough):
    # gamma_5 D is Hermitian, so its Schur complement gamma_5 D_hat is Hermitian too
    Qhat, _ = dhat_dense(rough, 0.1, gamma5=True)
    Dhat, _ = dhat_dense(rough, 0.1)
    assert np.max(np.abs(Qhat - Qhat.conj().T)) < 1e-12 * np.abs(Qhat).max()
    assert np.max(np.abs(Dhat - Dhat.conj().T)) > 1e-3 * np.abs(Dhat).max()   # D_hat itself is not


def test_dhat_free_field_closed_form():
    # free field: A = 0, so D_oo = (4 + m0) and D_hat = (4 + m0) - H_eo H_oe / (4 + m0),
    # H the hopping part of D (D minus its diagonal), formed here without any inverse
    T, L = 4, 2
    op = WilsonDirac(GaugeConfig(T, L, unit_su3_field(T, L), None, 1.9, 1.0))
    m0 = -0.3
    D = op.dense_D(m0)
    H = D - (4.0 + m0) * np.eye(D.shape[0])
    p = np.repeat(parity(op.lat), 12)
    e, o = np.nonzero(p == 0)[0], np.nonzero(p == 1)[0]
    assert np.max(np.abs(H[np.ix_(e, e)])) == 0 and np.max(np.abs(H[np.ix_(o, o)])) == 0
    closed = (4.0 + m0) * np.eye(len(e)) - H[np.ix_(e, o)] @ H[np.ix_(o, e)] / (4.0 + m0)
    Dhat, e2 = dhat_dense(op, m0)
    assert np.array_equal(e, e2)
    assert np.max(np.abs(Dhat - closed)) < 1e-13
