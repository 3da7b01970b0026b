"""Pins of oracle/reweight.py (Sec. 4: rational approximation R, W_mass and its estimator)."""
import numpy as np
import pytest

from synth_inputs import make_config, random_spinor
from oracle.dirac import WilsonDirac
from oracle.reweight import (log_w_mass_estimate, log_w_mass_exact, log_w_mass_spectral, quad_forms,
                             r_matrices, rat_eval, ratapprox)


def _extrema_signs(e):
    """(value, sign) of the largest |e| on each run of one sign, in order."""
    out, start = [], 0
    for i in range(1, len(e) + 1):
        if i == len(e) or np.sign(e[i]) != np.sign(e[start]):
            k = start + int(np.argmax(np.abs(e[start:i])))
            out.append((abs(e[k]), np.sign(e[k])))
            start = i
    return out


def test_best_constant_closed_form():
    # n = 0: A y^p - 1 takes -delta at y_a and +delta at y_b
    ra, rb, p = 0.1, 2.0, 0.25
    A, nu, mu, d = ratapprox(0, ra, rb)
    ya, yb = (ra * ra) ** p, (rb * rb) ** p
    assert np.isclose(A, 2.0 / (ya + yb), rtol=1e-14)
    assert np.isclose(d, (yb - ya) / (yb + ya), rtol=1e-12)


@pytest.mark.parametrize("n,ratio", [(1, 10.0), (2, 10.0), (3, 30.0), (4, 100.0)])
def test_equioscillation_certifies_optimality(n, ratio):
    """Alternation theorem: a non-degenerate (n, n) rational function whose relative error
    reaches its maximum with alternating signs at 2n + 2 points is the best one; by de la
    Vallee Poussin's bound the least of 2n + 2 alternating extrema is a lower bound of the
    best error, so levelling to 1e-4 puts delta within 1e-4 of the optimum."""
    ra, rb = 1.0 / ratio, 1.0
    A, nu, mu, d = ratapprox(n, ra, rb)
    assert len(nu) == n and len(mu) == n and np.all(nu > 0) and np.all(mu > 0)
    y = np.exp(np.linspace(np.log(ra * ra), np.log(rb * rb), 400001))
    e = rat_eval(A, nu, mu, y) * y ** 0.25 - 1
    ext = _extrema_signs(e)
    assert len(ext) >= 2 * n + 2
    mags = np.array([m for m, _ in ext])
    top = np.sort(mags)[-(2 * n + 2):]
    assert np.max(mags) == pytest.approx(d, rel=1e-9)
    assert np.min(top) >= d * (1 - 1e-4)                      # levelled
    # the 2n + 2 largest ones alternate in sign
    idx = np.sort(np.argsort(mags)[-(2 * n + 2):])
    s = np.array([ext[i][1] for i in idx])
    assert np.all(s[1:] == -s[:-1])
    # zeros and poles interlace on the negative axis (R decreases like y^-1/4)
    lab = np.concatenate([np.zeros(n), np.ones(n)])[np.argsort(np.concatenate([mu, nu]))]
    assert np.all(lab[0::2] == 0) and np.all(lab[1::2] == 1)   # mu_1 < nu_1 < mu_2 < nu_2 ...


def test_error_falls_with_order():
    ds = [ratapprox(n, 0.05, 1.0)[3] for n in (1, 2, 3, 4)]
    assert all(b < 0.5 * a for a, b in zip(ds, ds[1:]))


@pytest.fixture(scope="module")
def rough():
    cfg = make_config(T=4, L=2, eps=0.8, theta_sigma=0.3, csw_su3=1.5, csw_u1=1.0, seed=9)
    return cfg, WilsonDirac(cfg)


def test_exact_w_mass_equals_spectral_ratio(rough):
    """prod_j 1/det(1 + R_j), with S_j and R_j as printed, equals
    det R(Q_hat_m^2) / det R(Q_hat_m'^2) for any nu, mu (the identity behind eq. Wmass)."""
    _, op = rough
    nu, mu = np.array([0.9, 0.35]), np.array([0.6, 0.2])
    for m, mp in [(-0.3, -0.28), (-0.3, -0.36), (0.1, 0.25)]:
        ex = log_w_mass_exact(op, m, mp, nu, mu)
        sp = log_w_mass_spectral(op, m, mp, 1.7, nu, mu)
        assert abs(ex - sp) <= 1e-9 * max(1.0, abs(sp)), (m, mp, ex, sp)
        assert abs(sp) > 1e-3                                    # not trivially zero
    # m' = m: no reweighting
    assert abs(log_w_mass_exact(op, -0.3, -0.3, nu, mu)) < 1e-12


def test_r_j_hermitian_and_one_plus_r_positive(rough):
    _, op = rough
    for R in r_matrices(op, -0.3, -0.27, np.array([0.8]), np.array([0.5])):
        assert np.max(np.abs(R - R.conj().T)) < 1e-12 * max(1.0, np.abs(R).max())
        assert np.min(np.linalg.eigvalsh(np.eye(R.shape[0]) + R)) > 0


def test_gaussian_estimator_is_inverse_determinant():
    """E[exp(-(eta, R eta))] = 1/det(1 + R) for complex eta with density ~ exp(-(eta, eta)),
    the sources of random_spinor; Monte Carlo within 4 standard errors."""
    rng = np.random.default_rng(1)
    M = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    R = 0.3 * (M + M.conj().T) / 2 + 0.2 * np.eye(3)
    assert np.min(np.linalg.eigvalsh(np.eye(3) + R)) > 0
    eta = random_spinor(5, 1, 1, nrhs=200000).reshape(200000, -1)[:, :3]
    f = np.exp(-np.real(np.einsum("li,ij,lj->l", eta.conj(), R, eta)))
    exact = 1.0 / np.real(np.linalg.det(np.eye(3) + R))
    assert abs(f.mean() - exact) < 4 * f.std() / np.sqrt(len(f))
    q = np.real(np.einsum("li,ij,lj->l", eta.conj(), R, eta))[None, :]
    assert np.isclose(log_w_mass_estimate(q), np.log(f.mean()), rtol=1e-12)


def test_quad_forms_match_dense_r(rough):
    cfg, op = rough
    nu, mu = np.array([0.7]), np.array([0.45])
    R = r_matrices(op, -0.3, -0.29, nu, mu)[0]
    from oracle.evenodd import dhat_dense
    _, e = dhat_dense(op, 0.0)
    eta = random_spinor(3, cfg.T, cfg.L, nrhs=2).reshape(2, -1)[:, e]
    q = quad_forms(op, -0.3, -0.29, nu, mu, eta)
    for l in range(2):
        assert np.isclose(q[0, l], np.real(eta[l].conj() @ R @ eta[l]), rtol=1e-12)
