"""W_mass (Sec. 4, eq. Wmass) through the C-ABI against the oracle's dense S_j and R_j.

The library forms S_j as the product b^-1 i gamma_5 (mu_j - nu_j) a^-1 and inverts the
shifted operators by FP64 CG; the oracle forms the three printed terms with dense inverses.
Tolerance: the CG stops at ||r|| <= 1e-12 ||b||; q = (eta, R_j eta) then agrees to 1e-9 of
||eta||^2, and log W_mass (a sum of logarithms of means of exp(-q)) to the same level."""
import numpy as np
import pytest

from synth_inputs import make_config, random_spinor
from oracle.dirac import WilsonDirac
from oracle.evenodd import dhat_dense
from oracle.reweight import log_w_mass_estimate, quad_forms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import paper_2108_11989_gb300 as qs
    return qs


def _sources(cfg, nsrc, seed):
    import torch
    eta = random_spinor(seed, cfg.T, cfg.L, nrhs=nsrc).reshape(nsrc, -1)
    dev = torch.from_numpy(np.ascontiguousarray(np.stack([eta.real, eta.imag], -1))).cuda()
    return eta, dev


@pytest.mark.parametrize("shape,m,mp", [((4, 2, 0b111), -0.30, -0.28), ((6, 2, 0b101), -0.25, -0.31)])
def test_quadratic_forms_against_dense_oracle(qs, shape, m, mp):
    T, L, mask = shape
    cfg = make_config(T=T, L=L, eps=0.7, theta_sigma=0.3, csw_su3=1.5, csw_u1=1.0, seed=13, cstar_mask=mask)
    lat = qs.Lattice(L, T, mask)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    op = WilsonDirac(cfg)
    A, nu, mu, d = qs.ratapprox(2, 0.05, 6.0)
    eta, dev = _sources(cfg, 3, 21)
    q, lw, iters = lat.w_mass(m, mp, nu, mu, dev, tol=1e-12)
    _, e = dhat_dense(op, 0.0)
    ref = quad_forms(op, m, mp, nu, mu, eta[:, e])
    scale = np.max(np.sum(np.abs(eta[:, e]) ** 2, axis=1))
    assert q.shape == ref.shape and iters > 0
    assert np.max(np.abs(q - ref)) <= 1e-9 * scale, np.max(np.abs(q - ref))
    assert abs(lw - log_w_mass_estimate(ref)) <= 1e-9 * scale
    assert np.max(np.abs(ref)) > 1e-3                                   # a real reweighting
    lat.close()


def test_no_reweighting_at_equal_masses(qs):
    cfg = make_config(T=4, L=2, eps=0.7, theta_sigma=0.3, csw_su3=1.5, csw_u1=1.0, seed=13)
    lat = qs.Lattice(2, 4)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    _, dev = _sources(cfg, 2, 5)
    q, lw, _ = lat.w_mass(-0.3, -0.3, [0.8], [0.4], dev)
    assert np.all(q == 0.0) and lw == 0.0                               # delta D = 0 exactly
    lat.close()


def test_rejects_bad_arguments(qs):
    import torch
    cfg = make_config(T=5, L=2, eps=0.5, theta_sigma=0.2, csw_su3=1.0, csw_u1=0.0, seed=1)
    lat = qs.Lattice(2, 5)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    x = torch.zeros(lat.n_sites * 24, dtype=torch.float64, device="cuda")
    with pytest.raises(qs.QStarError):              # odd T: hops join sites of one parity
        lat.w_mass(-0.3, -0.2, [0.8], [0.4], x)
    lat.close()
    cfg = make_config(T=4, L=2, eps=0.5, theta_sigma=0.2, csw_su3=1.0, csw_u1=0.0, seed=1)
    lat = qs.Lattice(2, 4)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    x = torch.zeros(lat.n_sites * 24, dtype=torch.float64, device="cuda")
    with pytest.raises(qs.QStarError):              # a shift must be positive
        lat.w_mass(-0.3, -0.2, [0.8], [0.0], x)
    lat.close()
