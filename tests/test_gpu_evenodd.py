"""W_eo and log|det D^oo| (Sec. 4) through the C-ABI against the oracle's definition.
Tolerance 1e-11 relative on log|det D^oo| (FP64 site-local LU, summed in FP64)."""
import numpy as np
import pytest

from synth_inputs import GaugeConfig, make_config, unit_su3_field
from oracle.dirac import WilsonDirac
from oracle.evenodd import log_det_oo, w_eo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import paper_2108_11989_gb300 as qs
    return qs


@pytest.mark.parametrize("shape", [(4, 2, 0b111), (5, 6, 0b101), (4, 4, 0b011)])
def test_log_det_oo_against_oracle(qs, shape):
    T, L, mask = shape
    cfg = make_config(T=T, L=L, eps=0.7, theta_sigma=0.4, csw_su3=1.9, csw_u1=1.0, seed=3, cstar_mask=mask)
    lat = qs.Lattice(L, T, mask)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    op = WilsonDirac(cfg, lazy=True)
    masses = [-0.4, -0.2963, 0.1, 1.5]
    got = qs.log_det_oo(lat.h, masses)
    for m, g in zip(masses, got):
        ref = log_det_oo(op, m)
        assert abs(g - ref) <= 1e-11 * abs(ref), (m, g, ref)
    w, lw = qs.w_eo(lat.h, -0.4, -0.38)
    ref_w = w_eo(op, -0.4, -0.38)
    assert abs(w - ref_w) <= 1e-9 * ref_w
    lat.close()


def test_w_eo_free_field(qs):
    T, L = 4, 4
    lat = qs.Lattice(L, T)
    lat.load_gauge(unit_su3_field(T, L), None, 1.9, 0.0)
    n_odd = 2 * L ** 3 * T // 2
    w, lw = qs.w_eo(lat.h, -0.3, 0.7)
    assert abs(lw - 6 * n_odd * np.log(4.7 / 3.7)) <= 1e-11 * abs(lw)
    lat.close()


@pytest.mark.parametrize("shape,gamma5", [((4, 2, 0b111), False), ((4, 2, 0b111), True), ((4, 4, 0b011), True)])
def test_apply_dhat_against_dense_schur_complement(qs, shape, gamma5):
    """D_hat = D_ee - D_eo (D_oo)^-1 D_oe (Sec. 4) on even-site vectors against the oracle's
    dense Schur complement; FP64 throughout, tolerance 1e-12 relative to the largest entry."""
    import torch
    from oracle.evenodd import dhat_dense
    T, L, mask = shape
    cfg = make_config(T=T, L=L, eps=0.7, theta_sigma=0.4, csw_su3=1.9, csw_u1=1.0, seed=11, cstar_mask=mask)
    lat = qs.Lattice(L, T, mask)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    op = WilsonDirac(cfg)
    m0 = -0.35
    Dhat, e = dhat_dense(op, m0, gamma5=gamma5)
    n = op.lat.n_sites * 12
    rng = np.random.default_rng(4)
    nrhs = 3
    x = rng.normal(size=(nrhs, n)) + 1j * rng.normal(size=(nrhs, n))   # odd entries must be ignored
    xd = torch.from_numpy(np.stack([x.real, x.imag], -1)).to("cuda")
    yd = torch.full_like(xd, np.nan)
    lat.apply_Dhat(m0, xd, yd, gamma5=gamma5)
    y = yd.cpu().numpy()
    y = y[..., 0] + 1j * y[..., 1]
    odd = np.setdiff1d(np.arange(n), e)
    assert np.all(y[:, odd] == 0)
    ref = x[:, e] @ Dhat.T
    err = np.max(np.abs(y[:, e] - ref))
    assert err <= 1e-12 * np.max(np.abs(ref)), err
    lat.close()


def test_apply_dhat_rejects_odd_extent(qs):
    import torch
    cfg = make_config(T=5, L=2, eps=0.5, theta_sigma=0.2, csw_su3=1.0, csw_u1=0.0, seed=1)
    lat = qs.Lattice(2, 5)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    x = torch.zeros(lat.n_sites * 24, dtype=torch.float64, device="cuda")
    with pytest.raises(qs.QStarError):
        lat.apply_Dhat(0.0, x, torch.empty_like(x))
    lat.close()


@pytest.mark.parametrize("shape", [(4, 2, 0b111), (6, 2, 0b101)])
def test_solve_D_even_odd_and_full_against_dense(qs, shape):
    """x = D^-1 b by the even-odd preconditioned solve of Sec. 4 (and by CG on the full Q^2)
    against numpy's dense solve; CG to 1e-12, compared to 1e-9 of the largest entry."""
    import torch
    from synth_inputs import random_spinor
    T, L, mask = shape
    cfg = make_config(T=T, L=L, eps=0.7, theta_sigma=0.3, csw_su3=1.5, csw_u1=1.0, seed=17, cstar_mask=mask)
    lat = qs.Lattice(L, T, mask)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    op = WilsonDirac(cfg)
    m0 = -0.3
    b = random_spinor(8, T, L, nrhs=2).reshape(2, -1)
    ref = np.linalg.solve(op.dense_D(m0), b.T).T
    bd = torch.from_numpy(np.ascontiguousarray(np.stack([b.real, b.imag], -1))).cuda()
    its = {}
    for eo in (True, False):
        xd = torch.full_like(bd, float("nan"))
        its[eo] = lat.solve_D(m0, bd, xd, even_odd=eo, tol=1e-12)
        x = xd.cpu().numpy()
        x = x[..., 0] + 1j * x[..., 1]
        err = np.max(np.abs(x - ref)) / np.max(np.abs(ref))
        assert err < 1e-9, (eo, err)
        assert its[eo] > 0
    print(f"\n[solve_D] CG iterations even-odd {its[True]}, full {its[False]}")
    lat.close()
