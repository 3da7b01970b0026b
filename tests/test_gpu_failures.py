"""Failure statuses of the C-ABI, each provoked on the host (no GPU fault is involved):
QS_ENOCONV for an iteration cap of zero, QS_ENUMERIC for a NaN in the host gauge
array, QS_EUNDECIDED for an exact zero mode at the target mass (free field at
m0 = 0, where the p = 0 modes of Q vanish: Sec. 3, lambda_bar = 0)."""
import numpy as np
import pytest

from synth_inputs import make_config, unit_su3_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import paper_2108_11989_gb300 as qs
    return qs


def test_zero_iteration_cap_is_enoconv(qs):
    cfg = make_config(T=4, L=2, eps=0.5, theta_sigma=0.3, csw_su3=1.5, csw_u1=1.0, seed=1)
    lat = qs.Lattice(cfg.L, cfg.T)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    ev, rs, st = lat.lowmodes_at_mass(-0.2, qs.eig_default_opts(k=8, nwant=2, max_iter=0), allow_noconv=True)
    assert st["status"] == -4
    with pytest.raises(qs.QStarError) as e:
        lat.pfaffian_sign(-0.2, qs.sign_default_opts(eig={"k": 8, "nwant": 2, "max_iter": 0}))
    assert e.value.code == -4 and e.value.report["fail_reason"] == 1
    lat.close()


@pytest.mark.parametrize("where", ["su3", "theta"])
def test_nan_in_gauge_field_is_enumeric(qs, where):
    cfg = make_config(T=4, L=2, eps=0.5, theta_sigma=0.3, csw_su3=1.5, csw_u1=1.0, seed=1)
    su3, th = cfg.su3.copy(), cfg.theta.copy()
    if where == "su3":
        su3[1, 0, 1, 0, 2, 1, 1] = np.nan
    else:
        th[3, 1, 0, 1, 0] = np.inf
    lat = qs.Lattice(cfg.L, cfg.T)
    with pytest.raises(qs.QStarError) as e:
        lat.load_gauge(su3, th, cfg.csw_su3, cfg.csw_u1)
    assert e.value.code == -6
    # nothing is loaded: the operator refuses to run
    import torch
    x = torch.zeros(cfg.n_sites * 24, dtype=torch.float64, device="cuda")
    with pytest.raises(qs.QStarError) as e2:
        lat.apply_Q(0.1, x, torch.empty_like(x))
    assert e2.value.code == -1
    # a clean field loads afterwards on the same handle
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    lat.close()


def test_free_field_zero_mode_is_undecided(qs):
    T, L = 4, 4
    lat = qs.Lattice(L, T)
    lat.load_gauge(unit_su3_field(T, L), None, 1.9, 0.0)
    opts = qs.sign_default_opts(eig={"k": 16, "nwant": 2, "tol": 1e-6, "precision": 0, "cheb_degree": 16})
    with pytest.raises(qs.QStarError) as e:
        lat.pfaffian_sign(0.0, opts)
    assert e.value.code == -7 and e.value.report["fail_reason"] == 6
    # just above the crossing the sign is decided: no eigenvalue crosses above m0 = 0.1
    s, rep = lat.pfaffian_sign(0.1, opts)
    assert s == 1
    lat.close()
