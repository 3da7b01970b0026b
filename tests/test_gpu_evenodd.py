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
