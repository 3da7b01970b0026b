"""The low modes of the benchmark field (16^3 x 32, N_s = 262144, n = 3.1M) certified by
the oracle: the GPU returns Ritz pairs (theta_i, v_i) with residual bounds r_i, and the
oracle's plain-loop C operator recomputes ||Q v_i - theta_i v_i|| for each.  By the
residual bound for Hermitian matrices an eigenvalue of Q lies within that distance of
theta_i, so the check certifies the eigenvalues without trusting the GPU's own numbers.
Also checked: orthonormality of the returned vectors and the double degeneracy of Sec. 3
(pairs of equal theta).  Tolerances: the oracle's residual may exceed the GPU's by 1e-6
relative plus 1e-12 (different summation order); Gram matrix within 1e-12 of 1."""
import numpy as np
import pytest

from synth_inputs import WORKLOADS, kappa_to_m0, make_config

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [2])      # the benchmark's FP16 filter storage
def test_16x32_ritz_pairs_certified_by_oracle_operator(precision):
    import torch
    import paper_2108_11989_gb300 as qs
    from oracle.dirac import WilsonDiracC
    cfg = make_config(seed=0, **WORKLOADS["qcdqed_16x16x16x32"])
    m0 = kappa_to_m0(0.135)
    lat = qs.Lattice(cfg.L, cfg.T)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    k, nw = 32, 8
    V = torch.zeros(k * cfg.n_sites * 24, dtype=torch.float64, device="cuda")
    opts = qs.eig_default_opts(k=k, nwant=nw, tol=1e-8, cheb_degree=48, precision=precision, warm_start=0)
    ev, rs, st = lat.lowmodes_at_mass(m0, opts, evecs=V)
    v = V.cpu().numpy().view(np.complex128).reshape(k, -1)[:nw].copy()
    del V
    lat.close()
    assert np.all(rs[:nw] <= 1e-8 * np.abs(ev[:nw]))
    op = WilsonDiracC(cfg)
    r = op.residuals(v, ev[:nw], m0)
    assert np.all(r <= rs[:nw] * (1 + 1e-6) + 1e-12), (r, rs[:nw])
    assert np.all(r <= 1e-8 * np.abs(ev[:nw]) * (1 + 1e-6) + 1e-12)
    G = v.conj() @ v.T
    assert np.abs(G - np.eye(nw)).max() < 1e-12
    s = np.sort(ev[:nw])
    assert np.allclose(s[0::2], s[1::2], rtol=1e-8)
