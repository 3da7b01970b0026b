"""qs_apply_Q_norm2_noalloc through the C-ABI: the allocation-free variant must give
the same Q in as qs_apply_Q and the norms of its output, on consecutive calls.

This file is collected last so that a stop-at-first-failure run has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from synth_inputs import make_config, random_spinor

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_noalloc_matches_apply_Q_on_two_calls(prec, tol):
    import torch
    import paper_2108_11989_gb300 as qs
    cfg = make_config(T=6, L=4, eps=0.4, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0, seed=21)
    lat = qs.Lattice(cfg.L, cfg.T)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    dt = torch.float64 if prec == "f64" else torch.float32
    nrhs = 3
    m0 = -0.17
    for call in range(2):
        psi = random_spinor(40 + call, cfg.T, cfg.L, nrhs)
        x = torch.from_numpy(psi.view(np.float64).copy()).to(dt).cuda().reshape(-1)
        ref = torch.empty_like(x)
        lat.apply_Q(m0, x, ref)
        out = torch.full_like(x, float("nan"))
        nrm = torch.full((nrhs,), float("nan"), dtype=torch.float64, device="cuda")
        n0 = qs.kernel_launches()
        qs.apply_Q_norm2_noalloc(lat.h, m0, x, out, nrm)
        assert qs.kernel_launches() - n0 == 3     # the operator and the two-stage norm
        torch.cuda.synchronize()
        a, b = out.double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.abs(a - b).max() <= tol * np.abs(b).max()
        want = (ref.double().reshape(nrhs, -1) ** 2).sum(dim=1).cpu().numpy()
        got = nrm.cpu().numpy()
        assert np.all(np.abs(got - want) <= tol * want)
    lat.close()


def test_noalloc_rejects_more_rhs_than_its_scratch():
    import torch
    import paper_2108_11989_gb300 as qs
    cfg = make_config(T=2, L=2, eps=0.4, seed=3)
    lat = qs.Lattice(cfg.L, cfg.T)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    n = 65 * cfg.n_sites * 24
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    y = torch.zeros_like(x)
    nrm = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(qs.QStarError) as e:
        qs.apply_Q_norm2_noalloc(lat.h, 0.1, x, y, nrm)
    assert e.value.code == -1
    lat.close()
