"""Low eigenvalues of Q (qs_lowmodes_at_mass through the C-ABI) against the oracle.

Tolerance: 1e-10 relative on every wanted eigenvalue (FP64 Rayleigh-Ritz), and
each reported residual must bound the distance to a true eigenvalue.
"""
import json
import os

import numpy as np
import pytest

from synth_inputs import WORKLOADS, kappa_to_m0, make_config
from oracle.dirac import WilsonDirac
from oracle.lowmodes import modes_dense

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def qs():
    import paper_2108_11989_gb300 as qs
    return qs


def lattice(qs, cfg):
    lat = qs.Lattice(cfg.L, cfg.T, cfg.cstar_mask, cfg.t_antiperiodic)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    return lat


def check_against(ev, rs, ref, nwant, rtol=1e-10):
    ref_sorted = ref[np.argsort(np.abs(ref), kind="stable")]
    for i in range(nwant):
        j = np.argmin(np.abs(ref_sorted - ev[i]))
        assert abs(ev[i] - ref_sorted[j]) <= rtol * abs(ref_sorted[j]) + 1e-14, (i, ev[i], ref_sorted[j])
        assert abs(ev[i] - ref_sorted[j]) <= rs[i] + 1e-12
    # the wanted Ritz values are the smallest |lambda| (pairs counted twice)
    assert np.allclose(np.sort(np.abs(ev[:nwant])), np.abs(ref_sorted[:nwant]), rtol=rtol, atol=1e-14)


@pytest.mark.parametrize("m0", [-0.6, 0.1])
def test_small_rough_lattice_dense_reference(qs, m0):
    cfg = make_config(T=4, L=2, eps=0.9, theta_sigma=0.4, csw_su3=1.3, csw_u1=0.8, seed=5)
    lat = lattice(qs, cfg)
    opts = qs.eig_default_opts(k=16, nwant=8, tol=1e-9, cheb_degree=16)
    ev, rs, st = lat.lowmodes_at_mass(m0, opts)
    ref = np.linalg.eigvalsh(WilsonDirac(cfg).dense_Q(m0))
    check_against(ev, rs, ref, 8)
    lat.close()


def test_tiny_workload_golden(qs):
    """4^4 workload: the 8 lowest |lambda| at the 4 golden masses (dense oracle values)."""
    g = json.load(open(os.path.join(HERE, "golden", "tiny_4x4x4x4_seed0.json")))
    cfg = make_config(seed=0, **WORKLOADS["tiny_4x4x4x4"])
    lat = lattice(qs, cfg)
    opts = qs.eig_default_opts(k=16, nwant=8, tol=1e-9, cheb_degree=24)
    for pt in g["points"]:
        ev, rs, st = lat.lowmodes_at_mass(pt["m0"], opts)
        ref = np.array(pt["lowest_abs_sorted_eigs_Q"])
        check_against(ev, rs, ref, 8)
    lat.close()


def test_pairs_are_degenerate(qs):
    cfg = make_config(T=4, L=4, eps=0.5, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0, seed=2)
    lat = lattice(qs, cfg)
    ev, rs, st = lat.lowmodes_at_mass(-0.2, qs.eig_default_opts(k=16, nwant=8, tol=1e-9))
    s = np.sort(ev[:8])
    assert np.allclose(s[0::2], s[1::2], rtol=1e-9, atol=1e-13)
    lat.close()


def test_eigenvectors_returned(qs):
    import torch
    cfg = make_config(T=4, L=2, eps=0.9, theta_sigma=0.4, csw_su3=1.3, csw_u1=0.8, seed=5)
    lat = lattice(qs, cfg)
    k = 8
    V = torch.zeros(k * cfg.n_sites * 24, dtype=torch.float64, device="cuda")
    ev, rs, st = lat.lowmodes_at_mass(-0.6, qs.eig_default_opts(k=k, nwant=4, tol=1e-9), evecs=V)
    v = V.cpu().numpy().view(np.complex128).reshape(k, -1)
    op = WilsonDirac(cfg)
    for i in range(4):
        r = op.apply_Q(v[i], -0.6) - ev[i] * v[i]
        assert np.linalg.norm(r) <= 1e-8 * abs(ev[i]) + 1e-12
        assert abs(np.linalg.norm(v[i]) - 1) < 1e-12
    lat.close()


def test_plain_fp64_form_matches(qs):
    """precision = QS_F64 (FP64 filter and Rayleigh-Ritz only) gives the same low
    eigenvalues as the dense oracle."""
    cfg = make_config(T=4, L=2, eps=0.9, theta_sigma=0.4, csw_su3=1.3, csw_u1=0.8, seed=5)
    lat = lattice(qs, cfg)
    opts = qs.eig_default_opts(k=16, nwant=8, tol=1e-9, cheb_degree=16, precision=0, max_iter=400)
    ev, rs, st = lat.lowmodes_at_mass(-0.6, opts)
    ref = np.linalg.eigvalsh(WilsonDirac(cfg).dense_Q(-0.6))
    check_against(ev, rs, ref, 8)
    assert st["dslash_f32"] == 0 and st["refine_passes"] == 0
    lat.close()


@pytest.mark.parametrize("precision", [2, 3])   # QS_F16, QS_BF16 filter storage
def test_16bit_filter_storage_keeps_fp64_accuracy(qs, precision):
    """The filter's vectors in 16 bits (per-site scale): the FP64 Rayleigh-Ritz and the
    mixed refinement still give the dense oracle's low eigenvalues to 1e-10."""
    cfg = make_config(T=4, L=2, eps=0.9, theta_sigma=0.4, csw_su3=1.3, csw_u1=0.8, seed=5)
    lat = lattice(qs, cfg)
    opts = qs.eig_default_opts(k=16, nwant=8, tol=1e-9, cheb_degree=16, precision=precision)
    ev, rs, st = lat.lowmodes_at_mass(-0.6, opts)
    ref = np.linalg.eigvalsh(WilsonDirac(cfg).dense_Q(-0.6))
    check_against(ev, rs, ref, 8)
    assert st["filter_passes"] > 0
    lat.close()


def test_16bit_filter_on_tiny_workload_golden(qs):
    g = json.load(open(os.path.join(HERE, "golden", "tiny_4x4x4x4_seed0.json")))
    cfg = make_config(seed=0, **WORKLOADS["tiny_4x4x4x4"])
    lat = lattice(qs, cfg)
    opts = qs.eig_default_opts(k=16, nwant=8, tol=1e-9, cheb_degree=24, precision=2)
    pt = g["points"][0]
    ev, rs, st = lat.lowmodes_at_mass(pt["m0"], opts)
    check_against(ev, rs, np.array(pt["lowest_abs_sorted_eigs_Q"]), 8)
    lat.close()


def test_cstar_partner_of_eigenvectors(qs):
    """qs_cstar_partner maps an eigenvector of Q (oracle) to an orthogonal eigenvector
    with the same eigenvalue (Sec. 3), equal to the oracle's C T gamma_5 v^*, and P^2 = -1."""
    import torch
    from oracle.dirac import gamma5_vec
    cfg = make_config(T=4, L=2, eps=0.9, theta_sigma=0.4, csw_su3=1.3, csw_u1=0.8, seed=5)
    op = WilsonDirac(cfg)
    lat = lattice(qs, cfg)
    m0 = -0.6
    w, V = np.linalg.eigh(op.dense_Q(m0))
    v = np.ascontiguousarray(V[:, [0, 5, 100]].T)
    x = torch.from_numpy(v.view(np.float64).copy()).cuda().reshape(-1)
    y = torch.empty_like(x)
    qs.cstar_partner(lat.h, x, y)
    u = y.cpu().numpy().view(np.complex128).reshape(3, -1)
    CT = op.CT_matrix()
    Q = op.dense_Q(m0)
    for i, col in enumerate([0, 5, 100]):
        ref = CT @ gamma5_vec(v[i].conj())
        assert np.abs(u[i] - ref).max() < 1e-14
        assert np.abs(Q @ u[i] - w[col] * u[i]).max() < 1e-11
        assert abs(np.vdot(v[i], u[i])) < 1e-11
    z = torch.empty_like(x)
    qs.cstar_partner(lat.h, y, z)
    assert torch.allclose(z, -x, atol=0, rtol=0)
    # the tiled layout gives the same map
    xt, yt = qs.to_tiled(x, cfg.n_sites), torch.empty_like(x)
    qs.cstar_partner(lat.h, xt, yt, tiled=True)
    assert torch.equal(qs.from_tiled(yt, cfg.n_sites), y)
    lat.close()


def test_graph_replayed_filter_on_own_stream(qs):
    """A handle with its own stream captures the filter loop as a CUDA graph after the
    first pass and replays it; the low eigenvalues still match the dense oracle (4^4
    golden), with FP16 and FP32 filter storage, and a gauge reload invalidates the graph."""
    import torch
    g = json.load(open(os.path.join(HERE, "golden", "tiny_4x4x4x4_seed0.json")))
    cfg = make_config(seed=0, **WORKLOADS["tiny_4x4x4x4"])
    st = torch.cuda.Stream()
    lat = qs.Lattice(cfg.L, cfg.T, stream=st)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    for precision in (2, 1):
        opts = qs.eig_default_opts(k=16, nwant=8, tol=1e-9, cheb_degree=24, precision=precision, warm_start=0)
        for pt in g["points"][:2]:
            ev, rs, stats = lat.lowmodes_at_mass(pt["m0"], opts)
            check_against(ev, rs, np.array(pt["lowest_abs_sorted_eigs_Q"]), 8)
            assert stats["filter_passes"] >= 2
    # a different field on the same handle: graphs captured with the old one are not reused
    other = make_config(T=4, L=4, eps=0.5, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0, seed=2)
    lat.load_gauge(other.su3, other.theta, other.csw_su3, other.csw_u1)
    ev, rs, _ = lat.lowmodes_at_mass(-0.2, qs.eig_default_opts(k=16, nwant=8, tol=1e-9, warm_start=0, precision=2))
    s = np.sort(ev[:8])
    assert np.allclose(s[0::2], s[1::2], rtol=1e-9, atol=1e-13)
    assert np.all(rs[:8] <= 1e-9 * np.abs(ev[:8]) + 1e-12)
    lat.close()
