"""Pins of oracle/dirac.py and oracle/lattice.py (Sec. 2 operator, Sec. 3 C* structure)."""
import itertools

import numpy as np
import pytest

from synth_inputs import GaugeConfig, make_config, unit_su3_field
from oracle.dirac import WilsonDirac, gamma5_vec
from oracle.gamma import CMAT


def free_cfg(T, L, t_anti=False, mask=0b111):
    return GaugeConfig(T, L, unit_su3_field(T, L), None, 1.7, 0.9, t_anti, mask)


def cstar_momenta(T, L, t_anti=False, mask=0b111):
    """Momenta allowed on the doubled lattice: x periodic over 2L, y/z shifted
    by L in x on wrap (C*) or periodic, t periodic/antiperiodic."""
    out = []
    for n1 in range(2 * L):
        p1 = np.pi * n1 / L
        for n2 in range(L):
            p2 = (p1 if mask & 2 else 0.0) + 2 * np.pi * n2 / L
            for n3 in range(L):
                p3 = (p1 if mask & 4 else 0.0) + 2 * np.pi * n3 / L
                for n0 in range(T):
                    p0 = (2 * n0 + (1 if t_anti else 0)) * np.pi / T
                    out.append((p0, p1, p2, p3))
    return np.array(out)


def free_Q_spectrum(T, L, m0, t_anti=False, mask=0b111):
    ev = []
    for p in cstar_momenta(T, L, t_anti, mask):
        M = m0 + np.sum(1 - np.cos(p))
        e = np.sqrt(M * M + np.sum(np.sin(p) ** 2))
        ev += [e] * 6 + [-e] * 6
    return np.sort(ev)


@pytest.mark.parametrize("T,L,t_anti,mask", [(2, 2, False, 0b111), (4, 2, True, 0b111),
                                             (2, 4, False, 0b011), (4, 2, False, 0b001)])
def test_free_field_plane_wave(T, L, t_anti, mask):
    """D e^{ipx} u = [m0 + sum(1 - cos p) + i sum gamma_mu sin p_mu] u e^{ipx}."""
    from oracle.gamma import GAMMA
    op = WilsonDirac(free_cfg(T, L, t_anti, mask))
    lat = op.lat
    rng = np.random.default_rng(1)
    m0 = -0.37
    ps = cstar_momenta(T, L, t_anti, mask)
    for p in ps[rng.choice(len(ps), 6, replace=False)]:
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (p[0] * lat.t + p[1] * lat.x + p[2] * lat.y + p[3] * lat.z))
        psi = phase[:, None, None] * u[None]
        Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(GAMMA[m] * np.sin(p[m]) for m in range(4))
        ref = phase[:, None, None] * (Dp @ u)[None]
        out = op.apply_D(psi.reshape(-1), m0).reshape(psi.shape)
        assert np.allclose(out, ref, atol=1e-12)


@pytest.mark.parametrize("T,L,t_anti", [(2, 2, False), (4, 2, True)])
def test_free_field_spectrum(T, L, t_anti):
    op = WilsonDirac(free_cfg(T, L, t_anti))
    m0 = 0.21
    w = np.linalg.eigvalsh(op.dense_Q(m0))
    assert np.allclose(w, free_Q_spectrum(T, L, m0, t_anti), atol=1e-12)


def rough_cfg(T=4, L=2, seed=5, mask=0b111):
    return make_config(T=T, L=L, eps=0.9, theta_sigma=0.4, csw_su3=1.3, csw_u1=0.8, seed=seed,
                       cstar_mask=mask)


@pytest.mark.parametrize("mask", [0b111, 0b011, 0b001])
def test_gamma5_hermiticity_and_antisymmetry(mask):
    op = WilsonDirac(rough_cfg(mask=mask))
    m0 = -0.6
    Q = op.dense_Q(m0)
    assert np.abs(Q - Q.conj().T).max() < 1e-14
    M = op.dense_CTD(m0)
    assert np.abs(M + M.T).max() < 1e-13 * np.abs(M).max()


def test_degenerate_partner():
    """If Q v = lambda v then C T gamma_5 v^* is an orthogonal eigenvector (Sec. 3)."""
    op = WilsonDirac(rough_cfg(seed=2))
    m0 = -0.4
    w, V = np.linalg.eigh(op.dense_Q(m0))
    CT = op.CT_matrix()
    for i in [0, 17, 300, len(w) - 1]:
        v = V[:, i]
        u = CT @ gamma5_vec(v.conj())
        assert np.allclose(op.dense_Q(m0) @ u, w[i] * u, atol=1e-11)
        assert abs(np.vdot(v, u)) < 1e-11
    assert np.abs(w[0::2] - w[1::2]).max() < 1e-11


def _rand_su3(rng, shape):
    X = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    Qm, R = np.linalg.qr(X)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Qm = Qm * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(Qm)
    return Qm / det[..., None, None] ** (1.0 / 3.0)


def test_gauge_covariance():
    """D[U^g](g psi) = g D[U] psi, g on the mirror half = g^* (C* compatible)."""
    T, L = 4, 2
    cfg = rough_cfg(T, L, seed=11)
    op = WilsonDirac(cfg)
    lat = op.lat
    rng = np.random.default_rng(4)
    gp = _rand_su3(rng, (T, L, L, L)).reshape(-1, 3, 3)
    ap = rng.standard_normal(T * L * L * L)
    phys, mirror = lat.physical_of()
    gd = gp[phys].copy(); gd[mirror] = gd[mirror].conj()
    ad = ap[phys].copy(); ad[mirror] = -ad[mirror]
    # transformed doubled links, then read back the physical half
    Ug = np.empty_like(op.U3); thg = np.empty_like(op.theta)
    for mu in range(4):
        fw, _ = lat.neighbour(mu, +1)
        Ug[:, mu] = gd @ op.U3[:, mu] @ gd[fw].conj().transpose(0, 2, 1)
        thg[:, mu] = op.theta[:, mu] + ad - ad[fw]
    sel = ~mirror
    order = np.argsort(phys[sel])
    su3_new = Ug[sel][order].reshape(T, L, L, L, 4, 3, 3)
    th_new = thg[sel][order].reshape(T, L, L, L, 4)
    # the transformed doubled field is again C*-consistent
    assert np.allclose(Ug[mirror], Ug[~mirror][np.argsort(phys[~mirror])][phys[mirror]].conj())
    from synth_inputs import GaugeConfig
    op2 = WilsonDirac(GaugeConfig(T, L, su3_new, th_new, cfg.csw_su3, cfg.csw_u1))
    psi = rng.standard_normal((lat.n_sites, 4, 3)) + 1j * rng.standard_normal((lat.n_sites, 4, 3))
    m0 = -0.3
    gpsi = np.einsum("xab,xsb->xsa", gd, psi) * np.exp(1j * ad)[:, None, None]
    lhs = op2.apply_D(gpsi.reshape(-1), m0).reshape(psi.shape)
    Dpsi = op.apply_D(psi.reshape(-1), m0).reshape(psi.shape)
    rhs = np.einsum("xab,xsb->xsa", gd, Dpsi) * np.exp(1j * ad)[:, None, None]
    assert np.allclose(lhs, rhs, atol=1e-12)


@pytest.mark.parametrize("group", ["u1", "su3"])
def test_clover_single_flux_plaquette(group):
    """One link (x0, x-direction) carries a phase phi; the plaquette P_xy(x0) then has
    flux phi and P_xy(x0 - y) flux -phi (and likewise in the xz and tx planes).  Site
    x0 + y touches only the first of them, so F_xy = (i/4) sin(phi) there and the SW
    term is c (i/4) 2 sigma_xy F_xy = (c/8) sin(phi) diag(1,-1,1,-1) (x) colour,
    since sigma_xy = -diag(s3, s3).  At x0 the two xy leaves cancel: A(x0) = 0.  On
    the mirror site the phase is conjugated, so the sign flips."""
    T, L = 4, 4
    phi = 0.7
    c = 1.3
    su3 = unit_su3_field(T, L)
    theta = np.zeros((T, L, L, L, 4))
    x0 = (1, 2, 1, 1)   # (t, z, y, x)
    if group == "u1":
        theta[x0 + (1,)] = phi
        cfg = GaugeConfig(T, L, su3, theta, 0.0, c)
        colour = np.eye(3) * np.sin(phi)
    else:
        su3[x0 + (1,)] = np.diag([np.exp(1j * phi), np.exp(-1j * phi), 1.0])
        cfg = GaugeConfig(T, L, su3, None, c, 0.0)
        colour = np.diag([np.sin(phi), -np.sin(phi), 0.0])
    op = WilsonDirac(cfg)
    lat = op.lat
    t, z, y, x = x0
    site = lat.index(t, z, y + 1, x)
    ref = (c / 8.0) * np.kron(np.diag([1, -1, 1, -1]), colour)
    assert np.allclose(op.A[site], ref, atol=1e-14)
    assert np.allclose(op.A[lat.index(t, z, y, x)], 0, atol=1e-14)
    assert np.allclose(op.A[lat.index(t, z, y + 1, x + L)], -ref, atol=1e-14)
    # far away the clover term vanishes
    assert np.allclose(op.A[lat.index((t + 2) % T, z, y, x)], 0, atol=1e-14)


def test_lazy_site_blocks_match_full_assembly():
    cfg = rough_cfg(T=4, L=2, seed=8)
    full, lazy = WilsonDirac(cfg), WilsonDirac(cfg, lazy=True)
    rng = np.random.default_rng(0)
    psi = rng.standard_normal(full.n) + 1j * rng.standard_normal(full.n)
    sites = np.array([0, 5, 17, 63])
    a = full.apply_Q(psi, -0.2).reshape(-1, 12)[sites]
    b = lazy.apply_Q(psi, -0.2, sites)
    assert np.allclose(a, b, atol=1e-14)
    assert np.allclose(full.sparse_Q(-0.2) @ psi, full.apply_Q(psi, -0.2), atol=1e-13)


def test_pfaffian_squared_is_det_D():
    """pf[C T D]^2 = det D (Sec. 3): with pf^2 = det for the antisymmetric C T D this
    needs det(C T) = 1 for the doubled-lattice C and T."""
    from oracle.pfaffian import pfaffian
    op = WilsonDirac(rough_cfg(T=2, L=2, seed=4))
    m0 = -0.35
    la, ph = pfaffian(op.dense_CTD(m0))
    sd, ld = np.linalg.slogdet(op.dense_D(m0))
    assert np.isclose(2 * la, ld, atol=1e-9)
    assert np.isclose(ph * ph, sd, atol=1e-9)
    sct, lct = np.linalg.slogdet(op.CT_matrix().toarray())
    assert np.isclose(lct, 0.0, atol=1e-12) and np.isclose(sct, 1.0)


@pytest.mark.parametrize("mask,t_anti", [(0b111, False), (0b011, True)])
def test_plain_loop_c_operator_matches_assembled_one(mask, t_anti):
    """oracle/dirac_c.c (explicit loops over spin and colour) against the numpy
    assembly of the same formula, D and Q, on a rough field."""
    from oracle.dirac import WilsonDiracC
    cfg = make_config(T=3, L=2, eps=0.8, theta_sigma=0.4, csw_su3=1.3, csw_u1=0.7, seed=9,
                      t_antiperiodic=t_anti, cstar_mask=mask)
    a, b = WilsonDirac(cfg), WilsonDiracC(cfg)
    rng = np.random.default_rng(3)
    psi = rng.standard_normal(a.n) + 1j * rng.standard_normal(a.n)
    for m0 in (-0.41, 0.3):
        assert np.allclose(b.apply_D(psi, m0), a.apply_D(psi, m0), atol=1e-13, rtol=0)
        assert np.allclose(b.apply_Q(psi, m0), a.apply_Q(psi, m0), atol=1e-13, rtol=0)


def test_plain_loop_c_operator_free_field_and_hermiticity():
    from oracle.dirac import WilsonDiracC
    from oracle.gamma import GAMMA
    T, L = 4, 4
    op = WilsonDiracC(free_cfg(T, L))
    lat = op.lat
    m0 = -0.23
    for p in cstar_momenta(T, L)[[5, 77, 300]]:
        u = np.arange(12).reshape(4, 3) + 1j
        phase = np.exp(1j * (p[0] * lat.t + p[1] * lat.x + p[2] * lat.y + p[3] * lat.z))
        psi = phase[:, None, None] * u[None]
        Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(GAMMA[m] * np.sin(p[m]) for m in range(4))
        assert np.allclose(op.apply_D(psi.reshape(-1), m0), (phase[:, None, None] * (Dp @ u)[None]).reshape(-1),
                           atol=1e-12)
    rough = WilsonDiracC(rough_cfg(T=4, L=2))
    rng = np.random.default_rng(8)
    f, g = (rng.standard_normal(rough.n) + 1j * rng.standard_normal(rough.n) for _ in range(2))
    assert np.isclose(np.vdot(f, rough.apply_Q(g, 0.2)), np.vdot(rough.apply_Q(f, 0.2), g), rtol=1e-12)
