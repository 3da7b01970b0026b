"""O(a)-improved Wilson-Dirac operator on the C*-doubled lattice (Sec. 2 and Sec. 3).

D = D_w + m0 with (Sec. 2: O(a)-improved Wilson fermions, SU(3) and U(1) SW terms)

  (D psi)(x) = (4 + m0) psi(x) + A(x) psi(x)
               - 1/2 sum_mu [ V(x,mu) (1 - g_mu) psi(x + mu)
                              + V(x - mu, mu)^dag (1 + g_mu) psi(x - mu) ],

  V(x,mu) = U(x,mu) exp(i theta(x,mu))     (SU(3) link times the U(1) phase),
  A(x)    = (i/4) sum_{mu,nu} sigma_{mu nu} (x) [ c_sw F^SU(3)_{mu nu}(x) + c_sw,U(1) F^U(1)_{mu nu}(x) ],
  F_{mu nu}(x) = (Q_{mu nu}(x) - Q_{nu mu}(x)) / 8, Q the sum of the four plaquette
  leaves around x in the (mu, nu) plane (clover),

and Q = gamma_5 D (Sec. 3).  The operator is stored as one 12x12 block per
(site, neighbour): the diagonal block (4 + m0 + A) and 8 hopping blocks; the
component index is spin * 3 + colour.

Readings (the paper is silent): mass normalisation with diagonal 4 + m0, so that
Q'(m0) = gamma_5 as Sec. 3 requires; no trace subtraction in F; the U(1) SW term
uses the plaquettes of the phases the quark sees, i.e. of theta itself.

Pinned by tests/test_oracle_dirac.py: free-field plane-wave spectrum (closed
form with C* momenta), gamma_5-hermiticity, antisymmetry of C T D, the
degenerate partner C T gamma_5 v^*, gauge covariance, and a closed form of the
clover term next to a single plaquette carrying flux.
"""
import ctypes

import numpy as np
import scipy.sparse as sp

from .gamma import GAMMA, GAMMA5, CMAT, SIGMA, ID4
from .lattice import DoubledLattice


def _dag(U):
    return np.conj(np.swapaxes(U, -1, -2))


def plaquette_leaves(lat, U, mu, nu, sites=None):
    """Q_{mu nu}(x): sum of the four plaquette leaves at x in the (mu, nu) plane.

    U has shape (n_sites, 4, n, n) (n = 3 for SU(3), n = 1 for U(1) phases);
    ``sites`` selects the sites x (default: all).
    """
    x = np.arange(lat.n_sites) if sites is None else np.asarray(sites)
    fmu, bmu = lat.neighbour(mu, +1)[0], lat.neighbour(mu, -1)[0]
    fnu, bnu = lat.neighbour(nu, +1)[0], lat.neighbour(nu, -1)[0]
    xpm, xmm, xpn, xmn = fmu[x], bmu[x], fnu[x], bnu[x]
    xmm_pn = fnu[xmm]      # x - mu + nu
    xmm_mn = bnu[xmm]      # x - mu - nu
    xmn_pm = fmu[xmn]      # x - nu + mu
    Um, Un = U[:, mu], U[:, nu]
    leaf1 = Um[x] @ Un[xpm] @ _dag(Um[xpn]) @ _dag(Un[x])
    leaf2 = Un[x] @ _dag(Um[xmm_pn]) @ _dag(Un[xmm]) @ Um[xmm]
    leaf3 = _dag(Um[xmm]) @ _dag(Un[xmm_mn]) @ Um[xmm_mn] @ Un[xmn]
    leaf4 = _dag(Un[xmn]) @ Um[xmn] @ Un[xmn_pm] @ _dag(Um[x])
    return leaf1 + leaf2 + leaf3 + leaf4


def field_strength(lat, U, mu, nu, sites=None):
    """Clover field strength F_{mu nu} = (Q_{mu nu} - Q_{nu mu}) / 8."""
    return (plaquette_leaves(lat, U, mu, nu, sites) - plaquette_leaves(lat, U, nu, mu, sites)) / 8.0


def clover_term(lat, U3, theta, csw_su3, csw_u1, sites=None):
    """A(x) = (i/4) sum_{mu,nu} sigma_{mu nu} (c_sw F^SU3 + c_sw,U1 F^U1), shape (n, 12, 12)."""
    n = lat.n_sites if sites is None else len(sites)
    A = np.zeros((n, 12, 12), dtype=np.complex128)
    phase = np.exp(1j * theta)[:, :, None, None]
    I3 = np.eye(3)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            F = csw_su3 * field_strength(lat, U3, mu, nu, sites)
            if csw_u1 != 0.0:
                F = F + csw_u1 * field_strength(lat, phase, mu, nu, sites)[:, 0, 0][:, None, None] * I3
            A += 0.25j * np.einsum("ab,xij->xaibj", SIGMA[mu, nu], F).reshape(n, 12, 12)
    return A


class WilsonDirac:
    """The operator for one gauge configuration (synth_inputs.GaugeConfig).

    With ``lazy=True`` the site blocks are built only for the output sites asked
    for (used for sampled checks on large lattices)."""

    def __init__(self, cfg, lazy=False):
        self.cfg = cfg
        self.lat = DoubledLattice(cfg.T, cfg.L, cfg.cstar_mask, cfg.t_antiperiodic)
        lat = self.lat
        self.U3, self.theta = lat.doubled_links(cfg.su3, cfg.theta)
        self.V = self.U3 * np.exp(1j * self.theta)[:, :, None, None]
        self.n = 12 * lat.n_sites
        self.nbr = [(lat.neighbour(mu, +1), lat.neighbour(mu, -1)) for mu in range(4)]
        self.lazy = lazy
        if not lazy:
            self.A = clover_term(lat, self.U3, self.theta, cfg.csw_su3, cfg.csw_u1)
            self.cols, self.blocks = self.site_blocks(np.arange(lat.n_sites), self.A)

    def site_blocks(self, sites, A=None):
        """Neighbour columns and 12x12 blocks of D(m0 = 0) for output ``sites``:
        slot 0 diagonal (4 + A), slot 1 + 2 mu forward hop, slot 2 + 2 mu backward hop."""
        s = np.asarray(sites)
        ns = len(s)
        if A is None:
            A = clover_term(self.lat, self.U3, self.theta, self.cfg.csw_su3, self.cfg.csw_u1, s)
        cols = np.zeros((ns, 9), dtype=np.int64)
        blocks = np.zeros((ns, 9, 12, 12), dtype=np.complex128)
        cols[:, 0] = s
        blocks[:, 0] = 4.0 * np.eye(12) + A
        for mu in range(4):
            (fw, bcf), (bw, bcb) = self.nbr[mu]
            fw, bcf, bw, bcb = fw[s], bcf[s], bw[s], bcb[s]
            cols[:, 1 + 2 * mu] = fw
            cols[:, 2 + 2 * mu] = bw
            Pm = ID4 - GAMMA[mu]
            Pp = ID4 + GAMMA[mu]
            blocks[:, 1 + 2 * mu] = -0.5 * bcf[:, None, None] * np.einsum(
                "ab,xij->xaibj", Pm, self.V[s, mu]).reshape(ns, 12, 12)
            blocks[:, 2 + 2 * mu] = -0.5 * bcb[:, None, None] * np.einsum(
                "ab,xij->xaibj", Pp, _dag(self.V[bw, mu])).reshape(ns, 12, 12)
        return cols, blocks

    # ---- matrix-free -------------------------------------------------------
    def apply_D(self, psi, m0, sites=None):
        """D(m0) psi; psi has n_sites*12 components (any shape).  If ``sites`` is
        given, only those output sites are computed (shape (len(sites), 12))."""
        p = psi.reshape(-1, 12)
        s = np.arange(self.lat.n_sites) if sites is None else np.asarray(sites)
        if self.lazy:
            cols, blocks = self.site_blocks(s)
        else:
            cols, blocks = self.cols[s], self.blocks[s]
        out = m0 * p[s]
        for j in range(9):
            out = out + np.einsum("xij,xj->xi", blocks[:, j], p[cols[:, j]])
        return out if sites is not None else out.reshape(psi.shape)

    def apply_Q(self, psi, m0, sites=None):
        out = self.apply_D(psi, m0, sites)
        o = out.reshape(-1, 4, 3).copy()
        o[:, 2:] *= -1.0                     # gamma_5 = diag(1, 1, -1, -1)
        return o.reshape(out.shape)

    # ---- assembled -----------------------------------------------------------
    def sparse_D(self, m0):
        ns = self.lat.n_sites
        r = (np.arange(ns)[:, None, None, None] * 12 + np.arange(12)[None, None, :, None])
        c = (self.cols[:, :, None, None] * 12 + np.arange(12)[None, None, None, :])
        r, c = np.broadcast_arrays(r, c)
        M = sp.coo_matrix((self.blocks.ravel(), (r.ravel(), c.ravel())),
                          shape=(self.n, self.n)).tocsr()
        return M + m0 * sp.identity(self.n, dtype=np.complex128, format="csr")

    def gamma5_big(self):
        return sp.kron(sp.identity(self.lat.n_sites), sp.kron(sp.csr_matrix(GAMMA5), sp.identity(3))).tocsr()

    def sparse_Q(self, m0):
        return (self.gamma5_big() @ self.sparse_D(m0)).tocsr()

    def dense_D(self, m0):
        return self.sparse_D(m0).toarray()

    def dense_Q(self, m0):
        return self.sparse_Q(m0).toarray()

    def CT_matrix(self):
        """The matrix C T: spin C = i g0 g2 on every site, T = translation by L along x."""
        ns = self.lat.n_sites
        Tidx = self.lat.translation_T()
        P = sp.csr_matrix((np.ones(ns), (np.arange(ns), Tidx)), shape=(ns, ns))
        return sp.kron(P, sp.kron(sp.csr_matrix(CMAT), sp.identity(3))).tocsr()

    def dense_CTD(self, m0):
        return (self.CT_matrix() @ self.sparse_D(m0)).toarray()


class WilsonDiracC:
    """The same operator applied by plain C loops (oracle/dirac_c.c, OpenMP), for
    lattices where the assembled 12 x 12 hopping blocks of ``WilsonDirac`` do not fit
    in memory.  Holds the doubled links V, the SW blocks A(x) of every site (from
    ``clover_term``), the neighbour tables and the gamma matrices.

    Pinned by tests/test_oracle_dirac.py: equal to ``WilsonDirac.apply_D`` / ``apply_Q``
    on rough small lattices (an independent evaluation of the same formula: numpy
    block assembly there, explicit loops over spin and colour here), the free-field
    plane-wave closed form, and gamma_5-hermiticity of Q."""

    def __init__(self, cfg):
        self.cfg = cfg
        self.lat = DoubledLattice(cfg.T, cfg.L, cfg.cstar_mask, cfg.t_antiperiodic)
        lat = self.lat
        U3, theta = lat.doubled_links(cfg.su3, cfg.theta)
        self.V = np.ascontiguousarray(U3 * np.exp(1j * theta)[:, :, None, None])
        self.A = np.ascontiguousarray(clover_term(lat, U3, theta, cfg.csw_su3, cfg.csw_u1))
        ns = lat.n_sites
        self.fw = np.zeros((4, ns), dtype=np.int64)
        self.bw = np.zeros((4, ns), dtype=np.int64)
        self.bcf = np.zeros((4, ns))
        self.bcb = np.zeros((4, ns))
        for mu in range(4):
            (self.fw[mu], self.bcf[mu]), (self.bw[mu], self.bcb[mu]) = lat.neighbour(mu, +1), lat.neighbour(mu, -1)
        self.gam = np.ascontiguousarray(GAMMA)
        self.n = 12 * ns
        self._lib = _load_c()

    def _args(self):
        P = ctypes.c_void_p
        return [ctypes.c_long(self.lat.n_sites), P(self.V.ctypes.data), P(self.A.ctypes.data),
                P(self.fw.ctypes.data), P(self.bw.ctypes.data), P(self.bcf.ctypes.data),
                P(self.bcb.ctypes.data), P(self.gam.ctypes.data)]

    def apply(self, psi, m0, gamma5):
        x = np.ascontiguousarray(psi, dtype=np.complex128).reshape(-1)
        out = np.empty_like(x)
        self._lib.wd_apply(*self._args(), ctypes.c_double(m0), ctypes.c_int(int(gamma5)),
                           ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(out.ctypes.data))
        return out.reshape(np.shape(psi))

    def apply_D(self, psi, m0):
        return self.apply(psi, m0, 0)

    def apply_Q(self, psi, m0):
        return self.apply(psi, m0, 1)

    def residuals(self, vecs, theta, m0):
        """||Q(m0) v_i - theta_i v_i|| for the rows v_i of vecs [k][n]."""
        v = np.ascontiguousarray(vecs, dtype=np.complex128)
        k = v.shape[0]
        th = np.ascontiguousarray(theta, dtype=np.float64)
        work = np.empty(self.n, dtype=np.complex128)
        res = np.zeros(k)
        self._lib.wd_residuals(*self._args(), ctypes.c_double(m0), ctypes.c_int(k), ctypes.c_void_p(v.ctypes.data),
                               ctypes.c_void_p(th.ctypes.data), ctypes.c_void_p(work.ctypes.data),
                               ctypes.c_void_p(res.ctypes.data))
        return res


_clib = None


def build_c(force=False):
    """Compile oracle/dirac_c.c into oracle/_build/libwdoracle.so (gcc, OpenMP)."""
    import os
    import subprocess
    here = os.path.dirname(os.path.abspath(__file__))
    out_dir = os.path.join(here, "_build")
    so = os.path.join(out_dir, "libwdoracle.so")
    src = os.path.join(here, "dirac_c.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        os.makedirs(out_dir, exist_ok=True)
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", src, "-o", so, "-lm"])
    return so


def _load_c():
    global _clib
    if _clib is None:
        _clib = ctypes.CDLL(build_c())
        _clib.wd_apply.restype = None
        _clib.wd_residuals.restype = None
    return _clib


def gamma5_vec(psi):
    o = psi.reshape(-1, 4, 3).copy()
    o[:, 2:] *= -1.0
    return o.reshape(psi.shape)
