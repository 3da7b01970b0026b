"""Even-odd structure of D and the exact reweighting factor W_eo (Sec. 4).

Sites of the doubled lattice have parity (t + z + y + x) mod 2 (x in [0, 2L); L is even,
so the C* shift of x by L keeps the parity).  The hopping terms of D connect sites of
opposite parity only, so D^oo, the operator restricted to the odd sites, is the
site-diagonal part 4 + m0 + A(x) there, and

  log|det D^oo_m0| = sum over odd sites x of log|det(4 + m0 + A(x))|   (12 x 12 blocks),
  W_eo(m -> m') = |det[D^oo_m' (D^oo_m)^-1]|^(1/2) = exp((log|det D^oo_m'| - log|det D^oo_m|) / 2).

``log_det_oo`` evaluates the definition block by block (numpy slogdet of each 12 x 12
block); ``dhat_dense`` forms the preconditioned operator D_hat = D^ee - D^eo (D^oo)^-1 D^oe
from the dense D, and ``schur_det`` the identity det D = det D^oo det D_hat.

Pins (tests/test_oracle_evenodd.py): the odd-odd part of the dense D has no entries
between different sites; the dense slogdet of that part equals ``log_det_oo``; the
Schur identity det D = det D^oo det D_hat holds on a rough field; the free field gives
the closed form log|det D^oo| = 12 N_odd log|4 + m0|; on the free field D_hat equals
(4 + m0) - H_eo H_oe / (4 + m0) with H the hopping part of the dense D; the block-elimination
identity D y = (b_e, 0) => D_hat y_e = b_e; gamma_5 D_hat is Hermitian.
"""
import numpy as np

from .dirac import clover_term


def parity(lat):
    """0 (even) or 1 (odd) for every doubled site."""
    return (lat.t + lat.z + lat.y + lat.x) % 2


def log_det_oo(op, m0):
    """sum over odd doubled sites of log|det(4 + m0 + A(x))| for a WilsonDirac op."""
    lat = op.lat
    odd = np.nonzero(parity(lat) == 1)[0]
    A = clover_term(lat, op.U3, op.theta, op.cfg.csw_su3, op.cfg.csw_u1, odd)
    blocks = A + (4.0 + m0) * np.eye(12)[None]
    _, logabs = np.linalg.slogdet(blocks)
    return float(np.sum(logabs))


def w_eo(op, m, mp):
    """W_eo(m -> m') of Sec. 4 by its definition."""
    return float(np.exp(0.5 * (log_det_oo(op, mp) - log_det_oo(op, m))))


def dhat_dense(op, m0, gamma5=False):
    """(D_hat, e): the Schur complement D^ee - D^eo (D^oo)^-1 D^oe of the dense D on the
    even sites (gamma_5 D_hat if asked), and the indices e of the even-site components
    in the flat canonical vector, in the order D_hat's rows use."""
    D = op.dense_D(m0)
    p = np.repeat(parity(op.lat), 12)
    e, o = np.nonzero(p == 0)[0], np.nonzero(p == 1)[0]
    Dhat = D[np.ix_(e, e)] - D[np.ix_(e, o)] @ np.linalg.solve(D[np.ix_(o, o)], D[np.ix_(o, e)])
    if gamma5:
        g5 = np.where(np.arange(D.shape[0]) % 12 >= 6, -1.0, 1.0)[e]   # chiral basis: spins 2, 3
        Dhat = g5[:, None] * Dhat
    return Dhat, e


def schur_det(op, m0):
    """(log|det D^oo|, log|det D_hat|, log|det D|) from the dense D."""
    D = op.dense_D(m0)
    o = np.nonzero(np.repeat(parity(op.lat), 12) == 1)[0]
    Dhat, _ = dhat_dense(op, m0)
    return (np.linalg.slogdet(D[np.ix_(o, o)])[1], np.linalg.slogdet(Dhat)[1], np.linalg.slogdet(D)[1])
