"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the method: it only draws random gauge
fields and spinors with fixed seeds, so that the CPU oracle and the GPU
library can be handed bit-identical inputs.  Nothing here knows about the
Dirac operator, the C* doubling or the Pfaffian.

Recipe (stands in for the 64x32^3 QCD / QCD+QED ensembles of Sec. 2, which
are not available):

* SU(3) links  U = exp(i * eps * H),  H = sum_a h_a lambda_a / 2,  h_a ~ N(0,1),
  lambda_a the eight Gell-Mann matrices.  The exponential is taken through the
  eigen-decomposition of the Hermitian H, so U is unitary with det U = 1 to
  rounding.
* U(1) angles  theta ~ N(0, sigma^2) per link (the phase the quark sees).
* Draw order: numpy ``default_rng(seed)`` (PCG64), first all h_a in array order
  [t][z][y][x][mu][a], then all theta in order [t][z][y][x][mu].

Array conventions (physical lattice, T x L^3):
  su3[t, z, y, x, mu, a, b]   complex128, mu = 0 (t), 1 (x), 2 (y), 3 (z)
  theta[t, z, y, x, mu]       float64
Spinors live on the doubled lattice T x L x L x 2L:
  psi[t, z, y, xd, spin, colour] complex128, xd in [0, 2L).
"""
import numpy as np

__all__ = ["gell_mann", "random_su3_field", "random_u1_field", "unit_su3_field",
           "random_spinor", "GaugeConfig", "make_config"]


def gell_mann():
    """The eight Gell-Mann matrices (standard normalisation tr(l_a l_b) = 2 d_ab)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j; l[1][1, 0] = 1j
    l[2][0, 0] = 1; l[2][1, 1] = -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j; l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j; l[6][2, 1] = 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return l


def random_su3_field(rng, T, L, eps):
    """exp(i eps H) per link, H Gaussian traceless Hermitian (see module doc).  All
    h_a are drawn first; the exponentials are then formed one time slice at a time
    (the same numbers as all at once, with bounded memory)."""
    h = rng.standard_normal((T, L, L, L, 4, 8))
    G = gell_mann()
    U = np.empty((T, L, L, L, 4, 3, 3), dtype=np.complex128)
    for t in range(T):
        H = np.einsum("...a,aij->...ij", h[t], G) / 2.0
        w, v = np.linalg.eigh(H)
        U[t] = np.einsum("...ik,...k,...jk->...ij", v, np.exp(1j * eps * w), v.conj())
    return U


def random_u1_field(rng, T, L, sigma):
    return rng.standard_normal((T, L, L, L, 4)) * sigma


def unit_su3_field(T, L):
    U = np.zeros((T, L, L, L, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def random_spinor(seed, T, L, nrhs=None):
    """Complex Gaussian spinor(s) on the doubled lattice, shape [.., T, L, L, 2L, 4, 3]."""
    rng = np.random.default_rng(seed)
    shape = (T, L, L, 2 * L, 4, 3) if nrhs is None else (nrhs, T, L, L, 2 * L, 4, 3)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


class GaugeConfig:
    """A synthetic configuration: physical links, U(1) angles and the c_sw's."""

    def __init__(self, T, L, su3, theta, csw_su3, csw_u1, t_antiperiodic=False, cstar_mask=0b111):
        self.T, self.L = T, L
        self.su3 = np.ascontiguousarray(su3, dtype=np.complex128)
        self.theta = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
        self.csw_su3, self.csw_u1 = float(csw_su3), float(csw_u1)
        self.t_antiperiodic = bool(t_antiperiodic)
        self.cstar_mask = int(cstar_mask)

    @property
    def n_sites(self):
        """Sites of the doubled lattice."""
        return 2 * self.L ** 3 * self.T


def make_config(T, L, eps, theta_sigma=0.0, csw_su3=1.5, csw_u1=0.0, seed=0,
                t_antiperiodic=False, cstar_mask=0b111, cache_dir=None):
    """A seeded synthetic configuration.  cache_dir (or the environment variable
    QS_FIELD_CACHE): keep the drawn links and angles there as .npy files and reuse them
    (large lattices take a minute to draw)."""
    import os
    cache_dir = cache_dir or os.environ.get("QS_FIELD_CACHE")
    path = None
    if cache_dir:
        tag = f"T{T}_L{L}_eps{eps!r}_th{theta_sigma!r}_seed{seed}"
        path = os.path.join(cache_dir, tag)
        if os.path.exists(path + "_su3.npy"):
            su3 = np.load(path + "_su3.npy")
            theta = np.load(path + "_theta.npy") if os.path.exists(path + "_theta.npy") else None
            return GaugeConfig(T, L, su3, theta, csw_su3, csw_u1, t_antiperiodic, cstar_mask)
    rng = np.random.default_rng(seed)
    su3 = random_su3_field(rng, T, L, eps)
    theta = random_u1_field(rng, T, L, theta_sigma) if theta_sigma > 0 else None
    if path:
        os.makedirs(cache_dir, exist_ok=True)
        np.save(path + "_su3.npy", su3)
        if theta is not None:
            np.save(path + "_theta.npy", theta)
    return GaugeConfig(T, L, su3, theta, csw_su3, csw_u1, t_antiperiodic, cstar_mask)


# Named workloads (sizes and link distributions of the synthetic ensembles).
WORKLOADS = {
    # 4^4, C* in x,y,z, SU(3) eps=0.3, U(1) off, c_sw=1.5
    "tiny_4x4x4x4": dict(T=4, L=4, eps=0.3, theta_sigma=0.0, csw_su3=1.5, csw_u1=0.0),
    # 16^3 x 32, SU(3) eps=0.2, theta ~ N(0, 0.3^2), c_sw = 1.9 / 1.0
    "qcdqed_16x16x16x32": dict(T=32, L=16, eps=0.2, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0),
    # 24^3 x 48, as above with eps=0.2
    "qcdqed_24x24x24x48": dict(T=48, L=24, eps=0.2, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0),
    # 32^3 x 64, SU(3) eps=0.15
    "qcdqed_32x32x32x64": dict(T=64, L=32, eps=0.15, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0),
}


def kappa_to_m0(kappa):
    """Bare mass from the hopping parameter, kappa = 1 / (2 (m0 + 4))."""
    return 1.0 / (2.0 * kappa) - 4.0


def mlp_init(seed, n_in, n_hidden, n_out):
    """Initial weights of the step-proposal network (random numbers only):
    [W1 (n_hidden x n_in), b1, W2 (n_hidden x n_hidden), b2, W3 (n_out x n_hidden), b3],
    W ~ N(0, 1/fan_in), b = 0, float32."""
    rng = np.random.default_rng(seed)
    shapes = [(n_hidden, n_in), (n_hidden,), (n_hidden, n_hidden), (n_hidden,), (n_out, n_hidden), (n_out,)]
    out = []
    for sh in shapes:
        if len(sh) == 2:
            out.append((rng.standard_normal(sh) / np.sqrt(sh[1])).astype(np.float32))
        else:
            out.append(np.zeros(sh, dtype=np.float32))
    return out
