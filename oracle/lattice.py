"""Orientifold-doubled lattice realising C* boundary conditions (Sec. 3, eq. defining T).

The C* condition psi(x + L k) = psi^C(x) for the spatial directions k makes the
Dirac operator act on the quark/antiquark doublet (a 24V x 24V matrix, Sec. 3).
Reading used here: stack the doublet along x, i.e. a lattice T x L x L x 2L whose
sites x1 in [0, L) carry psi and x1 in [L, 2L) carry psi^C.  Then

* the x direction is periodic with period 2L,
* crossing the y (or z) boundary, if C* holds in that direction, also moves
  x1 -> x1 + L (mod 2L)  (psi(x + L y) = psi^C(x)),
* time is periodic (Sec. 2), or antiperiodic for fermions if requested,
* links on the mirror half are the charge conjugates of the physical ones:
  U(x + L e1, mu) = U(x, mu)^*  (SU(3)), theta -> -theta (U(1)),
* T is the translation by L along x1: (T Psi)(x) = Psi(x + L e1).

Site index: ((t * L + z) * L + y) * 2L + x1.  Direction 0 = t, 1 = x, 2 = y, 3 = z.
Pinned through the operator tests (free-field momenta, C* antisymmetry of CTD,
gauge covariance) in tests/test_oracle_dirac.py.
"""
import numpy as np


class DoubledLattice:
    def __init__(self, T, L, cstar_mask=0b111, t_antiperiodic=False):
        if not (cstar_mask & 1):
            raise ValueError("the doubling runs along x: C* must hold in x (bit 0)")
        self.T, self.L = T, L
        self.cstar_mask = cstar_mask
        self.t_antiperiodic = t_antiperiodic
        self.shape = (T, L, L, 2 * L)
        self.n_sites = T * L * L * 2 * L
        t, z, y, x = np.meshgrid(np.arange(T), np.arange(L), np.arange(L),
                                 np.arange(2 * L), indexing="ij")
        self.t, self.z, self.y, self.x = (a.ravel() for a in (t, z, y, x))

    def index(self, t, z, y, x):
        L = self.L
        return ((t * L + z) * L + y) * (2 * L) + x

    def neighbour(self, mu, step):
        """Index of x + step*mu_hat (step = +1 or -1) and the fermion boundary factor."""
        T, L = self.T, self.L
        t, z, y, x = self.t.copy(), self.z.copy(), self.y.copy(), self.x.copy()
        bc = np.ones(self.n_sites)
        if mu == 0:
            t = t + step
            wrap = (t < 0) | (t >= T)
            t %= T
            if self.t_antiperiodic:
                bc[wrap] = -1.0
        elif mu == 1:
            x = (x + step) % (2 * L)
        else:
            c = y if mu == 2 else z
            c = c + step
            wrap = (c < 0) | (c >= L)
            c %= L
            if self.cstar_mask & (1 << (mu - 1)):
                x = np.where(wrap, (x + L) % (2 * L), x)
            if mu == 2:
                y = c
            else:
                z = c
        return self.index(t, z, y, x), bc

    def translation_T(self):
        """Index map of T: (T Psi)(x) = Psi(x + L e1)."""
        return self.index(self.t, self.z, self.y, (self.x + self.L) % (2 * self.L))

    def physical_of(self):
        """(physical flat index, mirror flag) of every doubled site."""
        L = self.L
        xp = self.x % L
        phys = ((self.t * L + self.z) * L + self.y) * L + xp
        return phys, self.x >= L

    def doubled_links(self, su3, theta=None):
        """SU(3) links and U(1) angles on the doubled lattice (mirror = conjugate)."""
        phys, mirror = self.physical_of()
        U = su3.reshape(-1, 4, 3, 3)[phys].copy()
        U[mirror] = U[mirror].conj()
        th = np.zeros((self.n_sites, 4))
        if theta is not None:
            th = theta.reshape(-1, 4)[phys].copy()
            th[mirror] = -th[mirror]
        return U, th
