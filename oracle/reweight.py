"""Mass reweighting of Sec. 4: the rational approximation R and the factor W_mass.
Test infrastructure only (tests/, the entry point's smoke check and the benchmark's CPU
baseline call it; the product path never does).

Rational approximation (eq. ratapprox): R(y) = A prod_i (y + nu_i^2) / (y + mu_i^2), the
(n, n) rational function of least uniform relative error |R(y) y^p - 1| on
y = x^2, x in [r_a, r_b] (p = 1/4: R(Q_hat^2) stands for (Q_hat^2)^(-1/4) in eq. detQ2).
``ratapprox`` finds it by the linearised rational Remez iteration: at 2n + 2 reference
points the levelled error E and the coefficients of P and Q (Chebyshev basis in y) solve
the generalised eigenproblem  w P - Q = E (-1)^k Q  (w = y^p); the eigenvalue of least |E|
whose Q keeps one sign on the interval is taken; the reference moves to the extrema of the
error; repeat until the error is levelled.  nu_i^2, mu_i^2 are minus the roots of P and Q.

W_mass (eq. Wmass, S_j, R_j), with D_hat the even-odd preconditioned operator (dense, from
``evenodd.dhat_dense``), delta D = D_hat(m') - D_hat(m) and, for j = 1 .. n,
  S_j = (D_hat(m) + i g5 nu_j)^-1 - (D_hat(m') + i g5 mu_j)^-1
        - (D_hat(m') + i g5 mu_j)^-1 delta D (D_hat(m) + i g5 nu_j)^-1,
  R_j = X^+ + X + X^+ X,  X = delta D S_j,
each written out as printed.  The Gaussian integral with weight exp(-(eta, eta)) gives
E[exp(-(eta, R_j eta))] = 1 / det(1 + R_j); the estimate of W_mass is
prod_j (1/N) sum_l exp(-(eta_jl, R_j eta_jl)), and its exact value prod_j 1/det(1 + R_j)
equals det[R(Q_hat_m^2) R^-1(Q_hat_m'^2)] (the reading of the printed product and of its
range is recorded with the design notes).

Pins (tests/test_oracle_reweight.py): n = 0 closed form of the best constant; the
equioscillation certificate (alternation theorem: 2n + 2 alternating extrema of equal
magnitude) for n = 1 .. 4; the exact identity prod_j 1/det(1 + R_j) =
det R(Q_hat_m^2) / det R(Q_hat_m'^2) from the spectrum of Q_hat^2 on a rough field; the
Gaussian integral E[exp(-(eta, R eta))] = 1/det(1 + R) by Monte Carlo on a small matrix.
"""
import numpy as np
from numpy.polynomial import chebyshev as cheb
from scipy.linalg import eig

from .evenodd import dhat_dense


def _alternating_extrema(e, m):
    """Indices of the extrema of e on each run of one sign, cut to m alternating ones."""
    runs = np.split(np.arange(len(e)), np.nonzero(np.diff(np.sign(e)))[0] + 1)
    ext = [r[np.argmax(np.abs(e[r]))] for r in runs]
    while len(ext) > m:
        if abs(e[ext[0]]) < abs(e[ext[-1]]):
            ext = ext[1:]
        else:
            ext = ext[:-1]
    return ext


def ratapprox(n, ra, rb, p=0.25, npts=200001, iters=80):
    """(A, nu, mu, delta): best (n, n) relative approximation of y^-p on [ra^2, rb^2]."""
    ya, yb = ra * ra, rb * rb
    la, lb = np.log(ya), np.log(yb)
    grid = np.linspace(la, lb, npts)
    yg = np.exp(grid)
    xmap = lambda y: (2 * y - (ya + yb)) / (yb - ya)
    Vg, wg = cheb.chebvander(xmap(yg), n), yg ** p
    if n == 0:
        A = 2.0 / (ya ** p + yb ** p)
        return A, np.zeros(0), np.zeros(0), float(np.max(np.abs(A * wg - 1)))
    m = 2 * n + 2
    S = 0.5 * (la + lb) - 0.5 * (lb - la) * np.cos(np.pi * np.arange(m) / (m - 1))
    sg = (-1.0) ** np.arange(m)
    c = None
    for _ in range(iters):
        y = np.exp(S)
        V, w = cheb.chebvander(xmap(y), n), y ** p
        ev, vec = eig(np.hstack([w[:, None] * V, -V]), np.hstack([np.zeros_like(V), sg[:, None] * V]))
        best = None
        for E, v in zip(ev, vec.T):
            if not np.isfinite(E) or abs(E.imag) > 1e-10 * max(1.0, abs(E)):
                continue
            v = v.real / np.max(np.abs(v.real))
            Qg = Vg @ v[n + 1:]
            if (np.all(Qg > 0) or np.all(Qg < 0)) and (best is None or abs(E.real) < abs(best[0])):
                best = (E.real, v)
        if best is None:
            raise RuntimeError("ratapprox: no admissible levelled solution")
        E, c = best
        e = wg * (Vg @ c[:n + 1]) / (Vg @ c[n + 1:]) - 1
        ext = _alternating_extrema(e, m)
        if len(ext) < m:
            raise RuntimeError("ratapprox: the error lost its alternation")
        S = grid[ext]
        if np.max(np.abs(e)) - abs(E) < 1e-8 * np.max(np.abs(e)):
            break
    P, Q = c[:n + 1], c[n + 1:]
    # back to the product form: roots in y of P and Q (Chebyshev variable x -> y)
    zy = (cheb.chebroots(P) * (yb - ya) + (ya + yb)) / 2
    py = (cheb.chebroots(Q) * (yb - ya) + (ya + yb)) / 2
    nu2, mu2 = np.sort(-zy.real), np.sort(-py.real)
    if np.any(np.abs(zy.imag) > 1e-8 * np.abs(zy)) or np.any(nu2 <= 0) or np.any(mu2 <= 0):
        raise RuntimeError("ratapprox: zeros or poles off the negative real axis")
    y0 = np.sqrt(ya * yb)
    A = float((cheb.chebval(xmap(y0), P) / cheb.chebval(xmap(y0), Q)) / np.prod((y0 + nu2) / (y0 + mu2)))
    nu, mu = np.sqrt(nu2), np.sqrt(mu2)
    delta = float(np.max(np.abs(rat_eval(A, nu, mu, yg) * wg - 1)))
    return A, nu, mu, delta


def rat_eval(A, nu, mu, y):
    """R(y) = A prod_i (y + nu_i^2) / (y + mu_i^2)."""
    y = np.asarray(y, dtype=float)
    r = np.full_like(y, A)
    for a, b in zip(nu, mu):
        r = r * (y + a * a) / (y + b * b)
    return r


def _g5_even(op):
    """gamma_5 on the even-site components, in the row order of dhat_dense."""
    n = op.lat.n_sites * 12
    _, e = dhat_dense(op, 0.0)
    return np.where(np.arange(n) % 12 >= 6, -1.0, 1.0)[e]


def r_matrices(op, m, mp, nu, mu):
    """[R_j] (dense, even sites) for j = 1 .. n, each S_j in its three printed terms."""
    Dm, _ = dhat_dense(op, m)
    Dmp, _ = dhat_dense(op, mp)
    G = np.diag(_g5_even(op)).astype(complex)
    dD = Dmp - Dm
    out = []
    for a, b in zip(nu, mu):
        inv_a = np.linalg.inv(Dm + 1j * a * G)
        inv_b = np.linalg.inv(Dmp + 1j * b * G)
        S = inv_a - inv_b - inv_b @ dD @ inv_a
        X = dD @ S
        out.append(X.conj().T + X + X.conj().T @ X)
    return out


def log_w_mass_exact(op, m, mp, nu, mu):
    """log prod_j 1/det(1 + R_j) (the exact W_mass of the estimator)."""
    tot = 0.0
    for R in r_matrices(op, m, mp, nu, mu):
        sign, ld = np.linalg.slogdet(np.eye(R.shape[0]) + R)
        tot -= ld
    return float(tot)


def log_w_mass_spectral(op, m, mp, A, nu, mu):
    """log det[R(Q_hat_m^2) R^-1(Q_hat_m'^2)] from the eigenvalues of Q_hat^2."""
    y0 = np.linalg.eigvalsh(_q2(op, m))
    y1 = np.linalg.eigvalsh(_q2(op, mp))
    return float(np.sum(np.log(rat_eval(A, nu, mu, y0))) - np.sum(np.log(rat_eval(A, nu, mu, y1))))


def _q2(op, m):
    Qh, _ = dhat_dense(op, m, gamma5=True)
    return Qh.conj().T @ Qh


def quad_forms(op, m, mp, nu, mu, eta):
    """q[j][l] = (eta_l, R_j eta_l) for sources eta [nsrc][even components]."""
    Rs = r_matrices(op, m, mp, nu, mu)
    return np.array([[np.real(np.vdot(x, R @ x)) for x in eta] for R in Rs])


def log_w_mass_estimate(q):
    """log of prod_j (1/N) sum_l exp(-q[j][l])."""
    q = np.asarray(q, dtype=float)
    return float(np.sum(np.log(np.mean(np.exp(-q), axis=1))))
