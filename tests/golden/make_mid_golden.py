"""Writes tests/golden/mid_4x4x4x6_seed7.json from the CPU oracle only.

Field: 4^3 x 6 lattice, C* in x, y, z (doubled to 8x4x4x6), periodic t, SU(3) links
exp(i 0.45 H), U(1) angles N(0, 0.3^2), c_sw = 1.9 (SU(3)) and 1.0 (U(1)), seed 7
(synth_inputs).  n = 12 * 2 * 4^3 * 6 = 9216, the largest size at which the dense
oracle routes finish in minutes on a few host cores.

The real eigenvalues mu of D(m0 = 0) give every zero crossing of the flow: Q(m0) is
singular exactly at m0 = -mu (Sec. 3: pf[CTD(m0)] = prod_n lambda_n is analytic in m0
and changes sign where a pair crosses).  The masses are chosen around the densest
cluster of crossings (the doubler region near m0 = -2): below it, inside it where
W_sgn = -1, and above it, plus m0 at kappa = 0.135.  For each mass the file stores the
32 eigenvalues of the dense Q closest to zero (with multiplicity), the negative count,
and W_sgn computed twice (negative count; dense Pfaffian ratio to m_big), which must
agree.

Run:  python tests/golden/make_mid_golden.py      (about 15 minutes on 8 threads)
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from synth_inputs import kappa_to_m0, make_config  # noqa: E402
from oracle.dirac import WilsonDirac  # noqa: E402
from oracle.sign import m_big, sign_by_pfaffian  # noqa: E402

FIELD = dict(T=6, L=4, eps=0.45, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0, seed=7)
NLOW = 32


def crossing_masses(op):
    """m0 = -mu for every real eigenvalue mu of D(0), one per degenerate pair."""
    mu = np.linalg.eigvals(op.dense_D(0.0))
    real = np.sort(mu[np.abs(mu.imag) < 1e-8].real)
    assert len(real) % 2 == 0
    assert np.allclose(real[0::2], real[1::2], atol=1e-7)
    return np.sort(-real[0::2])


def pick_masses(cross):
    """Below the densest window of crossings, inside it (odd number of crossings below
    the mass and above it), above it; at least 1e-3 away from every crossing."""
    best, lo_i = -1, 0
    for i in range(len(cross)):
        n = int(np.sum((cross >= cross[i]) & (cross <= cross[i] + 0.15)))
        if n > best:
            best, lo_i = n, i
    lo, hi = cross[lo_i], cross[lo_i] + 0.15
    inside = cross[(cross >= lo) & (cross <= hi)]
    below = lo - 0.02
    # a mass in the cluster with an odd number of crossings above it inside the window
    mid = None
    for j in range(len(inside) - 1):
        cand = 0.5 * (inside[j] + inside[j + 1])
        if inside[j + 1] - inside[j] > 2e-3 and (len(inside) - 1 - j) % 2 == 1:
            mid = cand
            break
    above = inside[-1] + 0.03
    out = [kappa_to_m0(0.135), below, above]
    if mid is not None:
        out.insert(2, mid)
    for m in out:
        assert np.min(np.abs(cross - m)) > 1e-3, m
    return out, inside


def main():
    cfg = make_config(**FIELD)
    op = WilsonDirac(cfg)
    cross = crossing_masses(op)
    masses, cluster = pick_masses(cross)
    print("crossings in the cluster:", cluster, flush=True)
    out = {"field": FIELD, "n": op.n, "m_big": m_big(cfg), "crossing_masses": cross.tolist(),
           "cluster": cluster.tolist(), "points": []}
    for m in masses:
        w = np.linalg.eigvalsh(op.dense_Q(m))
        nneg = int(np.sum(w < 0))
        s_eig = 1 if (nneg // 2) % 2 == 0 else -1
        s_pf, ratio = sign_by_pfaffian(op, m, use_c=True)
        assert s_pf == s_eig, (m, s_pf, s_eig)
        # the sign from the crossings: each crossing above m flips it once (Sec. 3)
        s_cross = 1 if int(np.sum(cross > m)) % 2 == 0 else -1
        assert s_cross == s_eig, (m, s_cross, s_eig)
        low = w[np.argsort(np.abs(w), kind="stable")][:NLOW]
        out["points"].append({"m0": m, "sign": s_pf, "n_negative": nneg,
                              "pf_ratio_re": ratio.real, "pf_ratio_im": ratio.imag,
                              "lowest_abs_sorted_eigs_Q": low.tolist()})
        print(m, s_pf, low[:4], flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mid_4x4x4x6_seed7.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
