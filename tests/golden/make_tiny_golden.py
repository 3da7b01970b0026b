"""Writes tests/golden/tiny_4x4x4x4_seed0.json from the CPU oracle only.

Workload: 4^4 lattice, C* in x, y, z (doubled to 8x4x4x4), periodic t, SU(3)
links exp(i 0.3 H), U(1) off, c_sw = 1.5, seed 0 (synth_inputs).  n = 6144.

Masses: m0 = 1/(2 kappa) - 4 at kappa = 0.135, plus three masses around the pair of
zero crossings that the oracle finds for this field at m0 = -2.01333 and -1.99732
(real eigenvalues mu of D(m0 = 0) sit at m0 = -mu; sign pf(m0) = prod over real
mu of sign(mu + m0), Sec. 3).  The window between them has W_sgn = -1.  Each
stored sign is computed here twice, from the dense Pfaffian ratio to m_big and
from the negative-eigenvalue count of the dense Q, and the two must agree.

Run:  python tests/golden/make_tiny_golden.py      (about 5 minutes, 8 threads)
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from synth_inputs import WORKLOADS, kappa_to_m0, make_config  # noqa: E402
from oracle.dirac import WilsonDirac  # noqa: E402
from oracle.sign import m_big, sign_by_pfaffian  # noqa: E402

MASSES = [kappa_to_m0(0.135), -2.005, -1.98, -2.03]


def main():
    cfg = make_config(seed=0, **WORKLOADS["tiny_4x4x4x4"])
    op = WilsonDirac(cfg)
    out = {"workload": "tiny_4x4x4x4", "seed": 0, "m_big": m_big(cfg), "points": []}
    for m in MASSES:
        w = np.linalg.eigvalsh(op.dense_Q(m))
        nneg = int(np.sum(w < 0))
        s_eig = 1 if (nneg // 2) % 2 == 0 else -1
        s_pf, ratio = sign_by_pfaffian(op, m, use_c=True)
        assert s_pf == s_eig, (m, s_pf, s_eig)
        low = w[np.argsort(np.abs(w), kind="stable")][:24]
        out["points"].append({"m0": m, "sign": s_pf, "n_negative": nneg,
                              "pf_ratio_re": ratio.real, "pf_ratio_im": ratio.imag,
                              "lowest_abs_sorted_eigs_Q": low.tolist()})
        print(m, s_pf, low[:4], flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_4x4x4x4_seed0.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
