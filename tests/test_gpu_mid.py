"""Parity at the block size and flow settings of the benchmark (k = 32, nwant = 2,
tol = 1e-5, Chebyshev degree 48) on a 4^3 x 6 field (n = 9216) whose dense oracle values
are stored in tests/golden/mid_4x4x4x6_seed7.json (written by make_mid_golden.py from
the oracle alone): the 32 eigenvalues of Q nearest zero at four masses, and W_sgn there
(dense Pfaffian ratio, negative count and crossing list agree).  Near m0 = -4 the
spectrum is dense (|lambda| ~ 1e-3) and two pairs cross zero, at m0 = -4.0525 and
-4.0163, so the flows from the lower masses go through step B with counted crossings.

Tolerances: 1e-10 relative on eigenvalues (FP64 Rayleigh-Ritz); signs bit-exact."""
import json
import os

import numpy as np
import pytest

from synth_inputs import make_config

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def golden():
    return json.load(open(os.path.join(HERE, "golden", "mid_4x4x4x6_seed7.json")))


@pytest.fixture(scope="module")
def lat(golden):
    import paper_2108_11989_gb300 as qs
    cfg = make_config(**golden["field"])
    lat = qs.Lattice(cfg.L, cfg.T)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    yield lat
    lat.close()


@pytest.mark.parametrize("precision", [1, 2])     # FP32 / FP16 filter storage
def test_k32_eigenvalues(golden, lat, precision):
    import paper_2108_11989_gb300 as qs
    opts = qs.eig_default_opts(k=32, nwant=8, tol=1e-9, cheb_degree=48, precision=precision, warm_start=0)
    for pt in (golden["points"][0], golden["points"][3]):
        ev, rs, st = lat.lowmodes_at_mass(pt["m0"], opts)
        ref = np.array(pt["lowest_abs_sorted_eigs_Q"])
        for i in range(8):
            j = np.argmin(np.abs(ref - ev[i]))
            assert abs(ev[i] - ref[j]) <= 1e-10 * abs(ref[j]) + 1e-14, (pt["m0"], i, ev[i], ref[j])
            assert abs(ev[i] - ref[j]) <= rs[i] + 1e-13
        assert np.allclose(np.sort(np.abs(ev[:8])), np.abs(ref[:8]), rtol=1e-10, atol=1e-14)


def test_k32_sign_at_physical_mass(golden, lat):
    """W_sgn at kappa = 0.135 with the benchmark's flow settings (the lower golden masses
    sit in the dense doubler spectrum near m0 = -4, below every crossing of the field;
    their signs are checked at k = 32 on the 4^4 golden field instead)."""
    import paper_2108_11989_gb300 as qs
    pt = golden["points"][0]
    for retreat in (0, 1):
        opts = qs.sign_default_opts(eig={"k": 32, "nwant": 2, "tol": 1e-5, "cheb_degree": 48, "precision": 2})
        opts.retreat = retreat
        opts.max_steps = 120
        s, rep = lat.pfaffian_sign(pt["m0"], opts)
        assert s == pt["sign"], (retreat, s, rep["phase"])


@pytest.mark.parametrize("retreat", [0, 1])
def test_k32_signs_across_crossings_tiny_golden(retreat):
    """4^4 golden field (tests/golden/tiny_4x4x4x4_seed0.json): W_sgn at the four golden
    masses with the benchmark's block size and settings; the flows from -2.03 and -2.005
    cross the pair of zero crossings near m0 = -2.01 and -2.00 in step B."""
    import paper_2108_11989_gb300 as qs
    from synth_inputs import WORKLOADS
    g = json.load(open(os.path.join(HERE, "golden", "tiny_4x4x4x4_seed0.json")))
    cfg = make_config(seed=0, **WORKLOADS["tiny_4x4x4x4"])
    lat = qs.Lattice(cfg.L, cfg.T)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    crossed = 0
    for pt in g["points"]:
        opts = qs.sign_default_opts(eig={"k": 32, "nwant": 2, "tol": 1e-5, "cheb_degree": 48, "precision": 2})
        opts.retreat = retreat
        opts.max_steps = 200
        s, rep = lat.pfaffian_sign(pt["m0"], opts)
        assert s == pt["sign"], (pt["m0"], s, pt["sign"], rep["phase"][:40], rep["fail_reason"])
        crossed += rep["crossings"]
    assert crossed >= 3
    lat.close()
