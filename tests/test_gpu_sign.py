"""Pfaffian sign through the C-ABI (qs_pfaffian_sign) against the oracle: bit-exact."""
import json
import os

import numpy as np
import pytest

from synth_inputs import WORKLOADS, make_config
from oracle.dirac import WilsonDirac
from oracle.sign import sign_by_eigencount

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


def test_rough_small_lattice_negative_signs(qs):
    cfg = make_config(T=4, L=2, eps=2.0, theta_sigma=0.3, csw_su3=1.5, csw_u1=1.0, seed=2)
    op = WilsonDirac(cfg)
    lat = lattice(qs, cfg)
    opts = qs.sign_default_opts(eig={"k": 16, "nwant": 2, "tol": 1e-6, "cheb_degree": 16})
    got = []
    for m in [-2.05, -1.85, -1.65, -1.5, 0.3]:
        ref = sign_by_eigencount(op, m)
        s, rep = lat.pfaffian_sign(m, opts)
        assert s == ref, (m, s, ref, rep["phase"])
        got.append(s)
    assert -1 in got
    lat.close()


def test_tiny_workload_golden_signs(qs):
    """4^4 workload at the 4 golden masses (dense Pfaffian and eigen-count agree)."""
    g = json.load(open(os.path.join(HERE, "golden", "tiny_4x4x4x4_seed0.json")))
    cfg = make_config(seed=0, **WORKLOADS["tiny_4x4x4x4"])
    lat = lattice(qs, cfg)
    opts = qs.sign_default_opts(eig={"k": 16, "nwant": 2, "tol": 1e-6, "cheb_degree": 24})
    signs = []
    for pt in g["points"]:
        s, rep = lat.pfaffian_sign(pt["m0"], opts)
        assert s == pt["sign"], (pt["m0"], s, pt["sign"], rep["phase"])
        signs.append(s)
    assert -1 in signs
    lat.close()


def test_large_mass_is_positive_in_one_step(qs):
    cfg = make_config(T=4, L=4, eps=0.5, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0, seed=3)
    lat = lattice(qs, cfg)
    s, rep = lat.pfaffian_sign(3 * (1.9 + 1.0) + 0.5, qs.sign_default_opts())
    assert s == 1 and rep["n"] == 1
    lat.close()


def test_batched_sign_matches_single_flows(qs):
    """qs_pfaffian_sign_batch over configurations of different volumes, each handle on
    its own stream: every sign equals the dense oracle's and the single-flow result."""
    import torch
    cfgs = [make_config(T=4, L=2, eps=2.0, theta_sigma=0.3, csw_su3=1.5, csw_u1=1.0, seed=2),
            make_config(seed=0, **WORKLOADS["tiny_4x4x4x4"]),
            make_config(T=6, L=2, eps=1.2, theta_sigma=0.3, csw_su3=1.5, csw_u1=1.0, seed=4)]
    masses = [-1.65, -2.005, -0.5]
    streams = [torch.cuda.Stream() for _ in cfgs]
    lats = []
    for c, st in zip(cfgs, streams):
        lat = qs.Lattice(c.L, c.T, stream=st)
        lat.load_gauge(c.su3, c.theta, c.csw_su3, c.csw_u1)
        lats.append(lat)
    opts = qs.sign_default_opts(eig={"k": 16, "nwant": 2, "tol": 1e-6, "cheb_degree": 24})
    out = qs.pfaffian_sign_batch(lats, masses, opts)
    for (s, status, rep), lat, m, c in zip(out, lats, masses, cfgs):
        assert status == 0
        ref = sign_by_eigencount(WilsonDirac(c), m) if c.n_sites * 12 <= 2000 else None
        if ref is not None:
            assert s == ref, (m, s, ref)
        s1, _ = lat.pfaffian_sign(m, opts)
        assert s1 == s
    assert out[1][0] == -1          # the 4^4 golden mass -2.005 has W_sgn = -1
    for lat in lats:
        lat.close()


def test_block_bounds_take_the_smallest_informative_lower_bound(qs):
    """Step A's bounds (Sec. 3, derivative bound) come from the whole block: the block is
    ordered by theta^2 + r^2, so the smallest |theta_j| - r_j can belong to a later value."""
    theta = [0.30, -0.31, 0.05, 0.9]
    res = [0.01, 0.10, 0.04, 0.5]
    # value 1 (r <= |theta| / 2) has the smallest lower bound, 0.21, below value 0's 0.29;
    # value 2 (r > |theta| / 2, beyond nwant) is an unconverged mixture and is skipped
    lb, lo = qs.block_bounds(theta, res, nwant=1)
    assert lb == 0.30 and abs(lo - 0.21) < 1e-15
    # within nwant every value counts, converged or not
    lb, lo = qs.block_bounds(theta, res, nwant=3)
    assert lb == 0.05 and abs(lo - 0.01) < 1e-15


def test_block_bounds_certify_the_exact_spectrum(qs):
    """On the rough 2^3x4 field: lo from a solved block lies below the exact smallest
    |lambda| of Q (dense oracle) and within the eigensolver's tolerance of it."""
    cfg = make_config(T=4, L=2, eps=2.0, theta_sigma=0.3, csw_su3=1.5, csw_u1=1.0, seed=2)
    op = WilsonDirac(cfg)
    lat = lattice(qs, cfg)
    for m in (-1.85, -1.5):
        o = qs.eig_default_opts(k=16, nwant=4, tol=1e-8, cheb_degree=16)
        ev, rs, _ = lat.lowmodes_at_mass(m, o)
        lb, lo = qs.block_bounds(ev, rs, nwant=4)
        exact = np.min(np.abs(np.linalg.eigvalsh(op.dense_Q(m))))
        # 1e-12: the rounding of the FP64 residual itself (about 1e-15 ||Q||) is not part of r
        assert lo <= exact + 1e-12 and exact <= lb + 1e-6, (m, lo, exact, lb)
        assert exact - lo < 1e-6 * max(1.0, exact)
    lat.close()


def test_checkpoint_resume_and_step_log(qs, tmp_path):
    """The JSON-lines log has one line per mass visited; a flow cut short by max_steps and
    resumed from its last certified mass gives the uninterrupted flow's (and the oracle's)
    sign; a checkpoint of another target mass is ignored."""
    cfg = make_config(T=4, L=2, eps=2.0, theta_sigma=0.3, csw_su3=1.5, csw_u1=1.0, seed=2)
    op = WilsonDirac(cfg)
    lat = lattice(qs, cfg)
    eig = {"k": 16, "nwant": 2, "tol": 1e-6, "cheb_degree": 16}
    m = -1.65
    log, ck, ck2 = tmp_path / "flow.jsonl", tmp_path / "full.json", tmp_path / "cut.json"
    s_full, rep = lat.pfaffian_sign(m, qs.sign_default_opts(eig=eig, log_path=log, checkpoint_path=ck))
    assert s_full == sign_by_eigencount(op, m)
    lines = [json.loads(x) for x in open(log)]
    assert [x["mass"] for x in lines] == rep["mass"] and "".join(x["phase"] for x in lines) == rep["phase"]
    assert all(x["lower_bound"] <= x["lambda_bar"] for x in lines)
    saved = json.load(open(ck))
    assert saved["m_target"] == m and saved["m"] in rep["mass"] and rep["checkpoint_errors"] == 0
    # cut short and resumed: at m = 0.3, away from the crossings, step A certifies its steps,
    # so the cut flow leaves a checkpoint beyond the target
    m2 = 0.3
    s_a, rep_a = lat.pfaffian_sign(m2, qs.sign_default_opts(eig=eig))
    assert rep_a["n"] >= 3 and s_a == sign_by_eigencount(op, m2)
    with pytest.raises(qs.QStarError):     # one step, then the cap
        lat.pfaffian_sign(m2, qs.sign_default_opts(eig=eig, max_steps=1, checkpoint_path=ck2))
    cut = json.load(open(ck2))
    # the same first step as the uninterrupted flow, up to the eigensolver's tolerance (the
    # handle's warm start differs between the runs)
    assert cut["m"] > m2 and cut["steps"] == 1 and abs(cut["m"] - rep_a["mass"][1]) < 1e-6
    s_res, rep_res = lat.pfaffian_sign(m2, qs.sign_default_opts(eig=eig, checkpoint_path=ck2, resume=1))
    assert s_res == s_a and rep_res["resumed_from"] == cut["m"]
    assert rep_res["mass"][0] == cut["m"]
    # another target: the checkpoint does not apply and the flow starts from the target
    s_other, rep_other = lat.pfaffian_sign(m, qs.sign_default_opts(eig=eig, checkpoint_path=ck2, resume=1))
    assert rep_other["resumed_from"] == m and s_other == s_full
    lat.close()
