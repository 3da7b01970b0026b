"""Host-side helpers of the package (no GPU work): the tiled-layout permutation and the
learned step's training-sample builder."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _package():
    spec = importlib.util.spec_from_file_location("_qs_build", os.path.join(ROOT, "paper_2108_11989_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    import paper_2108_11989_gb300 as qs
    return qs


def test_tiled_layout_round_trip_and_formula():
    import torch
    qs = _package()
    ns, n = 48, 3
    x = torch.arange(n * ns * 24, dtype=torch.float64)
    t = qs.to_tiled(x, ns)
    assert torch.equal(qs.from_tiled(t, ns), x)
    # element (rhs r, site s, spin-colour c, re/im q) sits at
    # r*ns*24 + (((s // 16) * 12 + c) * 16 + s % 16) * 2 + q
    for r, s, c, q in [(0, 0, 0, 0), (2, 47, 11, 1), (1, 17, 5, 0)]:
        canon = ((r * ns + s) * 12 + c) * 2 + q
        tiled = r * ns * 24 + (((s // 16) * 12 + c) * 16 + s % 16) * 2 + q
        assert t[tiled].item() == x[canon].item()


def test_samples_from_flow():
    from paper_2108_11989_gb300.learned import samples_from_flow
    # three step-A masses, lambda_bar doubling, then a B point
    W = np.zeros((4, 24))
    W[:, 0] = [0.1, 0.2, 0.4, 0.35]
    W[:, 1] = [-0.3, -0.25, 0.1, 0.2]
    rep = {"windows": W, "phase": "AAAB", "mass": [0.0, 0.19, 0.57, 0.6],
           "lambda_bar": [0.1, 0.2, 0.4, 0.35], "resid": [0.0, 0.0, 0.0, 0.0]}
    X, T = samples_from_flow(rep)
    assert X.shape == (2, 192) and T.shape == (2, 25)     # 1 step target + 24 crossing labels
    assert np.isclose(T[0, 0], np.log(0.95 * (0.1 + 0.2) / 0.1))
    assert X[0, 0] == np.float32(1.0)               # newest window / its lambda_bar
    assert X[1, 24] == np.float32(0.1 / 0.2)         # previous step-A window, scaled
    assert T[1, 2] == 1.0 and T[0, 2] == 0.0         # slot 1 changes sign between masses 1 and 2
    W[:, 23] = [0.5, -0.5, -0.5, 0.5]                # the last slot has its own label
    X, T = samples_from_flow(rep)
    assert T[0, 24] == 1.0 and T[1, 24] == 0.0
