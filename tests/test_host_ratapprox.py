"""qs_ratapprox (host computation, no GPU) against the oracle's rational Remez and the
alternation certificate (Sec. 4, eq. ratapprox)."""
import numpy as np
import pytest

from oracle.reweight import rat_eval, ratapprox as ratapprox_oracle


@pytest.fixture(scope="module")
def qs():
    import paper_2108_11989_gb300 as qs
    return qs


@pytest.mark.parametrize("n,ratio", [(1, 10.0), (2, 10.0), (3, 30.0), (4, 100.0)])
def test_matches_oracle(qs, n, ratio):
    """The best approximation is unique: both sides give the same R within a small fraction
    of the error level (the oracle levels its error to about 1e-4 relative)."""
    A, nu, mu, d = qs.ratapprox(n, 1.0 / ratio, 1.0)
    A2, nu2, mu2, d2 = ratapprox_oracle(n, 1.0 / ratio, 1.0)
    assert d == pytest.approx(d2, rel=1e-4)
    y = np.exp(np.linspace(np.log(1.0 / ratio ** 2), 0.0, 20001))
    assert np.max(np.abs(rat_eval(A, nu, mu, y) / rat_eval(A2, nu2, mu2, y) - 1)) <= 1e-3 * d
    assert np.allclose(nu, nu2, rtol=1e-3) and np.allclose(mu, mu2, rtol=1e-3)


def test_best_constant(qs):
    A, nu, mu, d = qs.ratapprox(0, 0.2, 3.0)
    a, b = 0.2 ** 0.5, 3.0 ** 0.5          # (r^2)^(1/4)
    assert A == pytest.approx(2 / (a + b), rel=1e-15) and d == pytest.approx((b - a) / (b + a), rel=1e-15)


@pytest.mark.parametrize("n,ratio", [(8, 1e3), (12, 1e4), (16, 1e5), (6, 1e6)])
def test_equioscillation_at_higher_order(qs, n, ratio):
    """Orders the oracle does not reach: the relative error alternates 2n + 2 times at the
    level delta (alternation theorem), levelled to 1e-6 (de la Vallee Poussin bound)."""
    A, nu, mu, d = qs.ratapprox(n, 1.0 / ratio, 1.0)
    y = np.exp(np.linspace(np.log(1.0 / ratio ** 2), 0.0, 400001))
    e = rat_eval(A, nu, mu, y) * y ** 0.25 - 1
    runs = np.split(np.arange(len(e)), np.nonzero(np.diff(np.sign(e)))[0] + 1)
    ext = np.array([np.max(np.abs(e[r])) for r in runs])
    assert len(ext) == 2 * n + 2
    assert np.max(ext) == pytest.approx(d, rel=1e-6)
    assert np.min(ext) >= d * (1 - 1e-6)
    assert np.all(np.diff(nu) > 0) and np.all(np.diff(mu) > 0)
    # zeros and poles interlace on the negative axis, mu_1 < nu_1 < mu_2 < ... (R decreases)
    lab = np.concatenate([np.zeros(n), np.ones(n)])[np.argsort(np.concatenate([mu, nu]))]
    assert np.all(lab[0::2] == 0) and np.all(lab[1::2] == 1)


def test_rejects_bad_arguments(qs):
    for args in [(-1, 0.1, 1.0), (33, 0.1, 1.0), (2, 0.0, 1.0), (2, 1.0, 0.5)]:
        with pytest.raises(qs.QStarError):
            qs.ratapprox(*args)
