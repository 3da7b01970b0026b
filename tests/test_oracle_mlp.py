"""Pins of oracle/mlp.py: finite-difference gradients, first Adam step."""
import numpy as np

from synth_inputs import mlp_init
from oracle import mlp


def small_problem(seed=0, B=7, n_in=6, n_h=5, n_out=4):
    rng = np.random.default_rng(seed)
    params = [p.astype(np.float64) for p in mlp_init(seed, n_in, n_h, n_out)]
    params = [p + 0.1 * rng.standard_normal(p.shape) for p in params]   # nonzero biases
    X = rng.standard_normal((B, n_in))
    T = np.concatenate([rng.standard_normal((B, 1)), (rng.random((B, n_out - 1)) < 0.5)], axis=1)
    return params, X, T


def test_gradients_match_finite_differences():
    params, X, T = small_problem()
    L, grads = mlp.value_and_grad(params, X, T)
    h = 1e-6
    for i, p in enumerate(params):
        it = np.nditer(p, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            pp = [q.copy() for q in params]
            pm = [q.copy() for q in params]
            pp[i][idx] += h
            pm[i][idx] -= h
            fd = (mlp.value_and_grad(pp, X, T)[0] - mlp.value_and_grad(pm, X, T)[0]) / (2 * h)
            assert abs(fd - grads[i][idx]) <= 1e-6 * (1 + abs(fd)), (i, idx, fd, grads[i][idx])


def test_loss_closed_form():
    # one row, zero logits: L = (y0 - t0)^2 / 2 + (n_out - 1) log 2
    Y = np.array([[1.5, 0.0, 0.0, 0.0]])
    T = np.array([[0.5, 1.0, 0.0, 1.0]])
    assert np.isclose(mlp.loss(Y, T), 0.5 + 3 * np.log(2.0))


def test_first_adam_step_is_sign_of_gradient():
    params, X, T = small_problem(seed=3)
    _, grads = mlp.value_and_grad(params, X, T)
    opt = mlp.Adam(params, lr=1e-2)
    new = opt.step(grads)
    for p, q, g in zip(params, new, grads):
        step = p - q
        mask = np.abs(g) > 1e-3        # step = lr g / (|g| + eps)
        assert np.allclose(step[mask], 1e-2 * np.sign(g[mask]), rtol=1e-4)


def test_adam_constant_gradient_moves_lr_every_step():
    """With a constant gradient g the bias corrections are exact: m / (1 - b1^t) = g and
    v / (1 - b2^t) = g^2 for every t, so each step moves p by lr g / (|g| + eps).  A
    wrong correction exponent breaks this from t = 2 on."""
    p0 = [np.array([0.3, -2.0, 5.0])]
    g = [np.array([0.7, -1.3, 0.02])]
    opt = mlp.Adam(p0, lr=0.05)
    prev = p0[0].copy()
    for t in range(1, 6):
        cur = opt.step(g)[0].copy()
        assert np.allclose(prev - cur, 0.05 * g[0] / (np.abs(g[0]) + 1e-8), rtol=1e-12, atol=0)
        prev = cur


def test_adam_two_steps_on_a_quadratic_by_hand():
    """f(p) = p^2 / 2, p0 = 1, lr = 0.1, eps = 0 (limit), Adam (Kingma & Ba):
    step 1: g = 1, m = 0.1, v = 0.001, m^ = 0.1 / 0.1 = 1, v^ = 0.001 / 0.001 = 1, p1 = 0.9.
    step 2: g = 0.9, m = 0.9 * 0.1 + 0.1 * 0.9 = 0.18, v = 0.999 * 0.001 + 0.001 * 0.81
    = 0.001809, m^ = 0.18 / (1 - 0.81) = 0.18 / 0.19, v^ = 0.001809 / (1 - 0.998001)
    = 0.001809 / 0.001999, p2 = 0.9 - 0.1 * (0.18 / 0.19) / sqrt(0.001809 / 0.001999)."""
    opt = mlp.Adam([np.array([1.0])], lr=0.1, eps=0.0)
    p1 = opt.step([np.array([1.0])])[0][0]
    assert p1 == 0.9
    p2 = opt.step([np.array([p1])])[0][0]
    expect = 0.9 - 0.1 * (0.18 / 0.19) / np.sqrt(0.001809 / 0.001999)
    assert abs(p2 - expect) < 1e-14
    # the values a swapped beta or a fixed t = 1 correction would give are far away
    assert abs(p2 - (0.9 - 0.1 * (0.18 / 0.1) / np.sqrt(0.001809 / 0.001))) > 1e-2
