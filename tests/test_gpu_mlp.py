"""The step-proposal network trained by the library's own kernels (qs_mlp_*) against
the FP64 oracle: forward, loss, gradients (FP32 vs FP64, relative 1e-4) and a short
Adam training run."""
import numpy as np
import pytest

from synth_inputs import mlp_init
from oracle import mlp as ref

pytestmark = pytest.mark.gpu


def problem(seed, B, ni=192, nh=128, no=25):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, ni)).astype(np.float32)
    T = np.concatenate([rng.standard_normal((B, 1)), rng.random((B, no - 1)) < 0.3], axis=1).astype(np.float32)
    return X, T


def test_forward_and_gradients_match_oracle():
    import torch
    import paper_2108_11989_gb300 as qs
    ni, nh, no, B = 192, 128, 25, 96
    p0 = mlp_init(7, ni, nh, no)
    p0 = [p + np.float32(0.05) * np.random.default_rng(i).standard_normal(p.shape).astype(np.float32)
          for i, p in enumerate(p0)]
    X, T = problem(1, B)
    net = qs.MLP(ni, nh, no, max_batch=256)
    net.set_params(p0)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    Y = net.forward(Xd).cpu().numpy()
    Yr, _ = ref.forward(p0, X)
    assert np.abs(Y - Yr).max() <= 1e-4 * np.abs(Yr).max()
    loss = net.train_step(Xd, Td, lr=1e-3)
    Lr, gr = ref.value_and_grad(p0, X, T)
    assert abs(loss - Lr) <= 1e-4 * abs(Lr)
    for g, h in zip(net.get_grads(), gr):
        assert np.abs(g - h).max() <= 1e-4 * np.abs(h).max() + 1e-7
    net.close()


def test_training_follows_oracle_and_reduces_loss():
    import torch
    import paper_2108_11989_gb300 as qs
    ni, nh, no, B = 192, 128, 25, 128
    p0 = mlp_init(11, ni, nh, no)
    X, T = problem(2, B)
    net = qs.MLP(ni, nh, no, max_batch=B)
    net.set_params(p0)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    opt = ref.Adam(p0, lr=1e-3)
    losses, ref_losses = [], []
    for _ in range(30):
        losses.append(net.train_step(Xd, Td, lr=1e-3))
        L, g = ref.value_and_grad(opt.p, X, T)
        ref_losses.append(L)
        opt.step(g)
    assert losses[-1] < 0.7 * losses[0]
    assert np.allclose(losses, ref_losses, rtol=2e-3)
    net.close()
