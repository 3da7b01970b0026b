"""Learned step proposals in the sign flow: the network is trained on flows the
library computes, by the library's kernels, and its proposals are accepted only
when the no-crossing certificate holds, so signs must equal the plain flow's.
The gain (mass points visited with / without the network) is printed."""
import numpy as np
import pytest

from synth_inputs import make_config, mlp_init

pytestmark = pytest.mark.gpu


def cfg(seed):
    return make_config(T=4, L=4, eps=0.6, theta_sigma=0.3, csw_su3=1.5, csw_u1=1.0, seed=seed)


def test_learned_steps_keep_signs_and_report_gain():
    import paper_2108_11989_gb300 as qs
    from paper_2108_11989_gb300.learned import samples_from_flow, train
    m_target = -0.45
    opts = qs.sign_default_opts(eig={"k": 16, "nwant": 2, "tol": 1e-6, "cheb_degree": 24})
    Xs, Ts = [], []
    for seed in range(8):
        c = cfg(seed)
        lat = qs.Lattice(c.L, c.T)
        lat.load_gauge(c.su3, c.theta, c.csw_su3, c.csw_u1)
        _, rep = lat.pfaffian_sign(m_target, opts, trace=True)
        X, T = samples_from_flow(rep)
        Xs.append(X)
        Ts.append(T)
        lat.close()
    X, T = np.concatenate(Xs), np.concatenate(Ts)
    assert len(X) >= 20
    net = qs.MLP(192, 128, 25, max_batch=512)
    net.set_params(mlp_init(0, 192, 128, 25))
    losses = train(net, X, T, steps=300, lr=2e-3)
    assert losses[-1] < losses[0]
    plain_n, learned_n, accepted, rejected = 0, 0, 0, 0
    held_X = []
    for seed in range(100, 104):
        c = cfg(seed)
        lat = qs.Lattice(c.L, c.T)
        lat.load_gauge(c.su3, c.theta, c.csw_su3, c.csw_u1)
        s0, r0 = lat.pfaffian_sign(m_target, opts, trace=True)
        held_X.append(samples_from_flow(r0)[0])
        s1, r1 = lat.pfaffian_sign(m_target, opts, step_model=net)
        assert s0 == s1
        plain_n += r0["n"]
        learned_n += r1["n"]
        accepted += r1["learned_accepted"]
        rejected += r1["learned_rejected"]
        lat.close()
    assert accepted + rejected > 0
    # the trained network on held-out windows: the library's forward pass equals the FP64
    # oracle's forward pass with the same parameters
    import torch
    from oracle import mlp as mlp_oracle
    Xh = np.concatenate(held_X)
    assert len(Xh) > 0
    Yg = net.forward(torch.from_numpy(np.ascontiguousarray(Xh, dtype=np.float32)).cuda()).cpu().numpy()
    Yr, _ = mlp_oracle.forward(net.get_params(), Xh)
    assert np.abs(Yg - Yr).max() <= 1e-4 * (1.0 + np.abs(Yr).max())
    print(f"\n[learned step] samples={len(X)} loss {losses[0]:.3f}->{losses[-1]:.3f}; mass points "
          f"plain={plain_n} learned={learned_n}; proposals accepted={accepted} rejected={rejected}")
    net.close()
