"""Training data and training loop of the step-proposal network.

Samples come from the sign flows the library itself runs (report["windows"] with
trace=True): for every step-A move from mass m_i to m_{i+1} the features are the
windows of the step-A masses up to m_i (newest first, 8 of them, divided by
lambda_bar(m_i), zero where missing) -- the same features qs_pfaffian_sign builds
for its proposals -- and the targets are
  y0 = log(dm* / lambda_bar_i), dm* = 0.95 ((lb_i - r_i) + (lb_{i+1} - r_{i+1})),
the longest step the no-crossing certificate of the observed pair would have
accepted, and, for each of the 24 window slots j, whether the signed value in slot j
changed sign between the two masses.  So T has 1 + 24 = 25 columns, the output width
of the step network.
"""
import numpy as np

WINDOW = 24
HIST = 8
N_IN = HIST * WINDOW     # network inputs: 8 windows of 24 scaled eigenvalues
N_OUT = 1 + WINDOW       # network outputs: log step + one crossing logit per slot


def samples_from_flow(report):
    """(X [n][8*24], T [n][1 + 24]) float32 from one flow report with windows."""
    W = report["windows"]
    ph = report["phase"]
    m = np.asarray(report["mass"])
    lb = np.asarray(report["lambda_bar"])
    r = np.asarray(report["resid"])
    a_idx = [i for i in range(len(ph)) if ph[i] == "A"]
    X, T = [], []
    for q in range(len(a_idx) - 1):
        i, j = a_idx[q], a_idx[q + 1]
        if j != i + 1 or not m[j] > m[i]:
            continue
        hist = [W[a_idx[p]] for p in range(q, max(-1, q - HIST), -1)]
        x = np.zeros((HIST, WINDOW))
        for h, w in enumerate(hist):
            x[h] = w / lb[i]
        dm = 0.95 * ((lb[i] - r[i]) + (lb[j] - r[j]))
        if not dm > 0:
            continue
        t = np.zeros(N_OUT)
        t[0] = np.log(dm / lb[i])
        t[1:] = (np.sign(W[i][:WINDOW]) * np.sign(W[j][:WINDOW]) < 0).astype(float)
        X.append(x.ravel())
        T.append(t)
    if not X:
        return np.zeros((0, N_IN), np.float32), np.zeros((0, N_OUT), np.float32)
    return np.asarray(X, np.float32), np.asarray(T, np.float32)


def train(net, X, T, steps=400, lr=2e-3, batch=256, seed=0):
    """Adam on random mini-batches, every step through qs_mlp_train_step; returns losses."""
    import torch
    rng = np.random.default_rng(seed)
    Xd = torch.from_numpy(X).cuda()
    Td = torch.from_numpy(T).cuda()
    losses = []
    for _ in range(steps):
        idx = torch.from_numpy(rng.integers(0, len(X), size=min(batch, len(X)))).cuda()
        losses.append(net.train_step(Xd[idx].contiguous(), Td[idx].contiguous(), lr))
    return losses
