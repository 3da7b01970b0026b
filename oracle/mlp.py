"""FP64 oracle of the step-proposal network (test infrastructure only).

The network proposes the next mass step of the sign flow from the recent low
spectrum (the learned part of the batched/learned form of the hot path; the paper
itself uses the fixed rule m <- m + c lambda_bar of Sec. 3).  Architecture:
  Z1 = X W1^T + b1, A1 = relu(Z1), Z2 = A1 W2^T + b2, A2 = relu(Z2), Y = A2 W3^T + b3.
Loss over a batch of B rows (T = targets, column 0 a regression target, columns
1.. binary labels):
  L = (1/B) sum_b [ (Y_b0 - T_b0)^2 / 2 + sum_{j>=1} (softplus(Y_bj) - T_bj Y_bj) ].
Adam (Kingma & Ba, ICLR 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Pinned by tests/test_oracle_mlp.py: the loss against a closed form, gradients
against central finite differences, the first Adam step (which moves every
parameter by lr * sign(g) + O(eps)), five steps with a constant gradient (exact bias
corrections: each moves p by lr g / (|g| + eps)), and two steps on p^2 / 2 against
values worked out by hand.
"""
import numpy as np


def forward(params, X):
    W1, b1, W2, b2, W3, b3 = [np.asarray(p, dtype=np.float64) for p in params]
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ W1.T + b1
    A1 = np.maximum(Z1, 0.0)
    Z2 = A1 @ W2.T + b2
    A2 = np.maximum(Z2, 0.0)
    Y = A2 @ W3.T + b3
    return Y, (X, Z1, A1, Z2, A2)


def loss(Y, T):
    B = Y.shape[0]
    r = Y[:, 0] - T[:, 0]
    z, t = Y[:, 1:], T[:, 1:]
    sp = np.logaddexp(0.0, z)
    return (0.5 * np.sum(r * r) + np.sum(sp - t * z)) / B


def loss_grad(Y, T):
    B = Y.shape[0]
    d = np.empty_like(Y)
    d[:, 0] = (Y[:, 0] - T[:, 0]) / B
    d[:, 1:] = (1.0 / (1.0 + np.exp(-Y[:, 1:])) - T[:, 1:]) / B
    return d


def backward(params, cache, dY):
    W1, b1, W2, b2, W3, b3 = [np.asarray(p, dtype=np.float64) for p in params]
    X, Z1, A1, Z2, A2 = cache
    dW3 = dY.T @ A2
    db3 = dY.sum(axis=0)
    dZ2 = (dY @ W3) * (Z2 > 0)
    dW2 = dZ2.T @ A1
    db2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * (Z1 > 0)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(axis=0)
    return [dW1, db1, dW2, db2, dW3, db3]


def value_and_grad(params, X, T):
    Y, cache = forward(params, X)
    T = np.asarray(T, dtype=np.float64)
    return loss(Y, T), backward(params, cache, loss_grad(Y, T))


class Adam:
    def __init__(self, params, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.p = [np.asarray(x, dtype=np.float64).copy() for x in params]
        self.m = [np.zeros_like(x) for x in self.p]
        self.v = [np.zeros_like(x) for x in self.p]
        self.lr, self.b1, self.b2, self.eps, self.t = lr, beta1, beta2, eps, 0

    def step(self, grads):
        self.t += 1
        for i, g in enumerate(grads):
            self.m[i] = self.b1 * self.m[i] + (1 - self.b1) * g
            self.v[i] = self.b2 * self.v[i] + (1 - self.b2) * g * g
            mh = self.m[i] / (1 - self.b1 ** self.t)
            vh = self.v[i] / (1 - self.b2 ** self.t)
            self.p[i] = self.p[i] - self.lr * mh / (np.sqrt(vh) + self.eps)
        return self.p
