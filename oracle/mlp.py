"""FP64 reference of the learned proposer's network.

TEST INFRASTRUCTURE ONLY: the GPU training kernels are checked against it.
A 3-layer MLP x -> relu(W1 x + b1) -> relu(W2 h1 + b2) -> W3 h2 + b3 with the
loss (1/2n) sum_i (f(x_i) - y_i)^2, written out with numpy in FP64:
forward, and the analytic backward pass by the chain rule, layer by layer.
Parameters are one flat array W1 (H x F), b1 (H), W2 (H x H), b2 (H), W3 (H), b3 (1).
"""
import numpy as np


def unpack(p, F, H):
    p = np.asarray(p, np.float64)
    i = 0
    out = []
    for shape in [(H, F), (H,), (H, H), (H,), (H,), (1,)]:
        n = int(np.prod(shape))
        out.append(p[i:i + n].reshape(shape))
        i += n
    assert i == p.size
    return out


def forward(p, X, F, H):
    W1, b1, W2, b2, W3, b3 = unpack(p, F, H)
    X = np.asarray(X, np.float64)
    Z1 = X @ W1.T + b1
    H1 = np.maximum(Z1, 0)
    Z2 = H1 @ W2.T + b2
    H2 = np.maximum(Z2, 0)
    return H2 @ W3 + b3[0], (X, Z1, H1, Z2, H2)


def loss_and_grad(p, X, y, F, H):
    W1, b1, W2, b2, W3, b3 = unpack(p, F, H)
    P, (X, Z1, H1, Z2, H2) = forward(p, X, F, H)
    n = X.shape[0]
    e = P - np.asarray(y, np.float64)
    loss = float(e @ e) / (2 * n)
    dP = e / n
    gW3 = dP @ H2
    gb3 = np.array([dP.sum()])
    dH2 = np.outer(dP, W3)
    dZ2 = dH2 * (Z2 > 0)
    gW2 = dZ2.T @ H1
    gb2 = dZ2.sum(0)
    dH1 = dZ2 @ W2
    dZ1 = dH1 * (Z1 > 0)
    gW1 = dZ1.T @ X
    gb1 = dZ1.sum(0)
    return loss, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])


def loss_only(p, X, y, F, H):
    P, _ = forward(p, X, F, H)
    e = P - np.asarray(y, np.float64)
    return float(e @ e) / (2 * X.shape[0])
