"""Pair-screening MLP, float64 numpy reference (forward, backward, Adam).

Test infrastructure only.  Not from the paper: the benchmark configuration asks for a small
network that predicts log|<phi_a|V|phi_b>| from the two quasiparticle momentum sets and skips
the Pfaffian of pairs it predicts negligible.

Features of a pair (NS state a, R state b) of a chain of length L, D_IN = 2 Q + 4, Q = 8:
  x[0:Q]      k/pi of a's modes, ascending, zero padded
  x[Q:2Q]     k/pi of b's modes, ascending, zero padded (k = pi for the R mode at pi)
  x[2Q]       M_a / Q
  x[2Q+1]     M_b / Q
  x[2Q+2]     24 / L
  x[2Q+3]     1
Target: y = log10|X_ab| + (M_a + M_b)/2 log10(L/24), clipped below at -30 (each quasiparticle
carries a 1/sqrt(L) plane-wave normalisation; the target removes it so that one network can
serve several L).

Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3; loss = mean (y - t)^2.
Parameters are flattened in the order W1 [H, D_IN], b1 [H], W2 [H, H], b2 [H], w3 [H], b3 [1].
"""
import math

import numpy as np

Q = 8
D_IN = 2 * Q + 4


def features(L, modes_a, modes_b, nlab_ns, nlab_r):
    """Feature rows for lists of (NS modes, R modes); nlab_* are the momentum labels n of the
    modes (k = pi n / L), as in oracle.modes.momenta_n."""
    x = np.zeros((len(modes_a), D_IN))
    for r, (ma, mb) in enumerate(zip(modes_a, modes_b)):
        for i, m in enumerate(ma):
            x[r, i] = nlab_ns[m] / L
        for i, m in enumerate(mb):
            x[r, Q + i] = nlab_r[m] / L
        x[r, 2 * Q] = len(ma) / Q
        x[r, 2 * Q + 1] = len(mb) / Q
        x[r, 2 * Q + 2] = 24.0 / L
        x[r, 2 * Q + 3] = 1.0
    return x


def target(L, X, M_a, M_b):
    ax = np.abs(X)
    y = np.where(ax > 0, np.log10(np.maximum(ax, 1e-300)), -30.0)
    return np.maximum(y + 0.5 * (np.asarray(M_a) + np.asarray(M_b)) * math.log10(L / 24.0), -30.0)


def shapes(H):
    return [(H, D_IN), (H,), (H, H), (H,), (H,), (1,)]


def unflatten(theta, H):
    out, o = [], 0
    for s in shapes(H):
        n = int(np.prod(s))
        out.append(theta[o:o + n].reshape(s))
        o += n
    return out


def n_params(H):
    return sum(int(np.prod(s)) for s in shapes(H))


def init(H, seed):
    """He-normal weights, zero biases."""
    g = np.random.default_rng(seed)
    W1 = g.standard_normal((H, D_IN)) * math.sqrt(2.0 / D_IN)
    W2 = g.standard_normal((H, H)) * math.sqrt(2.0 / H)
    w3 = g.standard_normal(H) * math.sqrt(1.0 / H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), w3, np.zeros(1)])


def forward(theta, H, x):
    W1, b1, W2, b2, w3, b3 = unflatten(theta, H)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3[0]
    return y, (z1, h1, z2, h2)


def loss_and_grad(theta, H, x, t):
    """Mean squared error and its gradient by back-propagation through the three layers."""
    W1, b1, W2, b2, w3, b3 = unflatten(theta, H)
    y, (z1, h1, z2, h2) = forward(theta, H, x)
    B = x.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B
    dw3 = h2.T @ dy
    db3 = np.array([dy.sum()])
    dz2 = np.outer(dy, w3) * (z2 > 0)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    dW1 = dz1.T @ x
    db1 = dz1.sum(0)
    return loss, np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, db3])


def adam_step(theta, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
