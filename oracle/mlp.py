"""Float64 reference of the frontier predictor -- TEST INFRASTRUCTURE ONLY.

The predictor is a two-hidden-layer perceptron over one node's local view:
its head symbol, the head symbols of its arguments (symbol 0 = no argument)
and whether each argument is in normal form.  The input is the concatenation
of one-hot codes x = [onehot(h), onehot(a_0), ..., onehot(a_{MA-1}), b_0..b_{MA-1}]
of dimension D = nsym * (1 + MA) + MA, and

    h1 = relu(W1 x + b1)        W1: H x D
    h2 = relu(W2 h1 + b2)       W2: H x H
    z  = w3 . h2 + b3           p = sigmoid(z)

trained with the mean binary cross-entropy (positives weighted by pos_weight)
and Adam.  The flat parameter vector is [W1 (row-major), b1, W2 (row-major),
b2, w3, b3]; features are int rows [h, a_0..a_{MA-1}, bits] with bit j of
`bits` set when argument j is in normal form.  Plain numpy, no batching tricks,
so each line can be checked against the formulas above.
"""
from __future__ import annotations

import numpy as np


def dims(nsym: int, ma: int, hidden: int):
    d = nsym * (1 + ma) + ma
    sizes = [hidden * d, hidden, hidden * hidden, hidden, hidden, 1]
    return d, sizes


def unpack(theta, nsym, ma, hidden):
    d, sizes = dims(nsym, ma, hidden)
    parts, at = [], 0
    for s in sizes:
        parts.append(np.asarray(theta[at:at + s], dtype=np.float64))
        at += s
    W1, b1, W2, b2, w3, b3 = parts
    return W1.reshape(hidden, d), b1, W2.reshape(hidden, hidden), b2, w3, b3[0]


def encode(feat, nsym, ma):
    """One-hot input matrix (n x D) from feature rows."""
    feat = np.asarray(feat, dtype=np.int64)
    n = len(feat)
    d = nsym * (1 + ma) + ma
    X = np.zeros((n, d), dtype=np.float64)
    rows = np.arange(n)
    X[rows, feat[:, 0]] = 1.0
    for j in range(ma):
        X[rows, nsym * (1 + j) + feat[:, 1 + j]] = 1.0
        X[rows, nsym * (1 + ma) + j] = (feat[:, 1 + ma] >> j) & 1
    return X


def forward(theta, feat, nsym, ma, hidden):
    W1, b1, W2, b2, w3, b3 = unpack(theta, nsym, ma, hidden)
    X = encode(feat, nsym, ma)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    z = h2 @ w3 + b3
    return z, (X, z1, h1, z2, h2)


def prob(theta, feat, nsym, ma, hidden):
    z, _ = forward(theta, feat, nsym, ma, hidden)
    return 1.0 / (1.0 + np.exp(-z))


def loss(theta, feat, y, nsym, ma, hidden, pos_weight=1.0):
    z, _ = forward(theta, feat, nsym, ma, hidden)
    y = np.asarray(y, dtype=np.float64)
    # -[w y log s(z) + (1-y) log(1-s(z))], written with log1p(exp(-|z|)) for range
    log_s = -(np.maximum(-z, 0) + np.log1p(np.exp(-np.abs(z))))
    log_1ms = -(np.maximum(z, 0) + np.log1p(np.exp(-np.abs(z))))
    return float(np.mean(-(pos_weight * y * log_s + (1 - y) * log_1ms)))


def grad(theta, feat, y, nsym, ma, hidden, pos_weight=1.0):
    """Gradient of `loss` with respect to theta (same flat layout)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta, nsym, ma, hidden)
    z, (X, z1, h1, z2, h2) = forward(theta, feat, nsym, ma, hidden)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    s = 1.0 / (1.0 + np.exp(-z))
    dz = (s * (pos_weight * y + 1 - y) - pos_weight * y) / n
    dw3 = h2.T @ dz
    db3 = dz.sum()
    dh2 = np.outer(dz, w3) * (z2 > 0)
    dW2 = dh2.T @ h1
    db2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (z1 > 0)
    dW1 = dh1.T @ X
    db1 = dh1.sum(axis=0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])


def adam_step(theta, g, m, v, t, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
