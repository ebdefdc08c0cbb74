"""Pins of the float64 predictor reference (oracle/mlp.py): central finite
differences for the gradient, a hand-computed tiny network, and the Adam
update written out for one scalar."""
import numpy as np

from oracle import mlp


def _rand(nsym=5, ma=2, hidden=4, n=7, seed=0):
    rng = np.random.default_rng(seed)
    d, sizes = mlp.dims(nsym, ma, hidden)
    theta = rng.normal(0, 0.7, size=sum(sizes))
    feat = np.zeros((n, 2 + ma), dtype=np.int64)
    feat[:, 0] = rng.integers(1, nsym, n)
    for j in range(ma):
        feat[:, 1 + j] = rng.integers(0, nsym, n)
    feat[:, 1 + ma] = rng.integers(0, 1 << ma, n)
    y = rng.integers(0, 2, n).astype(np.float64)
    return theta, feat, y, nsym, ma, hidden


def test_gradient_matches_finite_differences():
    for seed in range(3):
        theta, feat, y, nsym, ma, h = _rand(seed=seed)
        for pw in (1.0, 3.0):
            g = mlp.grad(theta, feat, y, nsym, ma, h, pw)
            eps = 1e-6
            num = np.zeros_like(theta)
            for i in range(len(theta)):
                tp, tm = theta.copy(), theta.copy()
                tp[i] += eps
                tm[i] -= eps
                num[i] = (mlp.loss(tp, feat, y, nsym, ma, h, pw) -
                          mlp.loss(tm, feat, y, nsym, ma, h, pw)) / (2 * eps)
            assert np.max(np.abs(num - g)) < 1e-7 * max(1.0, np.max(np.abs(g))) + 1e-9


def test_tiny_network_by_hand():
    # nsym=2, ma=1, hidden=1: D = 2*2+1 = 5; x = [oh(h) (2), oh(a0) (2), b0]
    nsym, ma, h = 2, 1, 1
    W1 = np.array([[0.5, -1.0, 2.0, 0.25, 1.5]])
    b1 = np.array([0.1])
    W2 = np.array([[2.0]])
    b2 = np.array([-0.3])
    w3 = np.array([1.5])
    b3 = 0.2
    theta = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, [b3]])
    feat = np.array([[1, 0, 1]])          # h=1, a0=0, b0=1
    # z1 = W1[1] + W1[2+0] + W1[4] + b1 = -1 + 2 + 1.5 + 0.1 = 2.6
    # h2 = relu(2*2.6 - 0.3) = 4.9; z = 1.5*4.9 + 0.2 = 7.55
    z, _ = mlp.forward(theta, feat, nsym, ma, h)
    assert abs(z[0] - 7.55) < 1e-12
    feat2 = np.array([[0, 1, 0]])         # z1 = 0.5 + 0.25 + 0.1 = 0.85, h2 = 1.4
    z2, _ = mlp.forward(theta, feat2, nsym, ma, h)
    assert abs(z2[0] - (1.5 * 1.4 + 0.2)) < 1e-12
    # loss of label 1 at z: log(1 + exp(-z))
    assert abs(mlp.loss(theta, feat, [1.0], nsym, ma, h) - np.log1p(np.exp(-7.55))) < 1e-12


def test_adam_scalar():
    th, m, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    g = np.array([0.5])
    th1, m1, v1 = mlp.adam_step(th, g, m, v, 1, lr=0.1)
    # first step: m_hat = g, v_hat = g^2, update = lr * g / (|g| + eps)
    assert abs(th1[0] - (1.0 - 0.1 * 0.5 / (0.5 + 1e-8))) < 1e-12
    assert abs(m1[0] - 0.05) < 1e-15 and abs(v1[0] - 0.00025) < 1e-15


def test_planted_sign_error_is_caught():
    """A gradient with a flipped sign in one block fails the finite-difference pin."""
    theta, feat, y, nsym, ma, h = _rand(seed=5)
    g = mlp.grad(theta, feat, y, nsym, ma, h)
    d, sizes = mlp.dims(nsym, ma, h)
    bad = g.copy()
    at = sizes[0] + sizes[1]
    bad[at:at + sizes[2]] *= -1          # dW2 with the wrong sign
    eps = 1e-6
    i = at + int(np.argmax(np.abs(g[at:at + sizes[2]])))
    tp, tm = theta.copy(), theta.copy()
    tp[i] += eps
    tm[i] -= eps
    num = (mlp.loss(tp, feat, y, nsym, ma, h) - mlp.loss(tm, feat, y, nsym, ma, h)) / (2 * eps)
    assert abs(num - g[i]) < 1e-6 and abs(num - bad[i]) > 1e-6
