"""Pins of the warm-start network oracle (oracle/mlp_oracle.py) against closed forms: a
hand-set ReLU network that computes |x| exactly, and the exact gradient of the mean squared
error of a single linear layer."""
import numpy as np

from oracle import mlp_oracle as M


def test_relu_network_computes_abs():
    dims = (2, 4, 2)
    W1 = np.array([[1, 0], [-1, 0], [0, 1], [0, -1]], float)
    W2 = np.array([[1, 1, 0, 0], [0, 0, 1, 1]], float)
    p = np.concatenate([W1.ravel(), np.zeros(4), W2.ravel(), np.zeros(2)])
    assert p.size == M.n_params(dims)
    X = np.random.default_rng(0).normal(size=(50, 2))
    assert np.allclose(M.forward(p, dims, X), np.abs(X), atol=0, rtol=1e-15)
    # standardisation: inputs shifted/scaled, outputs back in target units
    mu, sd = np.array([0.5, -1.0]), np.array([2.0, 0.5])
    out = M.forward(p, dims, X * sd + mu, x_mu=mu, x_sd=sd, y_mu=np.array([3.0, 4.0]), y_sd=np.array([2.0, 2.0]))
    assert np.allclose(out, 2.0 * np.abs(X) + np.array([3.0, 4.0]), rtol=1e-14)


def test_fd_gradient_of_linear_layer_is_exact():
    rng = np.random.default_rng(1)
    dims = (3, 2)
    n = 40
    X, Y = rng.normal(size=(n, 3)), rng.normal(size=(n, 2))
    W, b = rng.normal(size=(2, 3)), rng.normal(size=2)
    p = np.concatenate([W.ravel(), b])
    R = X @ W.T + b - Y
    gW = 2.0 / (n * 2) * R.T @ X
    gb = 2.0 / (n * 2) * R.sum(0)
    g = M.fd_grad(p, dims, X, Y, list(range(p.size)), eps=1e-5)
    assert np.allclose(g, np.concatenate([gW.ravel(), gb]), rtol=1e-8, atol=1e-10)
    assert M.loss(p, dims, X, Y) == np.mean(R ** 2)


def test_zero_loss_at_exact_targets():
    rng = np.random.default_rng(2)
    dims = (4, 5, 3)
    p = rng.normal(size=M.n_params(dims))
    X = rng.normal(size=(10, 4))
    Y = M.forward(p, dims, X)
    assert M.loss(p, dims, X, Y) == 0.0
    assert np.allclose(M.fd_grad(p, dims, X, Y, list(range(0, p.size, 3)), eps=1e-6), 0.0, atol=1e-9)
