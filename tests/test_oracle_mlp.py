"""The FP64 reference of the proposer network: its analytic gradient
against central finite differences of its loss (a pin independent of the
back-propagation code), and the forward pass against an explicit
per-sample evaluation of the formula."""
import numpy as np

from oracle import mlp as omlp


def _setup(n_in=5, H=7, n=13, seed=0):
    rng = np.random.default_rng(seed)
    npar = H * n_in + H + H * H + H + H + 1
    p = rng.normal(0, 0.5, npar)
    X = rng.normal(0, 1, (n, n_in))
    T = rng.normal(0, 1, n)
    return p, X, T, n_in, H


def test_gradient_matches_finite_differences():
    p, X, T, n_in, H = _setup()
    loss, g = omlp.loss_grad(p, X, T, n_in, H)
    h = 1e-6
    fd = np.empty_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (omlp.loss_grad(p + e, X, T, n_in, H)[0] - omlp.loss_grad(p - e, X, T, n_in, H)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))
    assert loss > 0


def test_forward_is_the_formula():
    p, X, T, n_in, H = _setup(seed=3)
    W1, b1, W2, b2, w3, b3 = omlp.unpack(p, n_in, H)
    y, _, _ = omlp.forward(p, X, n_in, H)
    for s in range(X.shape[0]):
        h1 = [np.tanh(sum(W1[j, i] * X[s, i] for i in range(n_in)) + b1[j]) for j in range(H)]
        h2 = [np.tanh(sum(W2[j, i] * h1[i] for i in range(H)) + b2[j]) for j in range(H)]
        ys = sum(w3[j] * h2[j] for j in range(H)) + b3
        assert abs(ys - y[s]) <= 1e-12
