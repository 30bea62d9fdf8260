"""Polynomial windows in the oracle (Sec. 3.4, 5.1: the window evaluated
through Chebyshev interpolants of order nu).

Pins against the exact windows, which are pinned by their Fourier transforms
elsewhere: the per-point polynomials reproduce the window to the accuracy
that Chebyshev interpolation of an analytic function reaches (falling with nu,
small against the tolerances they serve), their derivatives are the
derivatives of the same polynomials (central differences) and approximate the
window's derivative away from the support edge, and an evaluation with
polynomial windows differs from the exact-window one by far less than the
tolerance."""
import numpy as np
import pytest

from paper_2412_04595_gb300 import workloads


def _t(n=4000, seed=0):
    return np.random.default_rng(seed).uniform(-50.0, 50.0, n)


@pytest.mark.parametrize("kind", ["es", "kb", "gauss"])
def test_polynomials_reproduce_the_window(oracle_mod, kind):
    t = _t()
    for P, nu, bound in ((9, 10, 2e-7), (12, 10, 1e-8), (16, 10, 1e-9)):
        ex = oracle_mod.make_window(kind, P)
        po = oracle_mod.make_window(kind, P, nu=nu)
        g1, w1, _ = ex.weights(t)
        g2, w2, _ = po.weights(t)
        assert np.array_equal(g1, g2)
        assert np.max(np.abs(w2 - w1)) < bound, (kind, P, nu, np.max(np.abs(w2 - w1)))


def test_error_falls_with_the_degree(oracle_mod):
    t = _t()
    _, w_ex, _ = oracle_mod.make_window("es", 16).weights(t)
    errs = [np.max(np.abs(oracle_mod.make_window("es", 16, nu=nu).weights(t)[1] - w_ex))
            for nu in (4, 6, 8, 10)]
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 1e-10


def test_derivatives(oracle_mod):
    po = oracle_mod.make_window("es", 12, nu=10)
    ex = oracle_mod.make_window("es", 12)
    t = _t(500, 1)
    h = 1e-6
    _, wp, _ = po.weights(t + h)
    _, wm, _ = po.weights(t - h)
    _, _, d = po.weights(t)
    # the same support for t +- h (no particle within h of a support change)
    gp = po.weights(t + h)[0]
    gm = po.weights(t - h)[0]
    same = np.all(gp == gm, axis=1)
    fd = (wp - wm) / (2 * h)
    assert np.max(np.abs(fd[same] - d[same])) < 1e-6 * np.max(np.abs(d))
    # and d/dt of the exact window, away from the edge point of the support
    _, _, dex = ex.weights(t)
    assert np.max(np.abs(d[:, 1:-1] - dex[:, 1:-1])) < 1e-6 * np.max(np.abs(dex))


@pytest.mark.parametrize("L", [(10.0, 10.0, 10.0), (24.0, 24.0, 2.0)])
def test_evaluation_with_polynomial_windows(oracle_mod, L):
    N = 600
    q, r = workloads.uniform_neutral(N, L, 5)
    prm = oracle_mod.select_params(N, *L, 1e-6, n_nb=40)
    ref = oracle_mod.sog_eval(prm, q, r)
    pp = dict(prm, win_poly=10)
    out = oracle_mod.sog_eval(pp, q, r)
    assert abs(out["E"] - ref["E"]) < 1e-7 * abs(ref["E"])
    scale = np.sqrt(np.mean(np.sum(ref["F"] ** 2, 1)))
    assert np.sqrt(np.mean(np.sum((out["F"] - ref["F"]) ** 2, 1))) < 1e-6 * scale
