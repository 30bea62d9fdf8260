"""Pins of the oracle's spectral steps against plain definitions.

* Algorithm 1 (windowed, FFT) vs the direct Fourier sum over the same modes
  (differ by window error, Theorems 4.3 / 4.4);
* the direct Fourier sum vs the real-space Gaussian image sum (differ by
  Fourier truncation and z-padding, Theorems 4.2 / 4.4);
* Algorithm 2 + the k = 0 mode vs the closed form Eq. 4.40;
* Chebyshev interpolation of a Gaussian vs the bound of Theorem 3.1;
* window Fourier transforms vs a fine Riemann sum (Poisson summation).
"""
import math

import numpy as np
import pytest

from tests.conftest import uniform_system


@pytest.fixture(scope="module")
def sysA(oracle_mod):
    L = (10.0, 10.0, 10.0)
    q, r = uniform_system(200, L, 11)
    prm = oracle_mod.select_params(200, *L, 1e-6, n_nb=60)
    return q, r, L, prm


def test_mid_window_vs_direct_fourier(oracle_mod, sysA):
    q, r, L, prm = sysA
    pa, ga = oracle_mod.mid_direct_fourier(prm, q, r)
    scale = np.max(np.abs(pa))
    p = dict(prm, P_win=14, shape=1.9 * 14)
    pm, gm = oracle_mod.mid_range(p, q, r)
    assert np.max(np.abs(pm - pa)) < 3e-7 * scale
    assert np.max(np.abs(gm - ga)) < 3e-6 * scale
    # the error falls with the support, as Theorem 4.3 says
    errs = []
    for P in (6, 9, 12):
        pm, _ = oracle_mod.mid_range(dict(prm, P_win=P, shape=1.9 * P), q, r)
        errs.append(np.max(np.abs(pm - pa)))
    assert errs[0] > errs[1] > errs[2]
    # Gaussian window (Eq. 4.7, closed-form transform) converges as well
    pg, _ = oracle_mod.mid_range(dict(prm, window="gauss", P_win=16, shape=0.455 * math.pi * 16), q, r)
    assert np.max(np.abs(pg - pa)) < 1e-5 * scale
    # and the Kaiser-Bessel window (closed-form transform), like ES for the same P
    errs = []
    for P in (6, 9, 12, 14):
        pk, gk = oracle_mod.mid_range(dict(prm, window="kb", P_win=P, shape=2.0 * P), q, r)
        errs.append(np.max(np.abs(pk - pa)))
    assert errs[0] > errs[1] > errs[2] and errs[3] < 3e-7 * scale
    assert np.max(np.abs(gk - ga)) < 3e-6 * scale


def test_mid_direct_fourier_vs_real_space(oracle_mod, sysA):
    q, r, L, prm = sysA
    pa, ga = oracle_mod.mid_direct_fourier(prm, q, r)
    w, s = oracle_mod.sog_weights(prm["b"], prm["sigma"], prm["omega"], prm["M"])
    m = prm["m"]
    pb, gb = oracle_mod.gauss_images(q, r, L, w[:m + 1], s[:m + 1])
    scale = np.max(np.abs(pb))
    assert np.max(np.abs(pa - pb)) < 1e-7 * scale
    assert np.max(np.abs(ga - gb)) < 1e-6 * scale


def test_long_range_vs_closed_form(oracle_mod, sysA):
    q, r, L, prm = sysA
    pc, gc = oracle_mod.long_closed_form(prm, q, r, with_k0=False)
    pl, gl = oracle_mod.long_range(dict(prm, P_cheb=24, P_long=12, shape_long=1.9 * 12,
                                        I_long=(24, 24)), q, r)
    scale = np.max(np.abs(pc))
    assert np.max(np.abs(pl - pc)) < 1e-7 * scale
    assert np.max(np.abs(gl - gc)) < 1e-6 * scale


def test_long_range_direct_vs_closed_form(oracle_mod, sysA):
    """Algorithm 3 (direct Fourier sums, no window): with enough modes and
    Chebyshev points it reproduces Eq. 4.40 summed directly; with a cut at
    the selection's K_max it stays within the tolerance."""
    q, r, L, prm = sysA
    pc, gc = oracle_mod.long_closed_form(prm, q, r, with_k0=False)
    scale = np.max(np.abs(pc))
    pd, gd = oracle_mod.long_range_direct(dict(prm, P_cheb=24, I_long=(41, 41)), q, r)
    assert np.max(np.abs(pd - pc)) < 1e-10 * scale
    assert np.max(np.abs(gd - gc)) < 1e-9 * scale
    pg, gg = oracle_mod.long_range(dict(prm, P_cheb=24, P_long=12, shape_long=1.9 * 12,
                                        I_long=(24, 24)), q, r)
    assert np.max(np.abs(pd - pg)) < 1e-7 * scale


def test_long_k0_vs_closed_form(oracle_mod, sysA):
    q, r, L, prm = sysA
    pc, gc = oracle_mod.long_closed_form(prm, q, r, with_k0=True)
    pc1, gc1 = oracle_mod.long_closed_form(prm, q, r, with_k0=False)
    p0, g0 = oracle_mod.long_k0(dict(prm, P_cheb=24), q, r)
    scale = np.max(np.abs(pc - pc1))
    assert np.max(np.abs(p0 - (pc - pc1))) < 1e-10 * max(scale, 1.0)
    assert np.max(np.abs(g0 - (gc - gc1))) < 1e-9 * max(scale, 1.0)


@pytest.mark.parametrize("eta,P", [(0.5, 8), (0.5, 14), (1.0, 6), (1.0, 10), (0.3, 16)])
def test_chebyshev_interpolation_bound(oracle_mod, eta, P):
    """Theorem 3.1: |e^{-z^2/s^2} - interpolant| <= 1/(sqrt(P!) (2 sqrt2 eta)^P)
    on [-Lz/2, Lz/2] for s >= eta Lz (checked for s = eta Lz, shifted too).
    READING: the interpolation form of Eq. 3.2 carries a factor 2 (the node
    polynomial of P first-kind points is bounded by 2^(1-P)), so the bound is
    checked with that factor."""
    Lz = 7.0
    s = eta * Lz
    zc = oracle_mod.cheb_nodes(P, Lz)
    z = np.linspace(-Lz / 2, Lz / 2, 2001)
    Lt, _ = oracle_mod.lagrange(zc, z)
    bound = 1.0 / (math.sqrt(math.factorial(P)) * (2 * math.sqrt(2) * eta) ** P)
    for shift in (0.0, 0.3 * Lz, -0.5 * Lz):
        f = lambda x: np.exp(-((x - shift) / s) ** 2)
        err = np.max(np.abs(Lt @ f(zc) - f(z)))
        assert err <= 2.0 * bound * 1.0001 + 1e-15


def test_lagrange_basis_properties(oracle_mod):
    P, Lz = 9, 4.0
    zc = oracle_mod.cheb_nodes(P, Lz)
    assert np.allclose(np.sort(zc), np.sort(-zc), atol=1e-15)
    z = np.concatenate([np.linspace(-2, 2, 37), zc[:2]])
    Lt, dLt = oracle_mod.lagrange(zc, z)
    assert np.allclose(Lt.sum(1), 1.0, atol=1e-13)          # partition of unity
    assert np.allclose(dLt.sum(1), 0.0, atol=1e-11)
    poly = lambda x: 0.3 - x + 0.2 * x**3 - 0.01 * x**7     # degree < P: exact
    dpoly = lambda x: -1 + 0.6 * x**2 - 0.07 * x**6
    assert np.allclose(Lt @ poly(zc), poly(z), atol=1e-12)
    assert np.allclose(dLt @ poly(zc), dpoly(z), atol=1e-10)


@pytest.mark.parametrize("kind,P", [("es", 10), ("es", 7), ("gauss", 12), ("kb", 10), ("kb", 7)])
def test_window_transform_vs_riemann_sum(oracle_mod, kind, P):
    """Poisson summation: h sum_g W(g h) e^{-i k g h} = sum_n hatW(k + 2 pi n/h);
    with h = H/4000 the aliases are negligible, so the sum is hatW(k)."""
    win = oracle_mod.make_window(kind, P)
    H = 1.7
    h = H / 4000.0
    x = np.arange(-4000, 4001) * h
    Wx = win.phi(x / H)
    for k in (0.0, 0.9, 2.5, 6.0):
        riem = h * np.sum(Wx * np.cos(k * x))
        assert abs(riem - win.ft(np.array([k]), H)[0]) < 2e-7 * H
    # derivative of phi vs central differences
    v = np.linspace(-0.95, 0.95, 41)
    d = 1e-6
    assert np.allclose(win.dphi(v), (win.phi(v + d) - win.phi(v - d)) / (2 * d), atol=1e-6)


@pytest.mark.parametrize("window", ["es", "kb", "gauss"])
def test_selected_window_meets_the_tolerance(oracle_mod, sysA, window):
    """With the support and shape the selection picks for tol = 1e-6, the
    windowed mid range (Algorithm 1) stays within the tolerance of the
    direct Fourier sum over the same modes."""
    q, r, L, prm = sysA
    pw = oracle_mod.select_params(200, *L, 1e-6, n_nb=60, window=window)
    p = dict(prm, window=window, P_win=pw["P_win"], shape=pw["shape"])
    pa, _ = oracle_mod.mid_direct_fourier(p, q, r)
    pm, _ = oracle_mod.mid_range(p, q, r)
    assert np.max(np.abs(pm - pa)) < 1e-6 * np.max(np.abs(pa)), (window, pw["P_win"])
