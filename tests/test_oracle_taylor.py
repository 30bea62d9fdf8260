"""The Taylor-moment variant of Algorithm 2 (App. C) in the oracle.

Pins: the remainder bound of Lemma C.1 (reading g4: |z - z_j| <= Lz, bound
1 / (Q! eta^{2Q})); the coefficients A_p(k) (reading g2: |k|^2 in the
exponent) summed as a series in (d/Lz)^2 against the per-mode z-kernel of
Eq. 4.40 they expand; and the variant against the closed form of Eq. 4.40
(long_closed_form) on a confined box where every long-range Gaussian is
wide against Lz, where it must reach the same error floor as the
anterpolation form; on a box with eta < 1/2 its error must stay far above."""
import math

import numpy as np
import pytest

from paper_2412_04595_gb300 import workloads


def _confined(osog, N=400, L=(30.0, 30.0, 1.0)):
    q, r = workloads.uniform_neutral(N, L, 7)
    return osog.select_params(N, *L, 1e-6), q, r


def test_remainder_bound_holds(oracle_mod):
    prm, _, _ = _confined(oracle_mod)
    w, s = oracle_mod.sog_weights(prm["b"], prm["sigma"], prm["omega"], prm["M"])
    Lz = prm["L"][2]
    d = np.linspace(-Lz, Lz, 201)
    for Q in (2, 4, 6, 8):
        worst = 0.0
        for l in range(prm["m"] + 1, prm["M"] + 1):
            x = d * d / s[l] ** 2
            series = sum((-x) ** p / math.factorial(p) for p in range(Q))
            worst = max(worst, float(np.max(np.abs(np.exp(-x) - series))))
        assert worst <= oracle_mod.taylor_remainder_bound(prm, Q) * (1 + 1e-12)
        # and the bound is not vacuous here: within a factor 30 of the worst case
        assert worst >= oracle_mod.taylor_remainder_bound(prm, Q) / 30.0


def test_coefficients_expand_the_kernel(oracle_mod):
    prm, _, _ = _confined(oracle_mod)
    Lz = prm["L"][2]
    k2 = np.array([(2 * math.pi / 30.0) ** 2 * n for n in (1, 2, 5, 13)])
    d = np.linspace(-Lz, Lz, 41)
    A = oracle_mod.taylor_coefficients(prm, k2, 16)          # (Q, modes)
    series = sum(A[p][:, None] * (d[None, :] / Lz) ** (2 * p) for p in range(16))
    exact = oracle_mod.long_kernel(prm, k2[:, None], d[None, :])
    assert np.max(np.abs(series - exact) / np.abs(exact).max(axis=1, keepdims=True)) < 1e-12


def test_confined_box_reaches_the_anterpolation_floor(oracle_mod):
    prm, q, r = _confined(oracle_mod)
    tgt = np.arange(0, q.size, 8)
    cf, _ = oracle_mod.long_closed_form(prm, q, r, tgt, with_k0=False)
    an, _ = oracle_mod.long_range(prm, q, r, tgt)
    scale = np.abs(cf).max()
    e_an = np.abs(an - cf).max() / scale
    errs = []
    for Q in (2, 4, 8, 12):
        ty, _ = oracle_mod.long_range_taylor(prm, q, r, Q, tgt)
        errs.append(np.abs(ty - cf).max() / scale)
    assert errs[0] > errs[1] > errs[2]                        # converges with Q
    assert errs[3] <= 1.5 * e_an + 1e-12                      # down to the same floor
    assert e_an < 1e-6


def test_wide_slab_needs_many_terms(oracle_mod):
    """eta = s_{m+1} / Lz below 1/2: at Q = 8 the variant is still orders of
    magnitude less accurate than the anterpolation form."""
    N, L = 2000, (141.4, 141.4, 10.0)
    q, r = workloads.uniform_neutral(N, L, 7)
    prm = oracle_mod.select_params(N, *L, 1e-6)
    w, s = oracle_mod.sog_weights(prm["b"], prm["sigma"], prm["omega"], prm["M"])
    assert s[prm["m"] + 1] / L[2] < 0.5
    tgt = np.arange(0, N, 40)
    cf, _ = oracle_mod.long_closed_form(prm, q, r, tgt, with_k0=False)
    an, _ = oracle_mod.long_range(prm, q, r, tgt)
    ty, _ = oracle_mod.long_range_taylor(prm, q, r, 8, tgt)
    scale = np.abs(cf).max()
    assert np.abs(ty - cf).max() / scale > 1e3 * np.abs(an - cf).max() / scale
