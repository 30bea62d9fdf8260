"""Pins of the Ewald2D reference (Eq. 2.6 and its far-z limit, Eq. 2.5)."""
import math

import numpy as np


def small_system(seed, N=6, L=(3.0, 4.0, 2.0)):
    rng = np.random.default_rng(seed)
    r = np.column_stack([rng.uniform(-L[i] / 2, L[i] / 2, N) for i in range(3)])
    q = np.array([1.0, -1.0, 1.0, -1.0, 0.5, -0.5])[:N]
    return q, r, L


def test_alpha_independence(oracle_mod):
    q, r, L = small_system(1)
    ref, gref = oracle_mod.ewald2d(q, r, L, alpha=1.5)
    for a in (0.9, 2.6):
        p, g = oracle_mod.ewald2d(q, r, L, alpha=a)
        assert np.max(np.abs(p - ref)) < 1e-13 * np.max(np.abs(ref))
        assert np.max(np.abs(g - gref)) < 1e-12 * np.max(np.abs(gref))


def test_matches_brute_force_image_sum(oracle_mod):
    """Eq. 2.6 summed over squares of images of half-side R = 200, 400, 800,
    Richardson-extrapolated for an a/R + b/R^2 truncation error."""
    q, r, L = small_system(2)
    p = [oracle_mod.brute_images(q, r, L, R) for R in (200, 400, 800)]
    r1, r2 = 2 * p[1] - p[0], 2 * p[2] - p[1]
    extrap = (4 * r2 - r1) / 3
    ref, _ = oracle_mod.ewald2d(q, r, L)
    assert np.max(np.abs(extrap - ref)) < 2e-8
    # the unextrapolated sums approach it from one side at rate 1/R
    assert np.max(np.abs(p[2] - ref)) < np.max(np.abs(p[0] - ref))


def test_far_z_limit(oracle_mod):
    """Eq. 2.5: Phi -> +-(2 pi/(Lx Ly)) sum_j q_j z_j as z -> +-infinity."""
    q, r, L = small_system(3)
    A = L[0] * L[1]
    lim = 2 * math.pi / A * np.sum(q * r[:, 2])
    pts = np.array([[0.3, -0.2, 60.0], [-1.0, 1.1, 90.0], [0.3, -0.2, -60.0], [0.7, 0.0, -90.0]])
    p, g = oracle_mod.ewald2d_at(pts, q, r, L)
    assert np.allclose(p[:2], lim, rtol=0, atol=1e-12)
    assert np.allclose(p[2:], -lim, rtol=0, atol=1e-12)
    assert np.max(np.abs(g)) < 1e-12


def test_zero_net_force_and_energy_gradient(oracle_mod):
    rng = np.random.default_rng(4)
    N, L = 40, (5.0, 6.0, 4.0)
    r = np.column_stack([rng.uniform(-L[i] / 2, L[i] / 2, N) for i in range(3)])
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    p, g = oracle_mod.ewald2d(q, r, L)
    F = -q[:, None] * g
    assert np.max(np.abs(F.sum(0))) < 1e-11 * np.max(np.abs(F))
    # F_i = -dU/dr_i by central differences of U = 1/2 sum q Phi
    d = 1e-5
    for i in (0, 7):
        for ax in range(3):
            rp, rm = r.copy(), r.copy()
            rp[i, ax] += d
            rm[i, ax] -= d
            Up = 0.5 * np.sum(q * oracle_mod.ewald2d(q, rp, L)[0])
            Um = 0.5 * np.sum(q * oracle_mod.ewald2d(q, rm, L)[0])
            assert abs(-(Up - Um) / (2 * d) - F[i, ax]) < 1e-7 * max(1.0, abs(F[i, ax]))


def test_two_charges_far_apart_in_z(oracle_mod):
    """A +1/-1 pair far apart in z: each charge sees the other's periodic sheet
    through the k = 0 term -(2 pi/A) q |z| plus constants, so
    Phi(+) - Phi(-) grows by exactly (4 pi/A) per unit of separation once the
    k != 0 terms (decaying like exp(-2 pi |z|/L)) are negligible."""
    L = (2.0, 2.0, 1.0)
    A = L[0] * L[1]
    q = np.array([1.0, -1.0])
    diffs = []
    for dz in (40.0, 65.0):
        r = np.array([[0.1, 0.2, 0.0], [0.1, 0.2, dz]])
        p, _ = oracle_mod.ewald2d(q, r, L)
        diffs.append(p[0] - p[1])
    assert abs((diffs[1] - diffs[0]) - 4 * math.pi / A * 25.0) < 1e-10
