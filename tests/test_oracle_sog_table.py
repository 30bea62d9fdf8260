"""Pins of the SOG decomposition in the oracle (Sec. 2.2, Table 1)."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")


def table1_rows():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            v = line.split()
            rows.append((float(v[0]), float(v[1]), float(v[2]), float(v[3]), int(v[4])))
    return rows


def test_table1_fixture_matches_oracle_copy(oracle_mod):
    rows = table1_rows()
    assert len(rows) == len(oracle_mod.TABLE1) == 6
    for a, b in zip(rows, oracle_mod.TABLE1):
        assert a[0] == b[0] and a[1] == b[1] and a[2] == b[2] and a[4] == b[4]


@pytest.mark.parametrize("row", table1_rows())
def test_table1_rows_solve_c1_conditions(oracle_mod, row):
    """Every printed (b, r0, omega) satisfies Eq. 2.23 and 2.24 (scaled form
    Eq. 2.35, sigma = 1) to rounding: this pins the weights/bandwidths of
    Eq. 2.22 and the omega scaling of Eq. 2.25."""
    b, r0, om = row[:3]
    f1, f2 = oracle_mod.c1_residuals(b, r0, om)
    assert abs(f1) < 5e-14 and abs(f2) < 5e-14
    # sensitivity: a wrong omega is seen at once (r0 is ill-conditioned:
    # r F(r) stays within rounding of 1 over a range of r for small b)
    if b > 1.3:
        g1, g2 = oracle_mod.c1_residuals(b, r0, om * (1 + 1e-3))
        assert max(abs(g1), abs(g2)) > 1e-9


def test_newton_recovers_table1_from_nearby_start(oracle_mod):
    b, r0, om = table1_rows()[0][:3]
    r, o = oracle_mod.solve_r0_omega(b, r0 * 1.01, om * 0.999)
    assert abs(r - r0) < 1e-12 and abs(o - om) < 1e-12


@pytest.mark.parametrize("b", [2.0, 1.62976708826776469, 1.48783512395703226])
def test_bilateral_series_pointwise_error_bound(oracle_mod, b):
    """Eq. 2.17 / 2.18: the bilateral sum over all l (negative l included) has
    relative error below about 2 sqrt(2) exp(-pi^2/(2 log b)) for all r; the
    oracle's weights for l >= 0 (Eq. 2.22) are its l >= 0 part."""
    sigma = 0.7
    w, s = oracle_mod.sog_weights(b, sigma, 1.0, 400)
    lneg = np.arange(1, 400)
    wn = (math.pi / 2) ** -0.5 * b ** lneg / sigma * math.log(b)     # l = -1, -2, ...
    sn = math.sqrt(2) * b ** (-lneg) * sigma
    bound = 2 * math.sqrt(2) * math.exp(-math.pi**2 / (2 * math.log(b)))
    for r in np.geomspace(1e-2, 1e3, 60):
        tot = math.fsum(w * np.exp(-(r / s) ** 2)) + math.fsum(wn * np.exp(-(r / sn) ** 2))
        err = abs(1 - r * tot)
        assert err <= 1.05 * bound
    assert bound < 0.1


def test_truncated_kernel_continuity_at_cutoff(oracle_mod):
    """With the Table 1 row and sigma = rc/r0, the near kernel 1/r - F_M(r)
    and its derivative vanish at r = rc up to the dropped tail l > M."""
    b, r0, om, _, M = table1_rows()[3]
    rc = 3.0
    sigma = rc / r0
    w, s = oracle_mod.sog_weights(b, sigma, om, M)
    G = 1 / rc - np.sum(w * np.exp(-(rc / s) ** 2))
    dG = -1 / rc**2 + np.sum(2 * rc / s**2 * w * np.exp(-(rc / s) ** 2))
    wt, st = oracle_mod.sog_weights(b, sigma, om, M + 2000)
    tail = np.sum(wt[M + 1:])
    assert abs(G) <= 1.01 * tail + 1e-15
    assert abs(dG) < 1e-12
    assert tail < 1e-9
