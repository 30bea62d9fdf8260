"""Pins of the parameter selection (Sec. 4.3) in the oracle."""
import math

import pytest


def smooth8(n):
    if n % 8:
        return False
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


@pytest.mark.parametrize("N,L,tol", [
    (1000, (10, 10, 10), 1e-6),
    (100000, (100, 100, 100), 1e-6),
    (100000, (100, 100, 100), 1e-4),
    (1000000, (1000, 1000, 10), 1e-6),
    (1000000, (50, 50, 2000), 1e-6),
    (4000000, (400, 400, 100), 1e-5),
])
def test_selection_meets_its_constraints(oracle_mod, N, L, tol):
    prm = oracle_mod.select_params(N, *L, tol)
    Lx, Ly, Lz = L
    rho = N / (Lx * Ly * Lz)
    row = oracle_mod.table1_row_for(tol)
    assert prm["b"] == row[0] and prm["M"] >= row[4]
    assert prm["rc"] <= 0.5 * min(Lx, Ly) + 1e-12
    assert abs(prm["sigma"] * row[1] - prm["rc"]) < 1e-12 * prm["rc"]
    w, s = oracle_mod.sog_weights(prm["b"], prm["sigma"], prm["omega"], prm["M"])
    m = prm["m"]
    assert -1 <= m <= prm["M"]
    if m >= 0:
        Ix, Iy, Izs = prm["I"]
        assert all(smooth8(n) for n in prm["I"])
        eps = 0.3 * tol
        K = 2 * math.sqrt(math.log(1 / eps)) / s[0]
        assert math.pi * Ix / Lx >= K * (1 - 1e-12) and math.pi * Iy / Ly >= K * (1 - 1e-12)
        assert math.pi / prm["hz"] >= K * (1 - 1e-12)
        pad = Izs * prm["hz"] - Lz
        assert pad >= s[m] * math.sqrt(math.log(1 / eps)) - 1e-9
        assert pad >= (prm["P_win"] - 1) * prm["hz"] - 1e-9
    if m < prm["M"]:
        assert prm["P_cheb"] >= 2
        if prm["long_direct"]:
            # Algorithm 3: odd mode counts 2K+1 whose modes cover |k| <= K_long
            # in each direction, at most 256 half-plane modes
            Kl = 2 * math.sqrt(math.log(1 / (0.3 * tol))) / s[m + 1]
            Ix, Iy = prm["I_long"]
            assert Ix % 2 == 1 and Iy % 2 == 1
            Kx, Ky = (Ix - 1) // 2, (Iy - 1) // 2
            assert 2 * math.pi * Kx / Lx >= Kl * (1 - 1e-12)
            assert 2 * math.pi * Ky / Ly >= Kl * (1 - 1e-12)
            assert Ky + Kx * (2 * Ky + 1) <= 256
            assert (Ky + Kx * (2 * Ky + 1)) * prm["P_cheb"] <= 8192
        else:
            assert all(smooth8(n) for n in prm["I_long"])
            assert min(prm["I_long"]) >= prm["P_long"] + 4
