"""End-to-end pins of the SOG oracle: against Ewald2D (the paper's reference,
Sec. 5) within the tolerance, and invariants the discrete scheme must keep."""
import math

import numpy as np
import pytest

from tests.conftest import uniform_system

L0 = (10.0, 10.0, 10.0)


@pytest.fixture(scope="module")
def sys300(oracle_mod):
    q, r = uniform_system(300, L0, 5)
    pe, ge = oracle_mod.ewald2d(q, r, L0)
    return q, r, pe, ge


def errors(out, q, pe, ge):
    Ee = 0.5 * math.fsum(q * pe)
    relE = abs(out["E"] - Ee) / abs(Ee)
    linf = np.max(np.abs(out["phi"] - pe)) / np.max(np.abs(pe))
    rmsF = math.sqrt(np.mean(np.sum((out["grad"] - ge) ** 2, 1)) / np.mean(np.sum(ge**2, 1)))
    return relE, linf, rmsF


@pytest.mark.parametrize("tol,bounds", [(1e-4, (1e-4, 5e-4, 1e-3)), (1e-6, (1e-6, 3e-6, 1e-5)),
                                        (1e-8, (1e-8, 3e-8, 1e-7))])
def test_sog_vs_ewald2d(oracle_mod, sys300, tol, bounds):
    q, r, pe, ge = sys300
    prm = oracle_mod.select_params(q.size, *L0, tol, n_nb=60)
    out = oracle_mod.sog_eval(prm, q, r)
    relE, linf, rmsF = errors(out, q, pe, ge)
    assert relE <= bounds[0] and linf <= bounds[1] and rmsF <= bounds[2], (relE, linf, rmsF)


def test_thin_slab_all_long_range(oracle_mod):
    """A box 12 x 12 x 1: the split sends most Gaussians to the long range
    (Remark 3.3); still within tolerance of Ewald2D."""
    L = (12.0, 12.0, 1.0)
    q, r = uniform_system(150, L, 8)
    pe, ge = oracle_mod.ewald2d(q, r, L)
    prm = oracle_mod.select_params(q.size, *L, 1e-6, n_nb=40)
    out = oracle_mod.sog_eval(prm, q, r)
    relE, linf, rmsF = errors(out, q, pe, ge)
    assert relE <= 1e-6 and linf <= 3e-6 and rmsF <= 1e-5, (relE, linf, rmsF, prm["m"])


def test_forces_are_energy_gradient(oracle_mod):
    """F_i = -dU/dr_i of the discrete scheme (spread = gather transpose)."""
    L = (6.0, 6.0, 6.0)
    q, r = uniform_system(40, L, 9)
    prm = oracle_mod.select_params(q.size, *L, 1e-6, n_nb=15)
    out = oracle_mod.sog_eval(prm, q, r)
    d = 1e-5
    for i in (0, 3, 17):
        for ax in range(3):
            rp, rm = r.copy(), r.copy()
            rp[i, ax] += d
            rm[i, ax] -= d
            g = -(oracle_mod.sog_eval(prm, q, rp)["E"] - oracle_mod.sog_eval(prm, q, rm)["E"]) / (2 * d)
            assert abs(g - out["F"][i, ax]) < 2e-6 * max(1.0, abs(out["F"][i, ax]))


def test_invariants(oracle_mod):
    L = (8.0, 7.0, 6.0)
    q, r = uniform_system(120, L, 12)
    prm = oracle_mod.select_params(q.size, *L, 1e-6, n_nb=30)
    base = oracle_mod.sog_eval(prm, q, r)
    # zero net force to the scheme's accuracy
    assert np.max(np.abs(base["F"].sum(0))) < 1e-5 * np.max(np.abs(base["F"]))
    # permutation equivariance
    perm = np.random.default_rng(0).permutation(q.size)
    o = oracle_mod.sog_eval(prm, q[perm], r[perm])
    assert np.allclose(o["phi"], base["phi"][perm], atol=1e-12)
    # translation in x,y by whole mid and long grid cells: exact
    Ix, Iy, _ = prm["I"]
    Ilx, Ily = prm["I_long"]
    sx = L[0] / math.gcd(Ix, Ilx) * 1.0
    rs = r.copy()
    rs[:, 0] = (rs[:, 0] + sx + L[0] / 2) % L[0] - L[0] / 2
    o = oracle_mod.sog_eval(prm, q, rs)
    assert np.allclose(o["phi"], base["phi"], atol=1e-11)
    # arbitrary translation in x,y: equal to the scheme's accuracy
    rs = r.copy()
    rs[:, 0] = (rs[:, 0] + 0.377 + L[0] / 2) % L[0] - L[0] / 2
    rs[:, 1] = (rs[:, 1] - 1.21 + L[1] / 2) % L[1] - L[1] / 2
    o = oracle_mod.sog_eval(prm, q, rs)
    assert np.max(np.abs(o["phi"] - base["phi"])) < 3e-6 * np.max(np.abs(base["phi"]))
    # linearity in the charges
    o = oracle_mod.sog_eval(prm, 2.0 * q, r)
    assert np.allclose(o["phi"], 2.0 * base["phi"], atol=1e-12)
    # mirror z -> -z: Phi unchanged, F_z flips
    rm = r * np.array([1.0, 1.0, -1.0])
    o = oracle_mod.sog_eval(prm, q, rm)
    assert np.allclose(o["phi"], base["phi"], atol=1e-9)
    assert np.allclose(o["F"][:, 2], -base["F"][:, 2], atol=1e-8)


def test_length_scaling(oracle_mod):
    """Phi has units 1/length: scaling positions, box, r_c and hz by s (grid
    sizes kept) scales every potential by 1/s and every force by 1/s^2."""
    L = (8.0, 7.0, 6.0)
    q, r = uniform_system(80, L, 13)
    prm = oracle_mod.select_params(q.size, *L, 1e-6, n_nb=25)
    base = oracle_mod.sog_eval(prm, q, r)
    s = 2.5
    p2 = dict(prm, L=tuple(s * x for x in L), rc=s * prm["rc"], sigma=s * prm["sigma"], hz=s * prm["hz"])
    o = oracle_mod.sog_eval(p2, q, s * r)
    assert np.allclose(o["phi"] * s, base["phi"], rtol=0, atol=1e-11)
    assert np.allclose(o["F"] * s * s, base["F"], rtol=0, atol=1e-10)
