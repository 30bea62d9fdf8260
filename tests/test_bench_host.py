"""Host logic of bench.py that feeds the reported roofline: the near field's
candidate and pair counts on the actual positions (the numerator of the
near field's FP32 work), checked against brute force on small systems, and
the stage work formulas."""
import math

import numpy as np
import pytest

import bench
from paper_2412_04595_gb300 import workloads

pytest.importorskip("scipy")


def _brute(prm, r):
    """Pairs within r_c (minimum image in x, y) per charge, and the
    candidate tests of the 27-cell (or fewer) neighbourhoods, by loops."""
    L, rc = prm["L"], prm["rc"]
    N = r.shape[0]
    d = r[:, None, :] - r[None, :, :]
    for k in (0, 1):
        d[:, :, k] -= L[k] * np.round(d[:, :, k] / L[k])
    r2 = np.sum(d * d, axis=2)
    np.fill_diagonal(r2, np.inf)
    pairs = np.sum(r2 < rc * rc)
    nc = [max(1, int(math.floor(L[k] / rc))) for k in range(3)]
    pos = r + 0.5 * np.array(L)
    cell = np.stack([np.minimum((np.mod(pos[:, k], L[k]) if k < 2 else np.clip(pos[:, k], 0, L[k]))
                                * nc[k] / L[k], nc[k] - 1).astype(int) for k in range(3)], 1)
    cand = 0
    for i in range(N):
        ok = np.ones(N, dtype=bool)
        for k in range(3):
            dc = cell[:, k] - cell[i, k]
            if k < 2 and nc[k] >= 3:
                dc = (dc + 1) % nc[k] - 1        # periodic neighbour offsets -1, 0, 1
                ok &= np.abs(dc) <= 1
            elif k == 2:
                ok &= np.abs(dc) <= 1
        cand += np.sum(ok)
    return pairs, cand


@pytest.mark.parametrize("L", [(12.0, 12.0, 12.0), (30.0, 30.0, 4.0), (8.0, 8.0, 40.0)])
def test_near_counts_match_brute_force(oracle_mod, L):
    N = 600
    q, r = workloads.uniform_neutral(N, L, 3)
    prm = oracle_mod.select_params(N, *L, 1e-6, n_nb=40)
    c = bench.near_counts(prm, r, samples=N)
    pairs, cand = _brute(prm, r)
    assert c["pairs"] == pytest.approx(pairs, rel=1e-12)
    assert c["cand"] == pytest.approx(cand, rel=1e-12)


def test_near_work_uses_the_counts(oracle_mod):
    N, L = 600, (12.0, 12.0, 12.0)
    prm = oracle_mod.select_params(N, *L, 1e-6, n_nb=40)
    bound, work, desc = bench.stage_work(prm, N, "near", 4, {"cand": 1000.0, "pairs": 100.0})
    assert bound == "alu" and work == 1000.0 * bench.CAND_FLOP + 100.0 * bench.PAIR_FLOP
    assert "counted on the positions" in desc
