"""The high-aspect-ratio and nonuniform workloads at full size: a thin slab
1000 x 1000 x 10 and a tall cell 50 x 50 x 2000 with 1e6 charges (tol 1e-6),
and an electric double layer 400 x 400 x 100 with 4e6 charges (tol 1e-5).

Each is compared element by element with the FP64 oracle on sampled targets
(the oracle's near field, mid range, long range and k = 0 mode all take a
target subset; the grids are built from every charge, so the full-size FFT
and tile paths are the ones checked): FP64 plans to 1e-10, mixed plans to
1e-5.  The method's own error is checked against Ewald2D (the paper's
reference, Sec. 5) on a few targets with the paper's measure, the largest
potential error relative to the largest potential.  Scaled down to 2e4
charges, both plans are compared with the oracle on every particle."""
import math

import numpy as np
import pytest

from paper_2412_04595_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CONFIGS = {
    "slab": (1000000, (1000.0, 1000.0, 10.0), 1e-6, "uniform"),
    "tall": (1000000, (50.0, 50.0, 2000.0), 1e-6, "uniform"),
    "edl": (4000000, (400.0, 400.0, 100.0), 1e-5, "edl"),
}
N_SAMPLE = 2000      # targets compared with the oracle
N_TRUTH = 16         # targets compared with Ewald2D (about 5 core-seconds each at N = 1e6)


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_2412_04595_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding


def _system(kind, N, L, seed):
    gen = workloads.uniform_neutral if kind == "uniform" else workloads.edl_neutral
    return gen(N, L, seed, dtype=np.float32)


def _run(B, N, L, tol, q, r, prec, manual=None):
    dev = torch.device("cuda:0")
    dt = torch.float64 if prec == B.SOG_PREC_FP64 else torch.float32
    plan = B.Plan(N, L, tol, precision=prec, manual=manual)
    qt = torch.tensor(q, dtype=dt, device=dev)
    rt = torch.tensor(r, dtype=dt, device=dev)
    phi = torch.empty(N, dtype=dt, device=dev)
    F = torch.empty(N, 3, dtype=dt, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    plan.eval(qt, rt, phi, E, F)
    torch.cuda.synchronize()
    st = plan.check()
    prm = plan.params
    plan.close()
    return dict(st=st, E=E.item(), F=F.double().cpu().numpy(), phi=phi.double().cpu().numpy(),
                prm=prm)


def _rms(a, b):
    return math.sqrt(np.mean(np.sum((a - b) ** 2, 1)) / np.mean(np.sum(b ** 2, 1)))


def _targets(r, n, seed):
    """n random targets plus the particles nearest the two walls and the box
    corners in x, y (where the wrap and the z clamping act)."""
    N = r.shape[0]
    rng = np.random.default_rng(seed)
    pick = set(rng.choice(N, n, replace=False).tolist())
    for col in (0, 1, 2):
        pick.update(np.argsort(r[:, col])[:4].tolist())
        pick.update(np.argsort(r[:, col])[-4:].tolist())
    return np.array(sorted(pick), dtype=np.int64)


@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_full_size_vs_oracle_sampled(B, oracle_mod, name):
    N, L, tol, kind = CONFIGS[name]
    q, r = _system(kind, N, L, 3)
    f64 = _run(B, N, L, tol, q, r, B.SOG_PREC_FP64)
    mix = _run(B, N, L, tol, q, r, B.SOG_PREC_MIXED, manual=f64["prm"])
    assert f64["st"] == 0 and mix["st"] == 0
    q64, r64 = q.astype(np.float64), r.astype(np.float64)
    tgt = _targets(r64, N_SAMPLE, 7)
    ref = oracle_mod.sog_eval(f64["prm"], q64, r64, tgt)
    scale = np.max(np.abs(ref["phi"]))
    for res, bound in ((f64, 1e-10), (mix, 1e-5)):
        err_phi = np.max(np.abs(res["phi"][tgt] - ref["phi"])) / scale
        err_F = _rms(res["F"][tgt], ref["F"])
        assert err_phi <= bound and err_F <= bound, (name, bound, err_phi, err_F)
    # the net force vanishes up to the method's error: far below the sum of
    # N forces of random direction
    Fs = f64["F"]
    assert np.abs(Fs.sum(0)).max() <= 1e-3 * math.sqrt(N * np.mean(np.sum(Fs ** 2, 1)))
    # the method against the true quasi-2D sum (Ewald2D) with the paper's
    # measure; alpha = 1.5 / min(Lx, Ly) keeps each pair's mode and image sums
    # short (the sum does not depend on alpha)
    tt = tgt[:: max(1, tgt.size // N_TRUTH)][:N_TRUTH]
    ph_true, _ = oracle_mod.ewald2d(q64, r64, L, tt, alpha=1.5 / min(L[0], L[1]))
    err_true = np.max(np.abs(mix["phi"][tt] - ph_true)) / np.max(np.abs(ph_true))
    assert err_true <= 3 * tol, (name, err_true)


@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_scaled_down_vs_oracle(B, oracle_mod, name):
    N0, L0, tol, kind = CONFIGS[name]
    N = 20000
    f = (N / N0) ** 0.5 if name != "tall" else (N / N0) ** (1.0 / 3.0)
    # slab and double layer keep their height (the z structure), the tall
    # cell keeps its aspect ratio
    L = (L0[0] * f, L0[1] * f, L0[2] if name != "tall" else L0[2] * f)
    q, r = _system(kind, N, L, 5)
    f64 = _run(B, N, L, tol, q, r, B.SOG_PREC_FP64)
    ref = oracle_mod.sog_eval(f64["prm"], q.astype(np.float64), r.astype(np.float64))
    assert f64["st"] == 0
    assert abs(f64["E"] - ref["E"]) <= 1e-10 * abs(ref["E"])
    assert _rms(f64["F"], ref["F"]) <= 1e-10
    mix = _run(B, N, L, tol, q, r, B.SOG_PREC_MIXED, manual=f64["prm"])
    assert mix["st"] == 0
    assert abs(mix["E"] - ref["E"]) <= 1e-5 * abs(ref["E"])
    assert _rms(mix["F"], ref["F"]) <= 1e-5
