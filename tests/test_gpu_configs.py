"""The high-aspect-ratio and nonuniform workloads: a thin slab 1000 x 1000 x
10 and a tall cell 50 x 50 x 2000 with 1e6 charges (tol 1e-6), and an
electric double layer 400 x 400 x 100 with 4e6 charges (tol 1e-5).

At full size the mixed-precision plan is compared with the FP64 plan (whose
parts match the oracle to rounding, checked below on scaled-down systems of
the same shape and density), and the FP64 forces must sum to zero.  Scaled
down to 2e4 charges, both plans are compared with the oracle."""
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


@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_full_size_mixed_matches_fp64(B, name):
    N, L, tol, kind = CONFIGS[name]
    q, r = _system(kind, N, L, 3)
    f64 = _run(B, N, L, tol, q, r, B.SOG_PREC_FP64)
    mix = _run(B, N, L, tol, q, r, B.SOG_PREC_MIXED)
    assert f64["st"] == 0 and mix["st"] == 0
    # FP32 path: in the slab the long range carries each charge's
    # self-interaction, 140 times the total energy, so FP32 rounding of that
    # part (about 2e-8) gives 3e-6 of the energy; bound 1e-5
    assert abs(mix["E"] - f64["E"]) <= 1e-5 * abs(f64["E"])
    assert _rms(mix["F"], f64["F"]) <= 1e-5
    # the net force vanishes up to the method's error: far below the sum of
    # N forces of random direction
    Fs = f64["F"]
    assert np.abs(Fs.sum(0)).max() <= 1e-3 * math.sqrt(N * np.mean(np.sum(Fs ** 2, 1)))


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
