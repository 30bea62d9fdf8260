"""The tile autotuner (sog_plan_autotune): after tuning, the evaluation still
matches the oracle, the chosen tiles are among the candidates, and the tuned
gridding + gathering stages are not slower than the default tiles'."""
import math

import numpy as np
import pytest

from paper_2412_04595_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SYSTEMS = {
    # gridded long range with several long tiles (no mid range)
    "slab": (20000, (141.4, 141.4, 10.0), 60),
    # mid grid and direct long range
    "cube": (20000, (58.5, 58.5, 58.5), 120),
}


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_2412_04595_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding


def _stage_ms(plan, qt, rt, stages, reps=5):
    plan.set_timing(2)
    out = []
    for _ in range(reps + 1):
        plan.eval(qt, rt)
        torch.cuda.synchronize()
        t = plan.timing()
        out.append(sum(t[k] for k in stages))
    plan.set_timing(0)
    return float(np.median(out[1:]))


@pytest.mark.parametrize("name", sorted(SYSTEMS))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotuned_plan_matches_oracle(B, oracle_mod, name, precision):
    N, L, nnb = SYSTEMS[name]
    q, r = workloads.uniform_neutral(N, L, 21)
    prm = oracle_mod.select_params(N, *L, 1e-6, n_nb=nnb)
    fp64 = precision == "fp64"
    if not fp64:
        r = r.astype(np.float32).astype(np.float64)
    dt = torch.float64 if fp64 else torch.float32
    plan = B.Plan(N, L, 1e-6, precision=B.SOG_PREC_FP64 if fp64 else B.SOG_PREC_MIXED,
                  manual=prm)
    dev = torch.device("cuda:0")
    qt = torch.tensor(q, dtype=dt, device=dev)
    rt = torch.tensor(r, dtype=dt, device=dev)
    before = plan.tiles()
    tiles = plan.autotune(qt, rt, reps=3)
    for k in ("mid_tile", "long_tile"):
        assert tiles[k] in (0, 8, 12, 16, 20, 23), tiles
    assert (tiles["mid_tile"] == 0) == (before["mid_tile"] == 0)
    phi = torch.empty(N, dtype=dt, device=dev)
    F = torch.empty(N, 3, dtype=dt, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    plan.eval(qt, rt, phi, E, F)
    torch.cuda.synchronize()
    assert plan.check() == 0
    ref = oracle_mod.sog_eval(prm, q, r)
    bound = 1e-10 if fp64 else 1e-5
    assert abs(E.item() - ref["E"]) <= bound * abs(ref["E"])
    Fr = ref["F"]
    Fg = F.double().cpu().numpy()
    assert math.sqrt(np.sum((Fg - Fr) ** 2) / np.sum(Fr ** 2)) <= bound
    plan.close()


def test_autotuned_stages_not_slower(B):
    N, L, nnb = 200000, (447.0, 447.0, 10.0), 60
    q, r = workloads.uniform_neutral(N, L, 22, dtype=np.float32)
    dev = torch.device("cuda:0")
    qt = torch.tensor(q, device=dev)
    rt = torch.tensor(r, device=dev)
    plan = B.Plan(N, L, 1e-6, precision=B.SOG_PREC_MIXED, n_nb=nnb)
    stages = [k for k in ("mid_spread", "mid_gather", "long_spread", "long_gather")]
    t0 = _stage_ms(plan, qt, rt, stages)
    tiles = plan.autotune(qt, rt, reps=3)
    t1 = _stage_ms(plan, qt, rt, stages)
    print("default %.3f ms, tuned %.3f ms, tiles %s" % (t0, t1, tiles))
    assert t1 <= 1.1 * t0
    plan.close()


def test_tune_cutoff_picks_the_fastest_feasible_candidate(B, oracle_mod):
    """sog_tune_cutoff (Sec. 4.3: the cutoff chosen by run time): the chosen
    neighbour count is a candidate with the least reported time, every
    candidate was timed, and a plan with the chosen cutoff still matches the
    oracle's evaluation with the same parameters (FP64 1e-10)."""
    N, L = 20000, (141.4, 141.4, 10.0)
    q, r = workloads.uniform_neutral(N, L, 23, dtype=np.float32)
    dev = torch.device("cuda:0")
    qt = torch.tensor(q, device=dev)
    rt = torch.tensor(r, device=dev)
    cands = (60.0, 120.0, 200.0)
    best, ms = B.sog_tune_cutoff(N, L, 1e-6, qt, rt, cands, reps=3)
    assert best in cands and all(ms[c] > 0 for c in cands)
    assert ms[best] == min(ms.values())
    q64, r64 = q.astype(np.float64), r.astype(np.float64)
    prm = oracle_mod.select_params(N, *L, 1e-6, n_nb=best)
    plan = B.Plan(N, L, 1e-6, precision=B.SOG_PREC_FP64, manual=prm)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    plan.eval(torch.tensor(q64, device=dev), torch.tensor(r64, device=dev), None, E, None)
    torch.cuda.synchronize()
    assert plan.check() == 0
    plan.close()
    ref = oracle_mod.sog_eval(prm, q64, r64)
    assert abs(E.item() - ref["E"]) <= 1e-10 * abs(ref["E"])
