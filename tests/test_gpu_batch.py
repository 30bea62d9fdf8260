"""Batches of independent systems (sog_batch_*) through the C ABI.

A batch must give, system by system, what one plan per system gives with the
same parameters, and (FP64) what the oracle gives.  Systems of the batched
workload: N log-uniform, density 0.1, aspect ratios Lz/Lx from thin slabs to
tall cells."""
import math

import numpy as np
import pytest

from paper_2412_04595_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_2412_04595_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding


def _tensors(systems, dt, dev):
    q = [torch.tensor(s[0], dtype=dt, device=dev) for s in systems]
    r = [torch.tensor(s[1], dtype=dt, device=dev) for s in systems]
    phi = [torch.empty(s[0].size, dtype=dt, device=dev) for s in systems]
    F = [torch.empty(s[0].size, 3, dtype=dt, device=dev) for s in systems]
    return q, r, phi, F


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_one_plan_per_system(B, precision):
    fp64 = precision == "fp64"
    dt = torch.float64 if fp64 else torch.float32
    prec = B.SOG_PREC_FP64 if fp64 else B.SOG_PREC_MIXED
    dev = torch.device("cuda:0")
    systems = workloads.batched_slabs(10, seed=3, nmin=300, nmax=4000)
    batch = B.Batch([(s[0].size, s[2]) for s in systems], 1e-6, precision=prec)
    q, r, phi, F = _tensors(systems, dt, dev)
    E = torch.zeros(len(systems), dtype=torch.float64, device=dev)
    for _ in range(2):  # second call replays the captured graph
        batch.eval(q, r, phi, E, F)
    st, bad = batch.check()
    assert st == 0, (st, bad)
    assert batch.launches() > 0
    tol = 1e-12 if fp64 else 2e-6
    for i, s in enumerate(systems):
        plan = B.Plan(s[0].size, s[2], 1e-6, precision=prec, manual=batch.params[i])
        phi1 = torch.empty_like(phi[i])
        F1 = torch.empty_like(F[i])
        E1 = torch.zeros(1, dtype=torch.float64, device=dev)
        plan.eval(q[i], r[i], phi1, E1, F1)
        torch.cuda.synchronize()
        assert plan.check() == 0
        plan.close()
        sc = phi1.abs().max().item()
        assert (phi[i] - phi1).abs().max().item() <= tol * sc, i
        assert (F[i] - F1).abs().max().item() <= 10 * tol * F1.abs().max().item(), i
        assert abs(E[i].item() - E1.item()) <= tol * abs(E1.item()), i
    batch.close()


def test_fp64_batch_matches_oracle(B, oracle_mod):
    dev = torch.device("cuda:0")
    systems = workloads.batched_slabs(4, seed=7, nmin=200, nmax=800)
    batch = B.Batch([(s[0].size, s[2]) for s in systems], 1e-6, precision=B.SOG_PREC_FP64)
    q, r, phi, F = _tensors(systems, torch.float64, dev)
    E = torch.zeros(len(systems), dtype=torch.float64, device=dev)
    batch.eval(q, r, phi, E, F)
    assert batch.check()[0] == 0
    for i, s in enumerate(systems):
        ref = oracle_mod.sog_eval(batch.params[i], s[0], s[1])
        assert abs(E[i].item() - ref["E"]) <= 1e-10 * abs(ref["E"]), i
        Fr = ref["F"]
        Fg = F[i].cpu().numpy()
        assert math.sqrt(np.mean(np.sum((Fg - Fr) ** 2, 1)) / np.mean(np.sum(Fr ** 2, 1))) <= 1e-10
    batch.close()


def test_batch_reports_the_failing_system(B):
    dev = torch.device("cuda:0")
    systems = workloads.batched_slabs(3, seed=11, nmin=200, nmax=400)
    batch = B.Batch([(s[0].size, s[2]) for s in systems], 1e-6)
    q, r, phi, F = _tensors(systems, torch.float32, dev)
    r[1][0, 2] = 10.0 * systems[1][2][2]  # z far outside the box of system 1
    batch.eval(q, r, phi, None, F)
    st, bad = batch.check()
    assert st == 3 and bad == 1  # SOG_ERR_OUT_OF_BOX
    batch.close()
